// Internal accessors used by the allocation-free entry point.
#pragma once
#include "../../include/pd_b300.h"
#include "pd_internal.h"

#define PD_NOALLOC_MAX_FREE 65536

// device-side state of a context, its CUDA device and whether A is factored
void pd_internal_state(pd_ctx* c, const pdk::Dev** d, int* device, int* factored);
void pd_internal_set_error(pd_ctx* c, const char* msg);
