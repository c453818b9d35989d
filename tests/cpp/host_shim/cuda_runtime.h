// Host stand-in for the CUDA runtime header, for compiling the library's
// per-element device math as plain C++ in the CPU tests: only the device
// intrinsics that math uses, written with the host's libm.
#pragma once
#include <cmath>
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline float cbrtf(float x) { return std::cbrt(x); }
using std::cbrt;

// explicitly rounded single-precision operations (round to nearest even, as
// the host's SSE arithmetic does; build with -ffp-contract=off so that no
// product and sum is fused behind the code's back)
struct float2 { float x, y; };
struct int4 { int x, y, z, w; };
struct int2 { int x, y; };
struct uint2 { unsigned x, y; };
inline float2 make_float2(float x, float y) { return float2{x, y}; }
inline float __double2float_rn(double x) { return (float)x; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
using std::isfinite;

// declared only: warp, block and grid intrinsics have no host meaning, and
// the host builds call none of the functions that use them
#define __host__
#define __shared__ static
struct host_dim3 { unsigned x, y, z; };
extern host_dim3 threadIdx, blockIdx, blockDim, gridDim;
float __shfl_xor_sync(unsigned mask, float v, int lane_mask);
double __shfl_xor_sync(unsigned mask, double v, int lane_mask);
int __shfl_xor_sync(unsigned mask, int v, int lane_mask);
void __syncthreads();
void __threadfence();
unsigned atomicAdd(unsigned* p, unsigned v);
