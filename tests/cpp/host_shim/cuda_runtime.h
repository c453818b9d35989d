// Host stand-in for the CUDA runtime header, for compiling the library's
// per-element device math as plain C++ in the CPU tests: only the device
// intrinsics that math uses, written with the host's libm.
#pragma once
#include <cmath>
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
