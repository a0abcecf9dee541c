// Host stand-in for <cuda_runtime.h>, used only by tests/host_fft/check_fft.cpp
// to compile the device FFT core (csrc/sfac_fft.cuh) with a host C++ compiler.
#pragma once
#include <cmath>
#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
struct double2 { double x, y; };
struct float2 { float x, y; };
inline float2 make_float2(float a, float b) { return {a, b}; }
typedef int cudaError_t;
typedef void* cudaStream_t;
using std::fma;
