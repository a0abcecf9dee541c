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
struct float4 { float x, y, z, w; };
inline float2 make_float2(float a, float b) { return {a, b}; }
// The packed two-lane FP32 operations: each lane rounds as the scalar operation.
inline float2 __fadd2_rn(float2 a, float2 b) { return {a.x + b.x, a.y + b.y}; }
inline float2 __fmul2_rn(float2 a, float2 b) { return {a.x * b.x, a.y * b.y}; }
inline float2 __ffma2_rn(float2 a, float2 b, float2 c) { return {std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)}; }
typedef int cudaError_t;
typedef void* cudaStream_t;
using std::fma;
