// lya_device.cuh -- device-side helpers shared by the library's kernels.
//
// Thin wrappers over documented PTX instructions (ex2/lg2/rcp .approx), the
// exact error-free transforms used for compensated sums, and a block-wide
// exclusive scan.  Nothing here reproduces a math-library routine: the
// transcendental work is the hardware MUFU instruction itself.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lya {

// 2^x on the MUFU unit (PTX ex2.approx.f32; subnormal results are kept).
__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2(x) on the MUFU unit (PTX lg2.approx.f32).
__device__ __forceinline__ float lg2(float x)
{
    float y;
    asm("lg2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x on the MUFU unit (PTX rcp.approx.f32).
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Kahan-compensated FP32 accumulator.  The adds are written with explicit
// round-to-nearest intrinsics so the compiler can neither contract nor
// reassociate them.
struct KahanF32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ float value() const { return __fsub_rn(s, c); }
};

// Inclusive warp scan of an int.
__device__ __forceinline__ int warp_inclusive_scan(int v)
{
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (unsigned)o) v += u;
    }
    return v;
}

// In-place exclusive scan of data[0..n) (ints in shared memory) by the
// whole block; returns the total on every thread.  warp_tot holds >= 32
// ints of shared scratch.  Contains __syncthreads(): call from all threads.
__device__ inline int block_exclusive_scan(int* data, int n, int* warp_tot)
{
    const int nt = blockDim.x;
    const int tid = threadIdx.x;
    const int per = (n + nt - 1) / nt;
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    int local = 0;
    for (int k = lo; k < hi; ++k) local += data[k];
    int inc = warp_inclusive_scan(local);
    const int warp = tid >> 5, lane = tid & 31, nwarps = (nt + 31) >> 5;
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nwarps ? warp_tot[lane] : 0;
        int wi = warp_inclusive_scan(w);
        if (lane < nwarps) warp_tot[lane] = wi - w;     // exclusive warp offsets
        if (lane == 31) warp_tot[32] = wi;              // total
    }
    __syncthreads();
    int run = warp_tot[warp] + inc - local;
    for (int k = lo; k < hi; ++k) {
        int c = data[k];
        data[k] = run;
        run += c;
    }
    int total = warp_tot[32];
    __syncthreads();
    return total;
}

}  // namespace lya
