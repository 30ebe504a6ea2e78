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

// 2^x on the MUFU unit (PTX ex2.approx.ftz.f32).  Results below 2^-126
// flush to zero: a line-profile term that small is ~1e-38 of its line's
// weight, and a transmitted flux that small is 0 to any tolerance used here.
__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x rounded to the nearest integer (ties to even), as a float and as an int,
// for |x| < 2^22: adding 1.5 * 2^23 leaves that integer in the low bits of
// the sum (its ulp is 1), all on the FMA and integer pipes (rintf and the
// float-to-int conversion would use the quarter-rate conversion unit).
__device__ __forceinline__ float round_to_int(float x, int& n)
{
    constexpr float kShift = 0x1.8p23f;
    const float s = __fadd_rn(x, kShift);
    n = __float_as_int(s) - __float_as_int(kShift);
    return __fsub_rn(s, kShift);
}

// log2(x) on the MUFU unit (PTX lg2.approx.ftz.f32; x is a normal positive
// temperature or density here).
__device__ __forceinline__ float lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x on the MUFU unit (PTX rcp.approx.ftz.f32).
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Bulk prefetch of bytes (a multiple of 16) at a 16-byte aligned global
// address into L2 (PTX cp.async.bulk.prefetch.L2): no registers, no shared
// memory, no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---- 1D bulk copies (the TMA engine) into shared memory --------------------------
// cp.async.bulk moves a contiguous run of global memory into this CTA's shared
// memory; an mbarrier counts the bytes that have landed (complete_tx).  Both
// addresses must be 16-byte aligned and the size a multiple of 16.
__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Waits for the phase of parity `parity` of bar to complete; gives up after
// `spins` polls (each poll may suspend the thread for a while) and returns
// false, so a copy that never lands cannot hang the kernel.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned spins)
{
    for (unsigned k = 0; k < spins; ++k) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
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

// A run of consecutive warps of the block that works on one skewer: threads
// [base, base + nt) with nt a multiple of 32 and base a multiple of 32, so
// lane numbers match the hardware's.  The whole block is the group with
// barrier 0 (__syncthreads); smaller groups synchronise on their own named
// barrier (PTX bar.sync id, nt).
struct Group {
    int tid;     // thread index within the group
    int nt;      // threads in the group
    int bar;     // 0: whole block; 1..15: named barrier of this group
    __device__ __forceinline__ void sync() const
    {
        if (bar == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
    }
};

__device__ __forceinline__ Group whole_block() { return Group{(int)threadIdx.x, (int)blockDim.x, 0}; }

// Each thread of a scan owns a contiguous chunk of the array.  The chunk
// length is odd, so the 32 lanes of a warp, one chunk apart, fall in 32
// different shared-memory banks.
__device__ __forceinline__ int scan_chunk(int n, int nt) { return ((n + nt - 1) / nt) | 1; }

// In-place exclusive scan of data[0..n) (ints in shared memory) by the
// group; returns the total on every thread.  warp_tot holds >= 33 ints of
// shared scratch private to the group.  Synchronises the group: call from
// all of its threads.  With marks (indices into data, -1 for none) and
// mark_out, the scanned values at those indices are also left in
// mark_out[0], mark_out[1] by the time the scan returns.
__device__ inline int block_exclusive_scan(int* data, int n, int* warp_tot, const Group& g,
                                           int mark_a = -1, int mark_b = -1, int* mark_out = nullptr)
{
    const int nt = g.nt;
    const int tid = g.tid;
    const int per = scan_chunk(n, nt);
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    int local = 0;
    for (int k = lo; k < hi; ++k) local += data[k];
    int inc = warp_inclusive_scan(local);
    const int warp = tid >> 5, lane = tid & 31, nwarps = (nt + 31) >> 5;
    if (lane == 31) warp_tot[warp] = inc;
    g.sync();
    if (warp == 0) {
        int w = lane < nwarps ? warp_tot[lane] : 0;
        int wi = warp_inclusive_scan(w);
        if (lane < nwarps) warp_tot[lane] = wi - w;     // exclusive warp offsets
        if (lane == 31) warp_tot[32] = wi;              // total
    }
    g.sync();
    int run = warp_tot[warp] + inc - local;
    for (int k = lo; k < hi; ++k) {
        int c = data[k];
        data[k] = run;
        run += c;
    }
    if (mark_out) {
        if (mark_a >= lo && mark_a < hi) mark_out[0] = data[mark_a];
        if (mark_b >= lo && mark_b < hi) mark_out[1] = data[mark_b];
    }
    int total = warp_tot[32];
    g.sync();
    return total;
}

__device__ inline int block_exclusive_scan(int* data, int n, int* warp_tot)
{
    return block_exclusive_scan(data, n, warp_tot, whole_block());
}

// Inclusive warp scan with max (ascending lanes) or min (descending lanes).
__device__ __forceinline__ int warp_scan_max(int v)
{
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (unsigned)o) v = max(v, u);
    }
    return v;
}
__device__ __forceinline__ int warp_suffix_min(int v)
{
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_down_sync(0xffffffffu, v, o);
        if (lane + (unsigned)o < 32u) v = min(v, u);
    }
    return v;
}

// In-place inclusive prefix max of data[0..n) by the group.
// warp_tmp holds >= 32 ints of the group's shared scratch.  Ends with a
// group barrier.
__device__ inline void block_prefix_max(int* data, int n, int* warp_tmp, int lowest, const Group& g)
{
    const int nt = g.nt, tid = g.tid;
    const int per = scan_chunk(n, nt);
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    int local = lowest;
    for (int k = lo; k < hi; ++k) local = max(local, data[k]);
    const int warp = tid >> 5, lane = tid & 31, nwarps = (nt + 31) >> 5;
    int inc = warp_scan_max(local);
    if (lane == 31) warp_tmp[warp] = inc;
    g.sync();
    if (warp == 0) {
        int w = lane < nwarps ? warp_tmp[lane] : lowest;
        int wi = warp_scan_max(w);
        int ex = __shfl_up_sync(0xffffffffu, wi, 1);
        if (lane < nwarps) warp_tmp[lane] = lane ? ex : lowest;   // max over earlier warps
    }
    g.sync();
    int ex_thread = __shfl_up_sync(0xffffffffu, inc, 1);
    int run = max(warp_tmp[warp], lane ? ex_thread : lowest);
    for (int k = lo; k < hi; ++k) {
        run = max(run, data[k]);
        data[k] = run;
    }
    g.sync();
}

// In-place inclusive suffix min of data[0..n) (data[k] = min data[k..n)) by
// the group.  Ends with a group barrier.
__device__ inline void block_suffix_min(int* data, int n, int* warp_tmp, int highest, const Group& g)
{
    const int nt = g.nt, tid = g.tid;
    const int per = scan_chunk(n, nt);
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    int local = highest;
    for (int k = lo; k < hi; ++k) local = min(local, data[k]);
    const int warp = tid >> 5, lane = tid & 31, nwarps = (nt + 31) >> 5;
    int inc = warp_suffix_min(local);                 // min over this and later lanes
    if (lane == 0) warp_tmp[warp] = inc;
    g.sync();
    if (warp == 0) {
        int w = lane < nwarps ? warp_tmp[lane] : highest;
        int wi = warp_suffix_min(w);
        int ex = __shfl_down_sync(0xffffffffu, wi, 1);
        if (lane < nwarps) warp_tmp[lane] = (lane + 1 < nwarps) ? ex : highest;   // min over later warps
    }
    g.sync();
    int ex_thread = __shfl_down_sync(0xffffffffu, inc, 1);
    int run = min(warp_tmp[warp], lane < 31 ? ex_thread : highest);
    for (int k = hi - 1; k >= lo; --k) {
        run = min(run, data[k]);
        data[k] = run;
    }
    g.sync();
}

}  // namespace lya
