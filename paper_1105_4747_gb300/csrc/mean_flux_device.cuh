// mean_flux_device.cuh -- device pieces of the mean-flux root-find (Sec. 2.3)
// shared by the single-request kernels (mean_flux.cu) and the batched serving
// kernels (serve_kernels.cu): the per-pixel exponential, block reductions,
// the root-find state and the steps taken on the reduced sums.
#pragma once

#include <cmath>
#include <cstdint>

#include "lya_device.cuh"
#include "lya_internal.h"

namespace lya {
namespace mfd {

constexpr int kThreads = 256;
constexpr double kLog2e = 1.4426950408889634;
constexpr float kLn2f = 0.69314718055994531f;

// Streams x[0..n) through f(index, value), thread tid of nthr.  When x is
// 16-byte aligned each thread keeps eight float4 loads in flight per step (the
// bytes in flight, not the instruction count, bound these HBM passes); the
// last n % 4 values and unaligned inputs take the scalar path.
template <typename Fn>
__device__ __forceinline__ void stream_f32(const float* __restrict__ x, long long n, long long tid,
                                           long long nthr, Fn&& f)
{
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        const float4* __restrict__ x4 = reinterpret_cast<const float4*>(x);
        const long long n4 = n >> 2;
        long long i = tid;
        for (; i + 7 * nthr < n4; i += 8 * nthr) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = x4[i + u * nthr];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const long long b = 4 * (i + u * nthr);
                f(b, v[u].x); f(b + 1, v[u].y); f(b + 2, v[u].z); f(b + 3, v[u].w);
            }
        }
        for (; i < n4; i += nthr) {
            const float4 v = x4[i];
            f(4 * i, v.x); f(4 * i + 1, v.y); f(4 * i + 2, v.z); f(4 * i + 3, v.w);
        }
        for (long long k = 4 * n4 + tid; k < n; k += nthr) f(k, x[k]);
    } else {
        for (long long k = tid; k < n; k += nthr) f(k, x[k]);
    }
}

// The same over the whole grid.
template <typename Fn>
__device__ __forceinline__ void stream_f32(const float* __restrict__ x, long long n, Fn&& f)
{
    stream_f32(x, n, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x, f);
}

// Quarter-octave histogram of log2(tau) over [2^-64, 2^64), built in the
// init pass; its bin centres give a cheap proxy of g(A) whose root starts
// the exact iteration close to the answer.
constexpr int kHistBins = 512;
constexpr float kHistPerOctave = 4.f;

struct MFState {
    double A, lo, hi, g, mean_tau, Ft, tol;
    long long n, n_zero, n_bad;
    int iter, max_iter, done, status;   // status: LYA_OK / LYA_EINVAL / LYA_ENOCONV (not yet converged)
    unsigned int ticket;
    unsigned long long hist[kHistBins + 1];   // + sampled zeros
};

struct Partial {
    double s0, s0c, s1, s2;
    long long z, bad;
};

// One CTA's share of the flux statistics: sums of (F - 1/2), (F - 1/2)^2 and
// the 21 PDF bin counts.
struct StatPart {
    double m1, m2;
    unsigned int pdf[21];
    unsigned int pad;
};

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of a few values; result valid on thread 0.
template <int K>
__device__ inline void block_sum(double (&v)[K], double (*sh)[32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = warp_sum_d(v[k]);
        if (lane == 0) sh[k][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double x = lane < nw ? sh[k][lane] : 0.0;
            v[k] = warp_sum_d(x);
        }
    }
    __syncthreads();
}

// Block sum of a few floats; result valid on every thread.
template <int K>
__device__ inline void block_sum_f(float (&v)[K], float (*sh)[32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][warp] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float x = 0.f;
        for (int w = 0; w < nw; ++w) x += sh[k][w];
        v[k] = x;
    }
    __syncthreads();
}

// The last block's totals of the per-CTA partials, summed by all its threads
// (GB300's FP64 latency makes a one-thread loop over ~1,200 partials slow).
template <int K, typename Get>
__device__ inline void partial_totals(const Partial* part, int nb, double (&tot)[K], double (*sh)[32], Get get)
{
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double x[K];
        get(part[b], x);
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] += x[k];
    }
    block_sum<K>(tot, sh);
}

// Returns true on exactly one of `count` arrivals at *ticket (one per block,
// after the block's partial is written): the last.  No waiting.
__device__ inline bool last_arrival(unsigned int* ticket, unsigned int count)
{
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == count - 1);
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// The last block of the grid to arrive.
__device__ inline bool last_block(unsigned int* ticket) { return last_arrival(ticket, gridDim.x); }

__device__ __forceinline__ int hist_bin(float t)
{
    const int b = (int)floorf((lg2(t) + 64.f) * kHistPerOctave);
    return min(max(b, 0), kHistBins - 1);
}

// Double-float split of a = A log2(e).
__device__ __forceinline__ void split_rate(double A, float& a_hi, float& a_lo)
{
    const double a = A * kLog2e;
    a_hi = (float)a;
    a_lo = (float)(a - (double)a_hi);
}

// e = 2^-(t a) as (main, correction) with t a = y_hi + y_lo exactly to ~2^-48.
__device__ __forceinline__ void exp_neg(float t, float a_hi, float a_lo, float& e, float& corr)
{
    const float y_hi = t * a_hi;
    const float y_lo = fmaf(t, a_lo, fmaf(t, a_hi, -y_hi));
    e = ex2(-y_hi);
    corr = -e * y_lo * kLn2f;
}

// Sec. 5.2 bin: k with (2k-1)/40 <= F < (2k+1)/40, clamped to [0, 20].  The
// guess floor(20 F + 1/2) is off by at most one; fma(F, 40, -(2k +- 1)) is
// the exact difference rounded once, so its sign decides the edge exactly.
__device__ __forceinline__ int pdf_bin(float F)
{
    if (!(F == F)) return 0;
    const float f = fminf(fmaxf(F, -1.f), 2.f);
    int k = (int)floorf(fmaf(f, 20.f, 0.5f));
    if (fmaf(f, 40.f, -(float)(2 * k - 1)) < 0.f) k -= 1;
    else if (fmaf(f, 40.f, -(float)(2 * k + 1)) >= 0.f) k += 1;
    return min(max(k, 0), 20);
}


// ---- start value from the init pass's log-histogram (whole block) -------------
// Newton on the proxy g_h(A) = (z + sum_b n_b e^{-A tau_b})/n_s - F_t over the
// sample (n_s values, z of them zero), tau_b the bin's geometric centre;
// convex and decreasing like g.  FP32 is plenty for a start value.  Replaces
// st->A (the Jensen bound) when the proxy's root is credible.
__device__ inline void proxy_start(MFState* st)
{
    __shared__ float s_A;
    __shared__ int s_stop;
    if (threadIdx.x == 0) {
        s_A = (float)st->A;
        s_stop = 0;
    }
    __syncthreads();
    __shared__ float shf[2][32];
    float cnt[1] = {0.f};
    for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x) cnt[0] += (float)st->hist[b];
    block_sum_f<1>(cnt, shf);
    const float inv_n = 1.f / cnt[0], Ft = (float)st->Ft;
    const float fz = (float)st->hist[kHistBins] * inv_n;
    if (!(fz < Ft)) return;                 // the sample's proxy has no root: keep the Jensen start
    const float A_jensen = s_A;
    float lo = s_A, hi = INFINITY;
    for (int it = 0; it < 60; ++it) {
        const float A = s_A;
        float v2[2] = {0.f, 0.f};
        for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) {
            const float c = (float)st->hist[b];
            if (c == 0.f) continue;
            const float tb = ex2(((float)b + 0.5f) / kHistPerOctave - 64.f);
            const float e = ex2(-A * tb * 1.44269504f);
            v2[0] += c * e;
            v2[1] += c * tb * e;
        }
        block_sum_f<2>(v2, shf);
        if (threadIdx.x == 0) {
            const float g = fz + v2[0] * inv_n - Ft, gp = -v2[1] * inv_n;
            if (g > 0.f) lo = A; else hi = A;
            float An = gp < 0.f ? A - g / gp : NAN;
            if (!isfinite(An) || An <= lo || An >= hi) An = isfinite(hi) ? 0.5f * (lo + hi) : 2.f * lo;
            s_stop = fabsf(An - A) <= 1e-6f * A;
            s_A = An;
        }
        __syncthreads();
        if (s_stop) break;
    }
    // a proxy root far from the Jensen bound means an unrepresentative sample
    if (threadIdx.x == 0 && s_stop && isfinite(s_A) && s_A >= A_jensen && s_A < 1e4f * A_jensen)
        st->A = (double)s_A;
}

// ---- the steps on the reduced sums (one thread) --------------------------------

// After the init pass: record <tau> and the zero/invalid counts; fail on an
// invalid value or when no A can reach F_t (the zero-tau pixels alone give
// <F> >= F_t); else start from the Jensen bound A0 = -ln(F_t)/<tau>, which is
// below the root.  Returns true when the iteration goes on.
__device__ inline bool init_finish(MFState* st, double sum_tau, long long zeros, long long bad)
{
    const long long n = st->n;
    st->ticket = 0;
    st->n_zero = zeros;
    st->n_bad = bad;
    st->mean_tau = sum_tau / (double)n;
    st->iter = 0;
    if (bad > 0 || !(st->mean_tau > 0.0)) {
        st->status = LYA_EINVAL;
        st->done = 1;
        return false;
    }
    if ((double)zeros / (double)n >= st->Ft) {       // <e^{-A tau}> >= zero fraction for all A
        st->status = LYA_ENOCONV;
        st->done = 1;
        return false;
    }
    st->A = -log(st->Ft) / st->mean_tau;
    st->lo = st->A;
    st->hi = INFINITY;
    st->status = LYA_ENOCONV;                         // until converged
    st->done = 0;
    return true;
}

// One safeguarded step from the sums S0 + S0c = sum e, S1 = sum tau e,
// S2 = sum tau^2 e at the current A: Halley's step, else Newton's, else
// bisection, whichever stays inside the bracket [lo, hi].
__device__ inline void halley_update(MFState* st, double S0, double S0c, double S1, double S2)
{
    st->ticket = 0;
    const double nn = (double)st->n;
    const double g = (S0 + S0c) / nn - st->Ft;
    const double g1 = -S1 / nn, g2 = S2 / nn;
    const double A = st->A;
    st->g = g;
    st->iter += 1;
    if (fabs(g) <= st->tol) {
        st->status = LYA_OK;
        st->done = 1;
        return;
    }
    if (g > 0.0) st->lo = A; else st->hi = A;
    const double den = 2.0 * g1 * g1 - g * g2;
    double An = den > 0.0 ? A - 2.0 * g * g1 / den : NAN;
    if (!isfinite(An) || An <= st->lo || An >= st->hi) An = g1 < 0.0 ? A - g / g1 : NAN;
    if (!isfinite(An) || An <= st->lo || An >= st->hi)
        An = isfinite(st->hi) ? 0.5 * (st->lo + st->hi) : 2.0 * st->lo;
    if (fabs(An - A) <= 4.0e-16 * fabs(A)) {        // stalled at FP64 resolution
        st->status = LYA_OK;
        st->done = 1;
        return;
    }
    st->A = An;
    if (st->iter >= st->max_iter) {
        st->status = LYA_ENOCONV;
        st->done = 1;
    }
}

// The check of the flux pass: the F just written is final when |g| <= tol at
// this A (or the iteration had already stopped at FP64 resolution).
__device__ inline void flux_update(MFState* st, double S0, double S0c)
{
    st->ticket = 0;
    const double g = (S0 + S0c) / (double)st->n - st->Ft;
    st->g = g;
    if (fabs(g) <= st->tol || (st->done && st->status == LYA_OK)) {
        st->status = LYA_OK;
        st->done = 1;
    } else {
        st->status = LYA_ENOCONV;                     // more passes needed
        st->done = 0;
    }
}

}  // namespace mfd
}  // namespace lya
