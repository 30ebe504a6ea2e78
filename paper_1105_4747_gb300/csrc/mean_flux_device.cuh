// mean_flux_device.cuh -- device pieces of the mean-flux root-find (Sec. 2.3)
// shared by the single-request kernels (mean_flux.cu) and the batched serving
// kernels (serve_kernels.cu): the per-pixel exponential, block reductions,
// the root-find state and the steps taken on the reduced sums.
#pragma once

#include <cmath>
#include <cstdint>

#include "exp2_table.h"
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

// stream_f32 with done() called after every step of at most 32 values per
// thread (the per-thread FP32 or float-pair sums move into FP64 there).
template <typename Fn, typename Done>
__device__ __forceinline__ void stream_f32_steps(const float* __restrict__ x, long long n, long long tid,
                                                 long long nthr, Fn&& f, Done&& done)
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
                f(v[u].x); f(v[u].y); f(v[u].z); f(v[u].w);
            }
            done();
        }
        for (; i < n4; i += nthr) {
            const float4 v = x4[i];
            f(v.x); f(v.y); f(v.z); f(v.w);
            done();
        }
        for (long long k = 4 * n4 + tid; k < n; k += nthr) f(x[k]);
    } else {
        int c = 0;
        for (long long k = tid; k < n; k += nthr) {
            f(x[k]);
            if (++c == 32) {
                done();
                c = 0;
            }
        }
    }
    done();
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
    unsigned int tau_max_bits;          // largest tau (float bits; tau >= 0 orders like its bits)
    int flux_ok;                        // the precise pass's F is the final F (no flux pass needed)
    int flux_pad;
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

// ---- precise passes: e = 2^-y to ~3e-14 on the FP32 pipe -------------------------
// GB300 runs FP64 at a small fraction of its FP32 rate, so a per-pixel FP64
// exponential would cost milliseconds per pass over 2.7e8 pixels; instead the
// exponential is formed in double-float arithmetic (pairs of floats) from the
// split y = t (a_hi + a_lo) = y_hi + y_lo (exact to ~2^-48 y):
//   y_hi = N/1024 + r,  N = rint(1024 y_hi),  |r| <= 2^-11 (r exact),
//   2^-y = 2^-(N >> 10) * 2^(-(N & 1023)/1024) * exp(u),  u = -(r + y_lo) ln 2,
// the middle factor a double-float from kExp2Tab (in shared memory), exp(u) =
// 1 + u + u^2/2 + u^3/6 with |u| <= 3.4e-4 (the next term is below 6e-16),
// u itself a double-float (ln 2 split into two floats).  Result: e_hi + e_lo,
// within ~3e-14 absolute for every y (what the mean of e needs): near e = 1
// the float pair's last rounding (~2^-46) sets it; at large y the relative
// error grows as ~1.5e-15 y^2 (the series omits the higher terms of u_lo ~
// y_lo ln 2) on values that shrink as 2^-y.
constexpr float kLn2Hi = 0x1.62e430p-1f;                 // float nearest ln 2

constexpr float kLn2Lo = -0x1.05c610p-29f;               // ln 2 - kLn2Hi, to float

// Copies kExp2Tab into shared memory (whole block; ends with a barrier).
__device__ __forceinline__ void load_exp2_table(float2* tab)
{
    for (int k = threadIdx.x; k < kExp2TabSize; k += blockDim.x) tab[k] = kExp2Tab[k];
    __syncthreads();
}

// (y is clamped at 100, where e < 1e-30 and its value no longer matters.)
__device__ __forceinline__ void exp2_neg_precise(float t, float a_hi, float a_lo, const float2* __restrict__ tab,
                                                 float& e_hi, float& e_lo)
{
    const float y_raw = t * a_hi;
    const float y_hi = fminf(y_raw, 100.f);
    const float y_lo = y_raw <= 100.f ? fmaf(t, a_lo, fmaf(t, a_hi, -y_hi)) : 0.f;
    int N;
    const float Nf = round_to_int(y_hi * 1024.f, N);
    const float r = fmaf(Nf, -1.f / 1024.f, y_hi);                     // exact
    const float u_hi = -r * kLn2Hi;
    const float u_lo = fmaf(-r, kLn2Hi, -u_hi) - fmaf(r, kLn2Lo, y_lo * kLn2Hi);
    // exp(u) - 1 = u_hi + d_lo, d_lo = u_lo + u_hi u_lo + u_hi^2/2 + u_hi^3/6
    const float d_lo = fmaf(u_hi, fmaf(u_hi, fmaf(u_hi, 1.f / 6.f, 0.5f), u_lo), u_lo);
    const float2 T = tab[N & (kExp2TabSize - 1)];
    // T (1 + u_hi + d_lo) with the product T.x u_hi exact (two-product)
    const float P = T.x * u_hi;
    const float Pe = fmaf(T.x, u_hi, -P);
    const float R_hi = T.x + P;
    float R_lo = (T.x - R_hi) + P;                                      // |T.x| > |P|: exact
    R_lo += Pe + fmaf(T.x, d_lo, fmaf(T.y, u_hi, T.y));
    const float scale = __int_as_float((127 - (N >> 10)) << 23);        // 2^-(N >> 10), exact
    e_hi = R_hi * scale;
    e_lo = R_lo * scale;
}

// e = 2^-y for the fast pass on the FMA pipe: y = n + r with n the nearest
// integer (round_to_int), 2^-y = 2^-n 2^f with f = (n - y_hi) - y_lo in
// [-1/2, 1/2] (up to y_lo), 2^f by a degree-6 polynomial fitted by least
// squares on Chebyshev nodes (exp2_poly_fit.py beside this file, degree 6):
// within ~8e-8 of 2^f in FP32 and ~1e-9 on average over f, where the MUFU
// ex2 errs by a few ulp the same way for neighbouring arguments.  y is
// clamped at 100 like exp2_neg_precise.
__device__ __forceinline__ float exp2_neg_fast(float t, float a_hi, float a_lo)
{
    const float y_raw = t * a_hi;
    const float y_hi = fminf(y_raw, 100.f);
    const float y_lo = y_raw <= 100.f ? fmaf(t, a_lo, fmaf(t, a_hi, -y_hi)) : 0.f;
    int n;
    const float nf = round_to_int(y_hi, n);
    const float f = (nf - y_hi) - y_lo;
    float p = 0x1.446c7ep-13f;
    p = fmaf(p, f, 0x1.5f48c8p-10f);
    p = fmaf(p, f, 0x1.3b29d8p-7f);
    p = fmaf(p, f, 0x1.c6aeccp-5f);
    p = fmaf(p, f, 0x1.ebfbe0p-3f);
    p = fmaf(p, f, 0x1.62e430p-1f);
    p = fmaf(p, f, 0x1p+0f);
    return p * __int_as_float((127 - n) << 23);                         // 2^-n, n <= 100: exact
}

// Per-thread sum of e_hi + e_lo values: a float pair (h, l) with |l| <=
// ulp(h)/2 after every addition (an exact two-sum, then the pair
// renormalised), so each addition errs by at most ~2^-48 of the pair's value;
// flush() moves the pair into an FP64 total after every stream step of at
// most 32 values, which bounds the pair's relative error by 32 * 2^-48 ~ 1e-13.
struct DFSum {
    double acc = 0.0;
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void add(float eh, float el)
    {
        const float s = __fadd_rn(h, eh);
        const float bp = __fsub_rn(s, h);
        const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(eh, bp));
        const float t = __fadd_rn(l, __fadd_rn(err, el));
        h = __fadd_rn(s, t);                          // renormalise: h + l = s + t exactly
        l = __fsub_rn(t, __fsub_rn(h, s));
    }
    __device__ __forceinline__ void flush()
    {
        acc += (double)h + (double)l;
        h = 0.f;
        l = 0.f;
    }
    __device__ __forceinline__ double value() const { return acc + ((double)h + (double)l); }
};

// Sec. 5.2 bin: k with (2k-1)/40 <= F < (2k+1)/40, clamped to [0, 20].  The
// guess floor(20 F + 1/2) is off by at most one; fma(F, 40, -(2k +- 1)) is
// the exact difference rounded once, so its sign decides the edge exactly.
__device__ __forceinline__ int pdf_bin(float F)
{
    if (!(F == F)) return 0;
    const float f = fminf(fmaxf(F, -1.f), 2.f);
    int k;
    const float kf = round_to_int(20.f * f, k);          // the nearest bin, or a neighbour of it
    if (fmaf(f, 40.f, -fmaf(2.f, kf, -1.f)) < 0.f) k -= 1;
    else if (fmaf(f, 40.f, -fmaf(2.f, kf, 1.f)) >= 0.f) k += 1;
    return min(max(k, 0), 20);
}

// pdf_bin for F in [0, 1] (a flux the root-find just formed): the bin is the
// nearest integer to 20 F, decided exactly by pdf_bin only when 20 F (one
// rounding, <= 2^-20 off) lies within 2^-18 of a bin edge k + 1/2.
__device__ __forceinline__ int pdf_bin_unit(float F)
{
    const float p = 20.f * F;
    int k;
    const float kf = round_to_int(p, k);
    if (fabsf(p - kf) >= 0.5f - 0x1p-18f) k = pdf_bin(F);
    return k;
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
// The iteration's state and steps are shared by the device passes (the
// single-request and batched root-finds) and the host driver of a root-find
// whose pixels are split over several devices (lya_mean_flux_step).

// Bound on the error of g(A) from an FP32 (MUFU) pass: its steps move A but
// never tighten the bracket with a sign that close to the root, and never end
// the iteration; only a precise pass (g to ~1e-13) decides convergence.
constexpr double kApproxGErr = 1e-6;
// Bounds used by the precise pass's certificate: on the error of its g
// (double-float exponentials, ~3e-14 per term at worst; float-pair partial
// sums of at most 32 terms, ~1e-13 relative at worst; FP64 beyond) and on
// the relative error of its g' (FP32 products and sums of at most 32
// nonnegative terms, ~2e-6 at worst, or compensated FP32; FP64 beyond).
constexpr double kPreciseGErr = 2e-13;
constexpr double kSlopeRelErr = 1e-5;

__host__ __device__ inline bool finite_d(double x) { return x == x && x - x == 0.0; }

// The iteration: A in the bracket [lo, hi], the last g (or, once a step is
// certified, the bound on |g| at the final A), passes taken, and whether it
// has ended (status LYA_OK, or an error).
struct MFIter {
    double A, lo, hi, g;
    int iter, max_iter, done, status;
};

// The start from the totals over all pixels: <tau> and the zero/invalid
// counts; fail on an invalid value or when no A can reach F_t (the zero-tau
// pixels alone give <F> >= F_t); else Newton's start A0 = -ln(F_t)/<tau>, the
// Jensen bound, which lies below the root.  Returns true when the iteration
// goes on.
__host__ __device__ inline bool mf_start(MFIter& it, double Ft, double n, double sum_tau, double zeros, double bad)
{
    const double mean_tau = sum_tau / n;
    it.iter = 0;
    it.g = 0.0;
    if (bad > 0.0 || !(mean_tau > 0.0)) {
        it.status = LYA_EINVAL;
        it.done = 1;
        return false;
    }
    if (zeros / n >= Ft) {                            // <e^{-A tau}> >= zero fraction for all A
        it.status = LYA_ENOCONV;
        it.done = 1;
        return false;
    }
    it.A = -log(Ft) / mean_tau;
    it.lo = it.A;
    it.hi = INFINITY;
    it.status = LYA_ENOCONV;                          // until converged
    it.done = 0;
    return true;
}

// One safeguarded step from the means at the current A of e (g = <e> - F_t),
// tau e (g' = -<tau e>) and tau^2 e (g'' = <tau^2 e>): Halley's step, else
// Newton's, else bisection, whichever stays inside the bracket [lo, hi].
// precise: g comes from a precise pass (else the FP32 approximation).
//
// A precise step ends the iteration when |g| <= tol at A, or when it can
// certify its Newton step: with dA = -g/g', Taylor's theorem gives
//   g(A + dA) = g''(xi) dA^2 / 2,  xi between A and A + dA,
// and g''(x) = <tau^2 e^{-x tau}> is decreasing, so g''(xi) <= g''(A) when
// dA > 0 and g''(xi) <= g''(A) e^{|dA| tau_max} when dA < 0; hence
//   |g(A + dA)| <= g''(A) dA^2 f / 2 + kPreciseGErr + |g| kSlopeRelErr
// (f = 1 or e^{|dA| tau_max}; the last two terms the errors of g and g'),
// and a bound <= tol makes A + dA final without evaluating g there again.
// tau_max = INFINITY when unknown (then only steps with dA > 0 certify).
__host__ __device__ inline void mf_step(MFIter& it, double g, double g1, double g2, double tol, double tau_max,
                                        bool precise)
{
    const double A = it.A;
    it.g = g;
    it.iter += 1;
    if (precise && fabs(g) <= tol) {
        it.status = LYA_OK;
        it.done = 1;
        return;
    }
    if (precise || fabs(g) > kApproxGErr) {
        if (g > 0.0) it.lo = A; else it.hi = A;
    }
    if (precise && g1 < 0.0) {
        const double dA = -g / g1;
        const double An = A + dA;
        const double f = dA >= 0.0 ? 1.0 : exp(-dA * tau_max);
        const double bound = 0.5 * g2 * dA * dA * f + kPreciseGErr + fabs(g) * kSlopeRelErr;
        if (An > it.lo && An < it.hi && bound <= tol) {
            it.A = An;
            it.g = bound;                             // the certified bound on |g| at the final A
            it.status = LYA_OK;
            it.done = 1;
            return;
        }
    }
    const double den = 2.0 * g1 * g1 - g * g2;
    double An = den > 0.0 ? A - 2.0 * g * g1 / den : NAN;
    if (!finite_d(An) || An <= it.lo || An >= it.hi) An = g1 < 0.0 ? A - g / g1 : NAN;
    if (!finite_d(An) || An <= it.lo || An >= it.hi) An = finite_d(it.hi) ? 0.5 * (it.lo + it.hi) : 2.0 * it.lo;
    if (fabs(An - A) <= 4.0e-16 * fabs(A)) {          // stalled at FP64 resolution
        if (precise) {
            it.status = LYA_OK;
            it.done = 1;
        }
        return;
    }
    it.A = An;
    if (it.iter >= it.max_iter) {
        it.status = LYA_ENOCONV;
        it.done = 1;
    }
}

__device__ inline MFIter iter_of(const MFState* st)
{
    return MFIter{st->A, st->lo, st->hi, st->g, st->iter, st->max_iter, st->done, st->status};
}
__device__ inline void set_iter(MFState* st, const MFIter& it)
{
    st->A = it.A;
    st->lo = it.lo;
    st->hi = it.hi;
    st->g = it.g;
    st->iter = it.iter;
    st->max_iter = it.max_iter;
    st->done = it.done;
    st->status = it.status;
}

// After the init pass (device): record <tau> and the counts, and start.
__device__ inline bool init_finish(MFState* st, double sum_tau, long long zeros, long long bad)
{
    st->ticket = 0;
    st->n_zero = zeros;
    st->n_bad = bad;
    st->mean_tau = sum_tau / (double)st->n;
    MFIter it = iter_of(st);
    const bool go = mf_start(it, st->Ft, (double)st->n, sum_tau, (double)zeros, (double)bad);
    set_iter(st, it);
    return go;
}

// A Halley pass's step from its sums S0 + S0c = sum e, S1 = sum tau e,
// S2 = sum tau^2 e (device).
__device__ inline void halley_update(MFState* st, double S0, double S0c, double S1, double S2, bool precise)
{
    st->ticket = 0;
    const double nn = (double)st->n;
    MFIter it = iter_of(st);
    mf_step(it, (S0 + S0c) / nn - st->Ft, -S1 / nn, S2 / nn, st->tol, (double)__uint_as_float(st->tau_max_bits),
            precise);
    set_iter(st, it);
}

// After the flux pass: the F just written is final when a precise pass has
// ended the iteration at this A (|g| <= tol, a certified step, or a step
// below FP64 resolution); else more passes are needed.  The pass's own FP32
// g is only a consistency check of that decision.
__device__ inline void flux_update(MFState* st, double S0, double S0c)
{
    st->ticket = 0;
    const double g = (S0 + S0c) / (double)st->n - st->Ft;
    if (st->done && st->status == LYA_OK) {
        if (!(fabs(g) <= kApproxGErr)) {             // cannot happen unless the sums are wrong
            st->status = LYA_ENOCONV;
            st->done = 0;
        }
    } else {
        st->g = g;
        st->status = LYA_ENOCONV;                     // more passes needed
        st->done = 0;
    }
}

}  // namespace mfd
}  // namespace lya
