// mean_flux.cu -- mean-flux rescaling, transmitted flux and flux statistics.
//
// Sec. 2.3: A solves g(A) = <exp(-A tau)> - F_t = 0 over every pixel of the
// request.  g is convex and decreasing and, by Jensen's inequality,
// g(A0) >= 0 at A0 = -ln(F_t)/<tau>, so Newton steps from A0 rise
// monotonically to the root; a bisection step replaces any step that is
// non-finite or leaves the bracket.
//
// Device-resident Newton: each pass is one grid-wide reduction of
// (sum e, sum tau e) with e = exp(-A tau); the last CTA to finish (an atomic
// ticket, no spin-wait) sums the per-CTA partials in a fixed order in FP64
// and updates A in device memory, so passes chain on the stream without a
// host round trip.  A pass launched after convergence returns at once.
//
// Precision: the first Halley pass of a round forms e = 2^-y, y = tau A log2(e)
// = y_hi + y_lo (a double-float argument), with an FP32 polynomial on the FMA
// pipe, summed in FP32 steps and FP64 across them (g to ~1e-9: a fast start
// that never ends the iteration).  The second Halley pass forms e in double-float arithmetic
// to ~3e-14 (exp2_neg_precise) and sums it in renormalised float pairs
// flushed to FP64 every 32 values, so g is known to ~1e-13; it ends the
// iteration when |g| <= tol (1e-12) or when its Newton step is certified to
// land within tol (halley_update).  It also writes F = e rounded to FP32,
// which is final when its step moved A too little to change F by more than
// kFluxShift; otherwise a flux pass (MUFU exponential) writes F at the final
// A.  CTAs and the final sums are FP64.
#include <cmath>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <atomic>
#include <mutex>

#include "lya_device.cuh"
#include "lya_internal.h"
#include "mean_flux_device.cuh"

namespace lya {
namespace {

using namespace mfd;

// ---- start value from a sample of tau ---------------------------------------------
// Every (smask + 1)-th value (all of them for n <= 2^22, else at least 2^22,
// a few MB read): the quarter-octave log-histogram and the mean of the
// sample.  The last CTA starts A at -ln(F_t)/<tau>_sample, refined by the
// root of the histogram proxy (proxy_start).  The checks over every value
// (invalid values, all zero, too many zeros for a root) and the largest tau
// come with the first Halley pass, which reads every value anyway.
__global__ void __launch_bounds__(kThreads) mf_sample_kernel(const float* __restrict__ tau, long long n,
                                                           MFState* st, Partial* part)
{
    __shared__ unsigned int h_s[kHistBins + 1];            // + the sample's zeros
    for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x) h_s[b] = 0;
    __syncthreads();
    long long smask = 0;
    while ((n >> 22) > smask) smask = 2 * smask + 1;        // sample stride - 1 (a power of 2 minus 1)
    const long long ns = (n + smask) / (smask + 1);
    KahanF32 s;
    unsigned int z = 0, cnt = 0;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nthr = (long long)gridDim.x * blockDim.x;
    auto take = [&](float t) {
        if (!(t >= 0.f) || !isfinite(t)) return;
        s.add(t);
        ++cnt;
        z += (t == 0.f);
        atomicAdd(&h_s[t == 0.f ? kHistBins : hist_bin(t)], 1u);
    };
    // four strided loads in flight per thread, then their values
    long long k = tid;
    for (; k + 3 * nthr < ns; k += 4 * nthr) {
        float t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = tau[(k + u * nthr) * (smask + 1)];
#pragma unroll
        for (int u = 0; u < 4; ++u) take(t[u]);
    }
    for (; k < ns; k += nthr) take(tau[k * (smask + 1)]);
    __shared__ double sh[3][32];
    double v[3] = {(double)s.value(), (double)z, (double)cnt};
    block_sum<3>(v, sh);
    for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x)
        if (h_s[b]) atomicAdd(&st->hist[b], (unsigned long long)h_s[b]);
    if (threadIdx.x == 0) part[blockIdx.x] = Partial{v[0], 0.0, 0.0, 0.0, (long long)v[1], (long long)v[2]};
    if (!last_block(&st->ticket)) return;
    double tot[3];
    partial_totals<3>(part, gridDim.x, tot, sh, [](const Partial& p, double (&x)[3]) {
        x[0] = p.s0; x[1] = (double)p.z; x[2] = (double)p.bad;
    });
    if (threadIdx.x == 0) {
        st->ticket = 0;
        const double mean = tot[2] > 0.0 ? tot[0] / tot[2] : 0.0;
        st->A = mean > 0.0 ? -log(st->Ft) / mean : 1.0;
        st->lo = 0.0;
        st->hi = INFINITY;
        st->iter = 0;
        st->done = 0;
        st->status = LYA_ENOCONV;                    // until converged
    }
    __syncthreads();
    proxy_start(st);
}

// ---- the root-find state set on the device (no host copy to wait for) -----------
__global__ void __launch_bounds__(kThreads) mf_state_init_kernel(MFState* st, double Ft, double tol, long long n,
                                                               int max_iter)
{
    unsigned long long* w = reinterpret_cast<unsigned long long*>(st);
    for (int k = threadIdx.x; k < (int)(sizeof(MFState) / sizeof(unsigned long long)); k += blockDim.x) w[k] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
        st->Ft = Ft;
        st->tol = tol;
        st->n = n;
        st->max_iter = max_iter;
        st->status = LYA_ENOCONV;
    }
}

// ---- the fast Halley pass: g, g' and g'' in one read of tau ------------------------
// The FP32 polynomial exponential (exp2_neg_fast: no systematic bias beyond
// ~1e-9), summed in FP32 over steps of at most 32 values and in
// FP64 across them: g to ~1e-9 in practice, but with no bound that could end
// the iteration, so it is a start for the precise pass, close enough that the
// precise pass's step seldom moves F.  It also makes the checks over every
// value (invalid values, all zero, too many zeros for a root) and finds the
// largest tau: t + 0 maps -0 to +0, and the largest of those float bits as
// unsigned is above 0x7f7fffff exactly when some value is negative, infinite
// or NaN, else it is the bits of the largest tau.
__global__ void __launch_bounds__(kThreads, 6) mf_newton_kernel(const float* __restrict__ tau, long long n,
                                                           MFState* st, Partial* part)
{
    if (st->done) return;
    float a_hi, a_lo;
    split_rate(st->A, a_hi, a_lo);
    __shared__ double sh[6][32];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned int z = 0, umax = 0;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    stream_f32_steps(tau, n, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x,
                     [&](float t) {
        const float e = exp2_neg_fast(t, a_hi, a_lo);
        s0 += e;
        const float te = t * e;
        s1 += te;
        s2 = fmaf(t, te, s2);
        const unsigned int b = __float_as_uint(t + 0.f);
        umax = max(umax, b);
        z += (b == 0u);
    }, [&] {
        v[0] += (double)s0;
        v[2] += (double)s1;
        v[3] += (double)s2;
        s0 = s1 = s2 = 0.f;
    });
    umax = __reduce_max_sync(0xffffffffu, umax);
    const bool bad = umax > 0x7f7fffffu;
    if ((threadIdx.x & 31) == 0 && umax > 0u && !bad) atomicMax(&st->tau_max_bits, umax);
    block_sum<4>(v, sh);
    double zb[2] = {(double)z, bad ? 1.0 : 0.0};
    block_sum<2>(zb, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = Partial{v[0], v[1], v[2], v[3], (long long)zb[0], (long long)zb[1]};
    if (!last_block(&st->ticket)) return;
    double tot[6];
    partial_totals<6>(part, gridDim.x, tot, sh, [](const Partial& p, double (&x)[6]) {
        x[0] = p.s0; x[1] = p.s0c; x[2] = p.s1; x[3] = p.s2; x[4] = (double)p.z; x[5] = (double)p.bad;
    });
    if (threadIdx.x == 0) {
        const double nn = (double)n;
        if (tot[5] > 0.0 || tot[4] >= nn) {                      // invalid values, or all zero
            st->status = LYA_EINVAL;
            st->done = 1;
        } else if (tot[4] / nn >= st->Ft) {                      // <e^{-A tau}> >= zero fraction: no root
            st->status = LYA_ENOCONV;
            st->done = 1;
        } else {
            halley_update(st, tot[0], tot[1], tot[2], tot[3], false);
        }
    }
}

struct StatsOut {
    double m1, m2;                // sums of (F - 0.5) and (F - 0.5)^2
    unsigned long long pdf[21];
    unsigned int ticket;
};

// Sums the per-CTA statistics into *sout (the last CTA, all of its threads).
__device__ inline void stats_totals(const StatPart* spart, StatsOut* sout, double (*sh)[32])
{
    double ms[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        ms[0] += spart[b].m1;
        ms[1] += spart[b].m2;
    }
    block_sum<2>(ms, sh);
    for (int k = threadIdx.x; k < 21; k += blockDim.x) {
        unsigned long long c = 0;
        for (int b = 0; b < (int)gridDim.x; ++b) c += spart[b].pdf[k];
        sout->pdf[k] = c;
    }
    if (threadIdx.x == 0) {
        sout->m1 = ms[0];
        sout->m2 = ms[1];
    }
}

// ---- the precise Halley pass, with F written at its A ------------------------------
// e = 2^-(tau A log2 e) in double-float arithmetic (exp2_neg_precise), summed
// in renormalised float pairs flushed to FP64, so g is known to ~1e-13 and
// the pass may end the iteration (halley_update).  The same e, rounded to
// FP32, is written as F (with its statistics when STATS).  A step from A to
// A' = A + dA changes e^{-A tau} by at most |dA| tau e^{-min(A, A') tau} <=
// |dA| / (e min(A, A')) (the maximum of tau e^{-x tau} is 1/(e x)), so when
// the pass ends the iteration and that bound is <= kFluxShift, the F written
// here is the final F (flux_ok) and no flux pass follows.
constexpr double kFluxShift = 6e-8;   // ~1 FP32 ulp of F in [1/2, 1); the MUFU flux pass errs by ~1.2e-7

template <bool STATS>
__global__ void __launch_bounds__(kThreads, 4) mf_precise_kernel(const float* __restrict__ tau, long long n,
                                                            MFState* st, Partial* part, float* __restrict__ F,
                                                            StatPart* spart, StatsOut* sout)
{
    if (st->done) return;
    __shared__ float2 tab[kExp2TabSize];
    // one private 21-bin counter row per thread (21 is odd: conflict-free)
    __shared__ unsigned int cnt[STATS ? kThreads * 21 : 1];
    unsigned int* mine = cnt + (STATS ? threadIdx.x * 21 : 0);
    if constexpr (STATS)
        for (int k = 0; k < 21; ++k) mine[k] = 0;
    load_exp2_table(tab);                             // ends with a barrier
    const double A = st->A;
    float a_hi, a_lo;
    split_rate(A, a_hi, a_lo);
    DFSum s0;                                         // sum e to ~1e-13 (float pairs, FP64)
    // sum tau e (g' enters the step's certificate) and sum tau^2 e in FP32
    // over a step of <= 32 values (nonnegative terms: <= 31 * 2^-24 relative),
    // FP64 across steps; likewise the statistics
    float s1 = 0.f, s2 = 0.f;
    double sd1 = 0.0, sd2 = 0.0;
    float m1 = 0.f, m2 = 0.f;
    double md1 = 0.0, md2 = 0.0;
    auto flush = [&] {
        s0.flush();
        sd1 += (double)s1;
        sd2 += (double)s2;
        s1 = 0.f;
        s2 = 0.f;
        if constexpr (STATS) {
            md1 += (double)m1;
            md2 += (double)m2;
            m1 = 0.f;
            m2 = 0.f;
        }
    };
    auto proc = [&](float t) {
        float eh, el;
        exp2_neg_precise(t, a_hi, a_lo, tab, eh, el);
        s0.add(eh, el);
        const float te = t * eh;
        s1 += te;
        s2 = fmaf(t, te, s2);
        // F: the pair rounded once; past the exponential's clamp (tau A log2 e
        // > 100) the MUFU value, which flushes below 2^-126
        const float y = t * a_hi;
        const float f = y <= 100.f ? __fadd_rn(eh, el) : ex2(-y);
        if constexpr (STATS) {
            const float d = f - 0.5f;
            m1 += d;
            m2 = fmaf(d, d, m2);
            mine[pdf_bin_unit(f)] += 1u;
        }
        return f;
    };
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nthr = (long long)gridDim.x * blockDim.x;
    if ((reinterpret_cast<uintptr_t>(tau) & 15) == 0 && (!F || (reinterpret_cast<uintptr_t>(F) & 15) == 0)) {
        const float4* __restrict__ t4 = reinterpret_cast<const float4*>(tau);
        float4* __restrict__ F4 = reinterpret_cast<float4*>(F);
        const long long n4 = n >> 2;
        long long i = tid;
        // eight float4 in flight per thread, four with the statistics (their
        // registers would otherwise push the kernel below four CTAs per SM)
        constexpr int U = STATS ? 4 : 8;
        for (; i + (U - 1) * nthr < n4; i += U * nthr) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = t4[i + u * nthr];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float4 o;
                o.x = proc(v[u].x);
                o.y = proc(v[u].y);
                o.z = proc(v[u].z);
                o.w = proc(v[u].w);
                if (F) __stcs(F4 + i + u * nthr, o);
            }
            flush();                                  // at most 32 values per step
        }
        for (; i < n4; i += nthr) {
            const float4 v = t4[i];
            float4 o;
            o.x = proc(v.x);
            o.y = proc(v.y);
            o.z = proc(v.z);
            o.w = proc(v.w);
            if (F) __stcs(F4 + i, o);
            flush();
        }
        for (long long k = 4 * n4 + tid; k < n; k += nthr) {
            const float f = proc(tau[k]);
            if (F) F[k] = f;
        }
    } else {
        int c = 0;
        for (long long k = tid; k < n; k += nthr) {
            const float f = proc(tau[k]);
            if (F) F[k] = f;
            if (++c == 32) {
                flush();
                c = 0;
            }
        }
    }
    flush();
    __shared__ double sh[4][32];
    double v[4] = {s0.value(), 0.0, sd1, sd2};
    block_sum<4>(v, sh);                              // ends with a barrier
    if constexpr (STATS) {
        double ms[2] = {md1, md2};
        block_sum<2>(ms, sh);
        for (int k = threadIdx.x; k < 21; k += blockDim.x) {
            unsigned int c = 0;
            for (int r = 0; r < (int)blockDim.x; ++r) c += cnt[r * 21 + k];
            spart[blockIdx.x].pdf[k] = c;
        }
        if (threadIdx.x == 0) {
            spart[blockIdx.x].m1 = ms[0];
            spart[blockIdx.x].m2 = ms[1];
        }
    }
    if (threadIdx.x == 0) part[blockIdx.x] = Partial{v[0], v[1], v[2], v[3], 0, 0};
    if (!last_block(&st->ticket)) return;
    double tot[4];
    partial_totals<4>(part, gridDim.x, tot, sh, [](const Partial& p, double (&x)[4]) {
        x[0] = p.s0; x[1] = p.s0c; x[2] = p.s1; x[3] = p.s2;
    });
    __shared__ int s_final;
    if (threadIdx.x == 0) {
        halley_update(st, tot[0], tot[1], tot[2], tot[3], true);
        const double An = st->A;
        const double shift = fabs(An - A) / (2.718281828459045 * fmin(A, An));
        st->flux_ok = st->done && st->status == LYA_OK && (An == A || shift <= kFluxShift);
        s_final = st->flux_ok;
    }
    __syncthreads();
    if (STATS && s_final) stats_totals(spart, sout, sh);
}

// ---- F = exp(-A tau) at the final A when the precise pass's F is not close
//      enough to it, the convergence check at that A and, optionally, the
//      statistics of that F (kept only when the check passes) ---------------

template <bool STATS>
__global__ void __launch_bounds__(kThreads) mf_flux_kernel(const float* __restrict__ tau, long long n,
                                                         MFState* st, Partial* part, float* __restrict__ F,
                                                         StatPart* spart, StatsOut* sout)
{
    // runs only after a precise pass ended the iteration without its own F
    // being final (an error, or more passes to come, leaves it at once)
    if (!st->done || st->status != LYA_OK || st->flux_ok) return;
    // one private 21-bin counter row per thread (21 is odd: conflict-free)
    __shared__ unsigned int cnt[STATS ? kThreads * 21 : 1];
    unsigned int* mine = cnt + (STATS ? threadIdx.x * 21 : 0);
    if constexpr (STATS)
        for (int k = 0; k < 21; ++k) mine[k] = 0;
    float a_hi, a_lo;
    split_rate(st->A, a_hi, a_lo);
    // F in FP32 (MUFU exponential, first-order argument correction); the sum
    // of e only cross-checks the precise pass's decision
    KahanF32 s0, m1, m2;
    float s0c = 0.f;
    auto proc = [&](float t) {
        float e, c;
        exp_neg(t, a_hi, a_lo, e, c);
        const float f = e + c;
        s0.add(e);
        s0c += c;
        if constexpr (STATS) {
            const float d = f - 0.5f;
            m1.add(d);
            m2.add(d * d);
            mine[pdf_bin(f)] += 1u;
        }
        return f;
    };
    // the values in the order stream_f32 gives them, F written back as float4
    // where tau and F are 16-byte aligned
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, nthr = (long long)gridDim.x * blockDim.x;
    if ((reinterpret_cast<uintptr_t>(tau) & 15) == 0 && (!F || (reinterpret_cast<uintptr_t>(F) & 15) == 0)) {
        const float4* __restrict__ t4 = reinterpret_cast<const float4*>(tau);
        float4* __restrict__ F4 = reinterpret_cast<float4*>(F);
        const long long n4 = n >> 2;
        long long i = tid;
        for (; i + 7 * nthr < n4; i += 8 * nthr) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = t4[i + u * nthr];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float4 o;
                o.x = proc(v[u].x);
                o.y = proc(v[u].y);
                o.z = proc(v[u].z);
                o.w = proc(v[u].w);
                if (F) F4[i + u * nthr] = o;
            }
        }
        for (; i < n4; i += nthr) {
            const float4 v = t4[i];
            float4 o;
            o.x = proc(v.x);
            o.y = proc(v.y);
            o.z = proc(v.z);
            o.w = proc(v.w);
            if (F) F4[i] = o;
        }
        for (long long k = 4 * n4 + tid; k < n; k += nthr) {
            const float f = proc(tau[k]);
            if (F) F[k] = f;
        }
    } else {
        for (long long k = tid; k < n; k += nthr) {
            const float f = proc(tau[k]);
            if (F) F[k] = f;
        }
    }
    constexpr int K = STATS ? 4 : 2;
    __shared__ double sh[K][32];
    double v[K];
    v[0] = (double)s0.value();
    v[1] = (double)s0c;
    if constexpr (STATS) {
        v[2] = (double)m1.value();
        v[3] = (double)m2.value();
    }
    block_sum<K>(v, sh);                                     // ends with a barrier
    if constexpr (STATS) {
        for (int k = threadIdx.x; k < 21; k += blockDim.x) {
            unsigned int c = 0;
            for (int r = 0; r < (int)blockDim.x; ++r) c += cnt[r * 21 + k];
            spart[blockIdx.x].pdf[k] = c;
        }
        if (threadIdx.x == 0) {
            spart[blockIdx.x].m1 = v[2];
            spart[blockIdx.x].m2 = v[3];
        }
    }
    if (threadIdx.x == 0) part[blockIdx.x] = Partial{v[0], v[1], 0.0, 0.0, 0, 0};
    if (!last_block(&st->ticket)) return;
    double tot[2];
    partial_totals<2>(part, gridDim.x, tot, sh, [](const Partial& p, double (&x)[2]) {
        x[0] = p.s0; x[1] = p.s0c;
    });
    if constexpr (!STATS) {
        if (threadIdx.x == 0) flux_update(st, tot[0], tot[1]);
    } else {
        __shared__ int s_final;
        if (threadIdx.x == 0) {
            flux_update(st, tot[0], tot[1]);
            s_final = st->done && st->status == LYA_OK;
        }
        __syncthreads();
        if (s_final) stats_totals(spart, sout, sh);
    }
}

// ---- flux statistics -----------------------------------------------------------------

__global__ void __launch_bounds__(kThreads) stats_kernel(const float* __restrict__ F, long long n,
                                                       StatsOut* out, double* part)
{
    // one private 21-bin counter row per thread: plain increments, no atomics;
    // rows are 21 words apart, and 21 is odd, so a warp's rows hit 32 banks
    __shared__ unsigned int cnt[kThreads * 21];
    unsigned int* mine = cnt + threadIdx.x * 21;
    for (int k = 0; k < 21; ++k) mine[k] = 0;
    KahanF32 m1, m2;
    stream_f32(F, n, [&](long long, float f) {
        const float d = f - 0.5f;
        m1.add(d);
        m2.add(d * d);
        mine[pdf_bin(f)] += 1u;
    });
    __shared__ double sh[2][32];
    double v[2] = {(double)m1.value(), (double)m2.value()};
    block_sum<2>(v, sh);                                     // ends with a barrier
    for (int k = threadIdx.x; k < 21; k += blockDim.x) {
        unsigned long long c = 0;
        for (int r = 0; r < (int)blockDim.x; ++r) c += cnt[r * 21 + k];
        if (c) atomicAdd(&out->pdf[k], c);
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = v[0];
        part[2 * blockIdx.x + 1] = v[1];
    }
    if (!last_block(&out->ticket)) return;
    double tot[2] = {0.0, 0.0};
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
        tot[0] += part[2 * k];
        tot[1] += part[2 * k + 1];
    }
    block_sum<2>(tot, sh);
    if (threadIdx.x != 0) return;
    out->m1 = tot[0];
    out->m2 = tot[1];
    out->ticket = 0;
}

// ---- field validation ---------------------------------------------------------------
// The check's totals start empty (no flags, maxima 0, the smallest positive
// rho at +inf); field_check_kernel accumulates into them with atomics, so a
// field may be checked in pieces.
__global__ void field_check_init_kernel(FieldCheck* out)
{
    if (threadIdx.x == 0) {
        out->bad_rho = out->bad_vpec = out->bad_temp = 0ull;
        out->temp_max_bits = 0u;
        out->rho_max_bits = 0u;
        out->rho_minpos_bits = 0x7f800000u;           // +inf
    }
}

__global__ void __launch_bounds__(kThreads) field_check_kernel(const float* __restrict__ rho,
                                                             const float* __restrict__ v,
                                                             const float* __restrict__ T, long long n,
                                                             FieldCheck* out)
{
    unsigned long long br = 0, bv = 0, bt = 0;
    float tmax = 0.f, rmax = 0.f, rmin = INFINITY;
    auto check = [&](float r, float u, float t) {
        const bool rok = r >= 0.f && isfinite(r);
        br += !rok;
        bv += !(isfinite(u) && fabsf(u) < 2.99792458e5f);
        if (rok && r > 0.f) {
            rmax = fmaxf(rmax, r);
            rmin = fminf(rmin, r);
        }
        if (T) {
            const bool ok = isfinite(t) && (t > 0.f || !(r > 0.f));
            bt += !ok;
            if (ok && r > 0.f) tmax = fmaxf(tmax, t);
        }
    };
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const bool aligned = ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(v) |
                           reinterpret_cast<uintptr_t>(T)) & 15) == 0;
    long long k0 = 0;
    if (aligned) {
        const long long n4 = n >> 2;
        for (long long i = tid; i < n4; i += nthr) {
            const float4 r = reinterpret_cast<const float4*>(rho)[i];
            const float4 u = reinterpret_cast<const float4*>(v)[i];
            const float4 t = T ? reinterpret_cast<const float4*>(T)[i] : make_float4(1.f, 1.f, 1.f, 1.f);
            check(r.x, u.x, t.x); check(r.y, u.y, t.y); check(r.z, u.z, t.z); check(r.w, u.w, t.w);
        }
        k0 = 4 * n4;
    }
    for (long long i = k0 + tid; i < n; i += nthr) check(rho[i], v[i], T ? T[i] : 1.f);
    for (int o = 16; o > 0; o >>= 1) {
        br += __shfl_down_sync(0xffffffffu, br, o);
        bv += __shfl_down_sync(0xffffffffu, bv, o);
        bt += __shfl_down_sync(0xffffffffu, bt, o);
        tmax = fmaxf(tmax, __shfl_down_sync(0xffffffffu, tmax, o));
        rmax = fmaxf(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
        rmin = fminf(rmin, __shfl_down_sync(0xffffffffu, rmin, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (br) atomicAdd(&out->bad_rho, br);
        if (bv) atomicAdd(&out->bad_vpec, bv);
        if (bt) atomicAdd(&out->bad_temp, bt);
        // non-negative floats order like their bit patterns
        atomicMax(&out->temp_max_bits, __float_as_uint(tmax));
        atomicMax(&out->rho_max_bits, __float_as_uint(rmax));
        atomicMin(&out->rho_minpos_bits, __float_as_uint(rmin));
    }
}

int grid_for(long long n)
{
    const long long want = (n + kThreads - 1) / kThreads;
    const long long cap = 4LL * sm_count();
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// The fast Halley pass's grid: six CTAs per SM (it holds 40 registers at that
// bound), so more of its loads are in flight than at the four of the other
// passes; at most `cap` CTAs (the partials the scratch holds).
int fast_grid_for(long long n, int cap)
{
    const long long want = (n + kThreads - 1) / kThreads;
    long long g = 6LL * sm_count();
    if (want < g) g = want > 0 ? want : 1;
    return (int)(g < cap ? g : cap);
}

}  // namespace

// SM count of the current device, cached per device (a relaxed atomic per
// slot: concurrent first calls may both query, and store the same value).
int sm_count()
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> cached[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < kMaxDev) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    v = v > 0 ? v : 1;
    if (dev >= 0 && dev < kMaxDev) cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

cudaMemPool_t scratch_pool()
{
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull;                      // never hand memory back on a synchronise
        (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

cudaError_t scratch_malloc(void** p, size_t bytes, cudaStream_t stream)
{
    cudaMemPool_t pool = scratch_pool();
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, stream) : cudaMallocAsync(p, bytes, stream);
}

size_t max_dynamic_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

cudaError_t launch_field_check_init(FieldCheck* d_out, cudaStream_t stream)
{
    field_check_init_kernel<<<1, 32, 0, stream>>>(d_out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_field_check_range(const float* rho, const float* vpec, const float* temp, int64_t n,
                                     FieldCheck* d_out, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    field_check_kernel<<<grid_for(n), kThreads, 0, stream>>>(rho, vpec, temp, n, d_out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_field_check(const float* rho, const float* vpec, const float* temp, int64_t n,
                               FieldCheck* d_out, cudaStream_t stream)
{
    cudaError_t e = launch_field_check_init(d_out, stream);
    if (e == cudaSuccess) e = launch_field_check_range(rho, vpec, temp, n, d_out, stream);
    return e;
}

#define LYA_TRY(call)                                   \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) { err = _e; goto done; } \
    } while (0)

namespace {

// The host side of one root-find on caller-chosen scratch: the sample pass
// (start value), then rounds of two Halley passes (MUFU with the checks over
// every value, then precise: the latter decides convergence) and one flux pass
// (which writes F, if asked, at the final A), reading the state back once per
// round.
static lya_status solve_on_scratch(const float* tau, int64_t n, double target, double tol, int max_iter,
                                   double* A_out, float* flux_out, MFState* st, Partial* part, int grid,
                                   int fast_grid, cudaStream_t stream, StatPart* spart = nullptr,
                                   StatsOut* sout = nullptr, lya_flux_stats_t* stats_out = nullptr)
{
    static_assert(sizeof(MFState) % 8 == 0, "state layout");
    MFState hs{};                                   // host copy of the state's header (no heap allocation)
    MFState* h = &hs;
    StatsOut hs2{};
    lya_status result = LYA_ENOCONV;
    // the state is set by a kernel, so nothing waits for the optical-depth
    // kernel ahead of it on the stream
    mf_state_init_kernel<<<1, kThreads, 0, stream>>>(st, target, tol, (long long)n, max_iter);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) {
        mf_sample_kernel<<<grid, kThreads, 0, stream>>>(tau, n, st, part);
        count_launch();
        err = cudaGetLastError();
    }
    for (int round = 0; err == cudaSuccess; ++round) {
        // a fast (MUFU) Halley pass, a precise one that writes F at its A, then
        // the flux pass at the final A, which leaves at once when the precise
        // pass's F is final
        mf_newton_kernel<<<fast_grid, kThreads, 0, stream>>>(tau, n, st, part);
        count_launch();
        err = cudaGetLastError();
        if (err == cudaSuccess) {
            if (spart)
                mf_precise_kernel<true><<<grid, kThreads, 0, stream>>>(tau, n, st, part, flux_out, spart, sout);
            else
                mf_precise_kernel<false><<<grid, kThreads, 0, stream>>>(tau, n, st, part, flux_out, nullptr, nullptr);
            count_launch();
            err = cudaGetLastError();
        }
        if (err != cudaSuccess) break;
        if (spart)
            mf_flux_kernel<true><<<grid, kThreads, 0, stream>>>(tau, n, st, part, flux_out, spart, sout);
        else
            mf_flux_kernel<false><<<grid, kThreads, 0, stream>>>(tau, n, st, part, flux_out, nullptr, nullptr);
        count_launch();
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaMemcpyAsync(h, st, offsetof(MFState, hist), cudaMemcpyDeviceToHost, stream);
        // the statistics ride along (kept only once the state says done), one wait for both
        if (err == cudaSuccess && stats_out)
            err = cudaMemcpyAsync(&hs2, sout, sizeof(StatsOut), cudaMemcpyDeviceToHost, stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
        if (err != cudaSuccess) break;
        if (h->done) {
            result = (lya_status)h->status;
            break;
        }
        if (h->iter >= max_iter) {
            result = LYA_ENOCONV;
            break;
        }
    }
    if (err == cudaSuccess && result == LYA_OK) *A_out = h->A;
    if (err == cudaSuccess && result == LYA_OK && stats_out) {
        const double nn = (double)n;
        const double m1 = hs2.m1 / nn, m2 = hs2.m2 / nn;
        stats_out->mean_flux = 0.5 + m1;
        stats_out->var_flux = m2 - m1 * m1;
        stats_out->tau_eff = -log(stats_out->mean_flux);
        for (int k = 0; k < 21; ++k) stats_out->pdf[k] = (int64_t)hs2.pdf[k];
        stats_out->n = n;
    }
    if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA;
    return result;
}

}  // namespace

lya_status mean_flux_solve(const float* tau, int64_t n, double target, double tol, int max_iter,
                           double* A_out, float* flux_out, cudaStream_t stream, lya_flux_stats_t* stats_out)
{
    const int grid = grid_for(n);
    const int fast_grid = fast_grid_for(n, 1 << 30);
    MFState* st = nullptr;
    Partial* part = nullptr;
    StatPart* spart = nullptr;
    StatsOut* sout = nullptr;
    cudaError_t err = scratch_malloc((void**)&st, sizeof(MFState), stream);
    if (err == cudaSuccess)
        err = scratch_malloc((void**)&part, sizeof(Partial) * (grid > fast_grid ? grid : fast_grid), stream);
    if (err == cudaSuccess && stats_out) err = scratch_malloc((void**)&spart, sizeof(StatPart) * grid, stream);
    if (err == cudaSuccess && stats_out) err = scratch_malloc((void**)&sout, sizeof(StatsOut), stream);
    lya_status result = err == cudaSuccess
        ? solve_on_scratch(tau, n, target, tol, max_iter, A_out, flux_out, st, part, grid, fast_grid, stream,
                           spart, sout, stats_out)
        : (err == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA);
    if (st) cudaFreeAsync(st, stream);
    if (part) cudaFreeAsync(part, stream);
    if (spart) cudaFreeAsync(spart, stream);
    if (sout) cudaFreeAsync(sout, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess && result == LYA_OK) result = LYA_ECUDA;
    return result;
}

lya_status flux_stats_run(const float* flux, int64_t n, lya_flux_stats_t* out, cudaStream_t stream)
{
    const int grid = grid_for(n);
    StatsOut* d = nullptr;
    double* part = nullptr;
    StatsOut h{};
    cudaError_t err = cudaSuccess;
    LYA_TRY(scratch_malloc((void**)&d, sizeof(StatsOut), stream));
    LYA_TRY(scratch_malloc((void**)&part, sizeof(double) * 2 * grid, stream));
    LYA_TRY(cudaMemsetAsync(d, 0, sizeof(StatsOut), stream));
    stats_kernel<<<grid, kThreads, 0, stream>>>(flux, n, d, part);
    count_launch();
    LYA_TRY(cudaGetLastError());
    LYA_TRY(cudaMemcpyAsync(&h, d, sizeof(StatsOut), cudaMemcpyDeviceToHost, stream));
    LYA_TRY(cudaStreamSynchronize(stream));
    {
        const double nn = (double)n;
        const double m1 = h.m1 / nn, m2 = h.m2 / nn;
        out->mean_flux = 0.5 + m1;
        out->var_flux = m2 - m1 * m1;
        out->tau_eff = -log(out->mean_flux);
        for (int k = 0; k < 21; ++k) out->pdf[k] = (int64_t)h.pdf[k];
        out->n = n;
    }
done:
    if (d) cudaFreeAsync(d, stream);
    if (part) cudaFreeAsync(part, stream);
    if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA;
    return LYA_OK;
}

}  // namespace lya

// ---- allocation-free mean-flux root-find -------------------------------------------
//
// For callers that cannot allocate device memory: plug-ins whose host
// application forbids allocation after start-up, or callers on a memory
// budget that is already fully handed out.  The root-find state and the
// per-CTA partials live in a fixed file-scope device array instead of
// stream-ordered allocations.  The array is kNoAllocScratchBytes (64 KiB) on
// every GPU that loads the library and stays there until the process exits;
// it fits the state plus kNoAllocMaxBlocks partials, so the reduction grid is
// capped at kNoAllocMaxBlocks CTAs (the grid-stride loops still cover any n).
//
// Every call shares the one array.  Nothing carries over from an earlier
// call: mf_state_init_kernel zeroes and sets the whole state at the start of
// each call, and every CTA writes its partial before the last CTA reads them.
// Two calls whose work overlaps on the GPU (different streams, or different
// host threads on one device) race on the array.  Like the allocating
// root-find, the call copies the state back and synchronises its stream after
// every round of passes, so it cannot run while the stream is capturing a
// CUDA graph.
namespace lya {
namespace {

constexpr size_t kNoAllocScratchBytes = 64 * 1024;
constexpr int kNoAllocMaxBlocks = 1024;
constexpr size_t kNoAllocStateBytes = 8192;     // MFState, padded to the array's alignment
static_assert(sizeof(MFState) <= kNoAllocStateBytes, "state does not fit its slot");
static_assert(kNoAllocStateBytes + kNoAllocMaxBlocks * sizeof(Partial) <= kNoAllocScratchBytes,
              "partials do not fit the scratch array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not its address).
cudaError_t noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

lya_status mean_flux_solve_noalloc(const float* tau, int64_t n, double target, double tol, int max_iter,
                                   double* A_out, float* flux_out, cudaStream_t stream)
{
    void* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return LYA_ECUDA;
    const int grid = grid_for(n) < kNoAllocMaxBlocks ? grid_for(n) : kNoAllocMaxBlocks;
    if (kNoAllocStateBytes + (size_t)grid * sizeof(Partial) > kNoAllocScratchBytes) return LYA_EINVAL;
    MFState* st = static_cast<MFState*>(scratch);
    Partial* part = reinterpret_cast<Partial*>(static_cast<unsigned char*>(scratch) + kNoAllocStateBytes);
    return solve_on_scratch(tau, n, target, tol, max_iter, A_out, flux_out, st, part, grid,
                            fast_grid_for(n, kNoAllocMaxBlocks), stream);
}

}  // namespace lya

// ---- building blocks for a root-find split over devices or processes ---------------
//
// When the pixels of one request live on several devices, each device reduces
// its own share and the caller combines the sums (one all-reduce of three
// numbers per pass) and steps A on the host; these calls are that per-device
// share.  The single-device root-find above keeps everything on the device.
namespace lya {
namespace {

struct SumsOut {
    double s[3];
    unsigned int ticket;
};

// sum tau (compensated), zero count, invalid count.
__global__ void __launch_bounds__(kThreads) mf_moments_kernel(const float* __restrict__ tau, long long n,
                                                            Partial* part, SumsOut* out)
{
    KahanF32 s;
    long long z = 0, bad = 0;
    stream_f32(tau, n, [&](long long, float t) {
        if (!(t >= 0.f) || !isfinite(t)) { ++bad; return; }
        s.add(t);
        z += (t == 0.f);
    });
    __shared__ double sh[3][32];
    double v[3] = {(double)s.value(), (double)z, (double)bad};
    block_sum<3>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = Partial{v[0], 0.0, 0.0, 0.0, (long long)v[1], (long long)v[2]};
    if (!last_block(&out->ticket)) return;
    double tot[3];
    partial_totals<3>(part, gridDim.x, tot, sh, [](const Partial& p, double (&x)[3]) {
        x[0] = p.s0; x[1] = (double)p.z; x[2] = (double)p.bad;
    });
    if (threadIdx.x != 0) return;
    out->s[0] = tot[0];
    out->s[1] = tot[1];
    out->s[2] = tot[2];
    out->ticket = 0;
}

// sum e, sum tau e, sum tau^2 e with e = exp(-A tau).
__global__ void __launch_bounds__(kThreads) mf_sums_kernel(const float* __restrict__ tau, long long n, double A,
                                                         Partial* part, SumsOut* out)
{
    __shared__ float2 tab[kExp2TabSize];
    load_exp2_table(tab);
    float a_hi, a_lo;
    split_rate(A, a_hi, a_lo);
    DFSum s0;                                   // sum e precise (double-float exponentials)
    float s1 = 0.f, s2 = 0.f;                   // as the precise pass: FP32 per step, FP64 across
    double sd1 = 0.0, sd2 = 0.0;
    stream_f32_steps(tau, n, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x,
                     [&](float t) {
        float eh, el;
        exp2_neg_precise(t, a_hi, a_lo, tab, eh, el);
        s0.add(eh, el);
        const float te = t * eh;
        s1 += te;
        s2 = fmaf(t, te, s2);
    }, [&] {
        s0.flush();
        sd1 += (double)s1;
        sd2 += (double)s2;
        s1 = 0.f;
        s2 = 0.f;
    });
    __shared__ double sh[4][32];
    double v[4] = {s0.value(), 0.0, sd1, sd2};
    block_sum<4>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = Partial{v[0], v[1], v[2], v[3], 0, 0};
    if (!last_block(&out->ticket)) return;
    double tot[4];
    partial_totals<4>(part, gridDim.x, tot, sh, [](const Partial& p, double (&x)[4]) {
        x[0] = p.s0; x[1] = p.s0c; x[2] = p.s1; x[3] = p.s2;
    });
    if (threadIdx.x != 0) return;
    out->s[0] = tot[0] + tot[1];
    out->s[1] = tot[2];
    out->s[2] = tot[3];
    out->ticket = 0;
}

__global__ void __launch_bounds__(kThreads) mf_flux_at_kernel(const float* __restrict__ tau, long long n,
                                                            double A, float* __restrict__ F)
{
    float a_hi, a_lo;
    split_rate(A, a_hi, a_lo);
    stream_f32(tau, n, [&](long long i, float t) {
        float e, c;
        exp_neg(t, a_hi, a_lo, e, c);
        F[i] = e + c;
    });
}

template <typename Launch>
lya_status run_sums(int64_t n, double* out3, cudaStream_t stream, Launch launch)
{
    const int grid = grid_for(n);
    Partial* part = nullptr;
    SumsOut* d = nullptr;
    SumsOut h{};
    cudaError_t e = scratch_malloc((void**)&part, sizeof(Partial) * grid, stream);
    if (e == cudaSuccess) e = scratch_malloc((void**)&d, sizeof(SumsOut), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(SumsOut), stream);
    if (e == cudaSuccess) {
        launch(grid, part, d);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(SumsOut), cudaMemcpyDeviceToHost, stream);
    if (part) cudaFreeAsync(part, stream);
    if (d) cudaFreeAsync(d, stream);
    const cudaError_t e2 = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA;
    for (int k = 0; k < 3; ++k) out3[k] = h.s[k];
    return LYA_OK;
}

}  // namespace

lya_status tau_moments_run(const float* tau, int64_t n, double* out3, cudaStream_t stream)
{
    return run_sums(n, out3, stream, [&](int grid, Partial* part, SumsOut* d) {
        mf_moments_kernel<<<grid, kThreads, 0, stream>>>(tau, n, part, d);
    });
}

lya_status mean_flux_sums_run(const float* tau, int64_t n, double A, double* out3, cudaStream_t stream)
{
    return run_sums(n, out3, stream, [&](int grid, Partial* part, SumsOut* d) {
        mf_sums_kernel<<<grid, kThreads, 0, stream>>>(tau, n, A, part, d);
    });
}

lya_status flux_at_run(const float* tau, int64_t n, double A, float* flux, cudaStream_t stream)
{
    mf_flux_at_kernel<<<grid_for(n), kThreads, 0, stream>>>(tau, n, A, flux);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? LYA_OK : LYA_ECUDA;
}

// ---- the split root-find stepped on the host --------------------------------------
namespace {
MFIter to_core(const lya_mean_flux_iter& it)
{
    return MFIter{it.A, it.lo, it.hi, it.g, it.iter, it.max_iter, it.done, (int)it.status};
}
void from_core(lya_mean_flux_iter& it, const MFIter& c)
{
    it.A = c.A;
    it.lo = c.lo;
    it.hi = c.hi;
    it.g = c.g;
    it.iter = c.iter;
    it.max_iter = c.max_iter;
    it.done = c.done;
    it.status = (lya_status)c.status;
}
}  // namespace

lya_status mean_flux_start(const double totals[4], double target, double tol, int max_iter, lya_mean_flux_iter* it)
{
    *it = lya_mean_flux_iter{};
    it->target = target;
    it->tol = tol;
    it->n = totals[3];
    it->max_iter = max_iter;
    MFIter c = to_core(*it);
    mf_start(c, target, totals[3], totals[0], totals[1], totals[2]);
    from_core(*it, c);
    return it->done ? it->status : LYA_OK;
}

lya_status mean_flux_step(lya_mean_flux_iter* it, const double sums[3])
{
    if (it->done) return it->status;
    MFIter c = to_core(*it);
    // the shares' sum of e is precise (lya_mean_flux_sums): every step may end
    // the iteration; tau_max is not summed over parts, so only steps from below
    // the root (dA > 0, the Newton iteration's side) are certified
    mf_step(c, sums[0] / it->n - it->target, -sums[1] / it->n, sums[2] / it->n, it->tol, INFINITY, true);
    from_core(*it, c);
    return it->done ? it->status : LYA_OK;
}

lya_status mean_flux_sharded(const float* tau, int64_t n, double target, double tol, int max_iter,
                             lya_allreduce_fn allreduce, void* user, double* A_out, int* iters_out, float* flux_out,
                             cudaStream_t stream)
{
    double tot[4] = {0.0, 0.0, 0.0, (double)n};
    if (n > 0) {
        const lya_status st = tau_moments_run(tau, n, tot, stream);
        if (st != LYA_OK) return st;
    }
    if (allreduce(tot, 4, user) != 0) return LYA_ECUDA;
    if (!(tot[3] > 0.0)) return LYA_EINVAL;
    lya_mean_flux_iter it;
    lya_status st = mean_flux_start(tot, target, tol, max_iter, &it);
    while (st == LYA_OK && !it.done) {
        double sums[3] = {0.0, 0.0, 0.0};
        if (n > 0) {
            st = mean_flux_sums_run(tau, n, it.A, sums, stream);
            if (st != LYA_OK) return st;
        }
        if (allreduce(sums, 3, user) != 0) return LYA_ECUDA;
        st = mean_flux_step(&it, sums);
    }
    if (st != LYA_OK) return st;
    *A_out = it.A;
    if (iters_out) *iters_out = it.iter;
    if (flux_out && n > 0) {
        st = flux_at_run(tau, n, it.A, flux_out, stream);
        if (st == LYA_OK && cudaStreamSynchronize(stream) != cudaSuccess) st = LYA_ECUDA;
    }
    return st;
}

}  // namespace lya
