// serve_kernels.cu -- the mean-flux root-find (Sec. 2.3) of many requests at
// once, for the serving loop.
//
// Every request in a step's root-find list is cut into units of consecutive
// pixels; a persistent grid of 256-thread CTAs walks the unit list.  Each
// unit is reduced by one CTA into its own partial; the last unit of a request
// to arrive (an atomic ticket in the request's state, no waiting) sums that
// request's partials in FP64 and takes the same step as the single-request
// kernels: init (the Jensen start refined by the histogram proxy), Halley
// passes (MUFU, then precise: the latter decides convergence), and the flux
// pass that writes F = exp(-A tau) and, once the root-find has ended, the
// request's flux statistics (Sec. 2.3, 5.2).
// Requests whose root-find has ended skip every later pass of the step.
#include <cstdint>

#include "lya_device.cuh"
#include "lya_internal.h"
#include "mean_flux_device.cuh"
#include "serve_internal.h"

namespace lya {
namespace serve {
namespace {

using namespace mfd;

struct View {
    const StepHeader* hdr;
    const RfSlot* rf;
    const RfUnit* units;
    __device__ View(const unsigned char* step)
        : hdr(reinterpret_cast<const StepHeader*>(step)),
          rf(step_table<RfSlot>(step, hdr->off_rf)),
          units(step_table<RfUnit>(step, hdr->off_units))
    {
    }
};

// Publish a finished (or failed) root-find to the slot's result.
__device__ void publish(const MFState* st, SlotResult* res, bool final)
{
    res->A = st->A;
    res->g = st->g;
    res->iter = st->iter;
    res->status = st->status;
    res->done = st->done;
    res->final = final ? 1 : 0;
}

// Reset the state of every request that starts its root-find this step.
__global__ void __launch_bounds__(kRfThreads) rf_reset_kernel(const unsigned char* __restrict__ step,
                                                            MFState* states, SlotResult* results)
{
    const View v(step);
    for (int r = blockIdx.x; r < v.hdr->n_rf; r += gridDim.x) {
        const RfSlot s = v.rf[r];
        if (!s.init) continue;
        MFState* st = states + s.state;
        for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x) st->hist[b] = 0;
        if (threadIdx.x == 0) {
            st->A = st->lo = st->hi = st->g = st->mean_tau = 0.0;
            st->Ft = s.Ft;
            st->tol = s.tol;
            st->n = s.n;
            st->n_zero = st->n_bad = 0;
            st->iter = 0;
            st->max_iter = s.max_iter;
            st->done = 0;
            st->status = LYA_ENOCONV;
            st->ticket = 0;
            st->tau_max_bits = 0u;
            SlotResult* res = results + s.state;
            res->final = 0;
            res->done = 0;
        }
    }
}

// Init pass: sum tau, zero and invalid counts, sampled log-histogram.
__global__ void __launch_bounds__(kRfThreads) rf_init_kernel(const unsigned char* __restrict__ step,
                                                           MFState* states, SlotResult* results, Partial* part)
{
    const View v(step);
    __shared__ unsigned int h_s[kHistBins + 1];
    __shared__ double sh[3][32];
    __shared__ int s_go;
    for (int u = blockIdx.x; u < v.hdr->n_units; u += gridDim.x) {
        const RfUnit U = v.units[u];
        const RfSlot s = v.rf[U.rf];
        if (!s.init) continue;
        MFState* st = states + s.state;
        for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x) h_s[b] = 0;
        __syncthreads();
        long long smask = 0;
        while ((s.n >> 22) > smask) smask = 2 * smask + 1;
        KahanF32 acc;
        long long z = 0, bad = 0;
        float tmax = 0.f;
        stream_f32(s.tau + U.begin, U.end - U.begin, threadIdx.x, blockDim.x, [&](long long i, float t) {
            if (!(t >= 0.f) || !isfinite(t)) { ++bad; return; }
            acc.add(t);
            z += (t == 0.f);
            tmax = fmaxf(tmax, t);
            if (((U.begin + i) & smask) == 0) atomicAdd(&h_s[t == 0.f ? kHistBins : hist_bin(t)], 1u);
        });
        double x[3] = {(double)acc.value(), (double)z, (double)bad};
        block_sum<3>(x, sh);
        for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&st->tau_max_bits, __float_as_uint(tmax));
        for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x)
            if (h_s[b]) atomicAdd(&st->hist[b], (unsigned long long)h_s[b]);
        if (threadIdx.x == 0) part[u] = Partial{x[0], 0.0, 0.0, 0.0, (long long)x[1], (long long)x[2]};
        if (!last_arrival(&st->ticket, (unsigned)s.unit_count)) continue;
        double tot[3];
        partial_totals<3>(part + s.unit_first, s.unit_count, tot, sh, [](const Partial& p, double (&y)[3]) {
            y[0] = p.s0; y[1] = (double)p.z; y[2] = (double)p.bad;
        });
        if (threadIdx.x == 0) {
            s_go = init_finish(st, tot[0], (long long)tot[1], (long long)tot[2]);
            if (!s_go) publish(st, results + s.state, true);
        }
        __syncthreads();
        if (s_go) proxy_start(st);
        __syncthreads();
    }
}

// One Halley pass over every request still iterating (PRECISE: the sum of e
// in double-float, which may end a request's iteration; else the MUFU form).
template <bool PRECISE>
__global__ void __launch_bounds__(kRfThreads) rf_halley_kernel(const unsigned char* __restrict__ step,
                                                             MFState* states, SlotResult* results, Partial* part)
{
    const View v(step);
    __shared__ double sh[4][32];
    __shared__ int s_skip;
    __shared__ double s_A;
    __shared__ float2 tab[PRECISE ? kExp2TabSize : 1];
    if constexpr (PRECISE) load_exp2_table(tab);
    for (int u = blockIdx.x; u < v.hdr->n_units; u += gridDim.x) {
        const RfUnit U = v.units[u];
        const RfSlot s = v.rf[U.rf];
        MFState* st = states + s.state;
        if (threadIdx.x == 0) {
            s_skip = st->done;
            s_A = st->A;
        }
        __syncthreads();
        if (s_skip) {
            __syncthreads();
            continue;
        }
        float a_hi, a_lo;
        split_rate(s_A, a_hi, a_lo);
        double x[4];
        if constexpr (PRECISE) {
            DFSum s0;
            KahanF32 s1;                              // g' enters the step's certificate
            float s2 = 0.f;
            stream_f32_steps(s.tau + U.begin, U.end - U.begin, threadIdx.x, blockDim.x, [&](float t) {
                float eh, el;
                exp2_neg_precise(t, a_hi, a_lo, tab, eh, el);
                s0.add(eh, el);
                const float te = t * eh;
                s1.add(te);
                s2 = fmaf(t, te, s2);
            }, [&] { s0.flush(); });
            x[0] = s0.value();
            x[1] = 0.0;
            x[2] = (double)s1.s - (double)s1.c;
            x[3] = (double)s2;
        } else {
            KahanF32 s0;
            float s0c = 0.f, s1 = 0.f, s2 = 0.f;
            stream_f32(s.tau + U.begin, U.end - U.begin, threadIdx.x, blockDim.x, [&](long long, float t) {
                float e, c;
                exp_neg(t, a_hi, a_lo, e, c);
                s0.add(e);
                s0c += c;
                const float te = t * e;
                s1 += te;
                s2 = fmaf(t, te, s2);
            });
            x[0] = (double)s0.value();
            x[1] = (double)s0c;
            x[2] = (double)s1;
            x[3] = (double)s2;
        }
        block_sum<4>(x, sh);
        if (threadIdx.x == 0) part[u] = Partial{x[0], x[1], x[2], x[3], 0, 0};
        if (!last_arrival(&st->ticket, (unsigned)s.unit_count)) continue;
        double tot[4];
        partial_totals<4>(part + s.unit_first, s.unit_count, tot, sh, [](const Partial& p, double (&y)[4]) {
            y[0] = p.s0; y[1] = p.s0c; y[2] = p.s1; y[3] = p.s2;
        });
        if (threadIdx.x == 0) {
            halley_update(st, tot[0], tot[1], tot[2], tot[3], PRECISE);
            if (st->done && st->status != LYA_OK) publish(st, results + s.state, true);
        }
        __syncthreads();
    }
}

// The flux pass: F = exp(-A tau), the check of g at that A, and the flux
// statistics of the request when the check passes.
__global__ void __launch_bounds__(kRfThreads) rf_flux_kernel(const unsigned char* __restrict__ step,
                                                           MFState* states, SlotResult* results, Partial* part,
                                                           StatPart* spart)
{
    const View v(step);
    // one private 21-bin counter row per thread (21 is odd: conflict-free)
    __shared__ unsigned int cnt[kRfThreads * 21];
    __shared__ double sh[4][32];
    __shared__ int s_skip;
    __shared__ double s_A;
    unsigned int* mine = cnt + threadIdx.x * 21;
    for (int u = blockIdx.x; u < v.hdr->n_units; u += gridDim.x) {
        const RfUnit U = v.units[u];
        const RfSlot s = v.rf[U.rf];
        MFState* st = states + s.state;
        if (threadIdx.x == 0) {
            // an error is final, and so is an F already written this step
            s_skip = (st->done && st->status != LYA_OK) || results[s.state].final;
            s_A = st->A;
        }
        __syncthreads();
        if (s_skip) {
            __syncthreads();
            continue;
        }
        for (int k = 0; k < 21; ++k) mine[k] = 0;
        float a_hi, a_lo;
        split_rate(s_A, a_hi, a_lo);
        KahanF32 s0, m1, m2;
        float s0c = 0.f;
        float* F = s.flux + U.begin;
        stream_f32(s.tau + U.begin, U.end - U.begin, threadIdx.x, blockDim.x, [&](long long i, float t) {
            float e, c;
            exp_neg(t, a_hi, a_lo, e, c);
            const float f = e + c;
            F[i] = f;
            s0.add(e);
            s0c += c;
            const float d = f - 0.5f;
            m1.add(d);
            m2.add(d * d);
            mine[pdf_bin(f)] += 1u;
        });
        double x[4] = {(double)s0.value(), (double)s0c, (double)m1.value(), (double)m2.value()};
        block_sum<4>(x, sh);                                  // ends with a barrier
        for (int k = threadIdx.x; k < 21; k += blockDim.x) {
            unsigned int c = 0;
            for (int r = 0; r < (int)blockDim.x; ++r) c += cnt[r * 21 + k];
            spart[u].pdf[k] = c;
        }
        if (threadIdx.x == 0) {
            part[u] = Partial{x[0], x[1], 0.0, 0.0, 0, 0};
            spart[u].m1 = x[2];
            spart[u].m2 = x[3];
        }
        if (!last_arrival(&st->ticket, (unsigned)s.unit_count)) continue;
        double tot[4];
        const Partial* pp = part + s.unit_first;
        const StatPart* sp = spart + s.unit_first;
        for (int k = 0; k < 4; ++k) tot[k] = 0.0;
        for (int b = threadIdx.x; b < s.unit_count; b += blockDim.x) {
            tot[0] += pp[b].s0;
            tot[1] += pp[b].s0c;
            tot[2] += sp[b].m1;
            tot[3] += sp[b].m2;
        }
        block_sum<4>(tot, sh);
        if (threadIdx.x == 0) {
            flux_update(st, tot[0], tot[1]);
            s_skip = !(st->done && st->status == LYA_OK);
        }
        __syncthreads();
        if (!s_skip) {
            SlotResult* res = results + s.state;
            for (int k = threadIdx.x; k < 21; k += blockDim.x) {
                unsigned long long c = 0;
                for (int b = 0; b < s.unit_count; ++b) c += sp[b].pdf[k];
                res->pdf[k] = c;
            }
            if (threadIdx.x == 0) {
                res->m1 = tot[2];
                res->m2 = tot[3];
                publish(st, res, true);
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t serve_state_bytes() { return sizeof(MFState); }
size_t serve_part_bytes() { return sizeof(Partial); }
size_t serve_spart_bytes() { return sizeof(StatPart); }

cudaError_t serve_rf_launch(const unsigned char* d_step, void* d_states, SlotResult* d_results, void* d_part,
                            void* d_spart, int grid, cudaStream_t stream, int* n_launched)
{
    MFState* st = static_cast<MFState*>(d_states);
    Partial* part = static_cast<Partial*>(d_part);
    StatPart* sp = static_cast<StatPart*>(d_spart);
    int n = 0;
    rf_reset_kernel<<<64, kRfThreads, 0, stream>>>(d_step, st, d_results);
    ++n;
    rf_init_kernel<<<grid, kRfThreads, 0, stream>>>(d_step, st, d_results, part);
    ++n;
    for (int r = 0; r < kRfRounds; ++r) {
        rf_halley_kernel<false><<<grid, kRfThreads, 0, stream>>>(d_step, st, d_results, part);
        rf_halley_kernel<true><<<grid, kRfThreads, 0, stream>>>(d_step, st, d_results, part);
        rf_flux_kernel<<<grid, kRfThreads, 0, stream>>>(d_step, st, d_results, part, sp);
        n += 3;
    }
    if (n_launched) *n_launched = n;
    return cudaGetLastError();
}

}  // namespace serve
}  // namespace lya
