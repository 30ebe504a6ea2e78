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
// Precision: the per-pixel exponential is FP32 (MUFU ex2) of a double-float
// argument y = tau * A log2(e) = y_hi + y_lo, i.e. e = 2^-y_hi (1 - y_lo ln 2);
// each thread accumulates in compensated FP32, CTAs and the final sum in FP64.
// The 2^-y_hi part and its first-order correction are summed separately, so
// g(A) stays smooth in A far below FP32 resolution and the FP64 Newton can
// reach |g| <= 1e-12.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "lya_device.cuh"
#include "lya_internal.h"

namespace lya {
namespace {

constexpr int kThreads = 256;
constexpr double kLog2e = 1.4426950408889634;
constexpr float kLn2f = 0.69314718055994531f;

struct MFState {
    double A, lo, hi, g, mean_tau, Ft, tol;
    double a_hi_unused;
    long long n, n_zero, n_bad;
    int iter, max_iter, done, status;   // status: LYA_OK / LYA_EINVAL / LYA_ENOCONV
    unsigned int ticket;
};

struct Partial {
    double s0, s0c, s1;
    long long z, bad;
};

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of a few values; result valid on thread 0.
template <int K>
__device__ void block_sum(double (&v)[K], double (*sh)[32])
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
}

// Returns true on exactly one block: the last to arrive.
__device__ bool last_block(unsigned int* ticket)
{
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// ---- init pass: <tau>, zero and invalid counts, A0 -------------------------------
__global__ void __launch_bounds__(kThreads) mf_init_kernel(const float* __restrict__ tau, long long n,
                                                         MFState* st, Partial* part)
{
    KahanF32 s;
    long long z = 0, bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float t = tau[i];
        if (!(t >= 0.f) || !isfinite(t)) { ++bad; continue; }
        s.add(t);
        z += (t == 0.f);
    }
    __shared__ double sh[3][32];
    double v[3] = {(double)s.value(), (double)z, (double)bad};
    block_sum<3>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = Partial{v[0], 0.0, 0.0, (long long)v[1], (long long)v[2]};
    if (!last_block(&st->ticket)) return;
    if (threadIdx.x != 0) return;
    double sum = 0.0;
    long long zz = 0, bb = 0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
        sum += part[b].s0;
        zz += part[b].z;
        bb += part[b].bad;
    }
    st->ticket = 0;
    st->n_zero = zz;
    st->n_bad = bb;
    st->mean_tau = sum / (double)n;
    st->iter = 0;
    if (bb > 0 || !(st->mean_tau > 0.0)) {
        st->status = LYA_EINVAL;
        st->done = 1;
        return;
    }
    if ((double)zz / (double)n >= st->Ft) {       // <e^{-A tau}> >= zero fraction for all A
        st->status = LYA_ENOCONV;
        st->done = 1;
        return;
    }
    st->A = -log(st->Ft) / st->mean_tau;
    st->lo = st->A;
    st->hi = INFINITY;
    st->status = LYA_ENOCONV;                    // until converged
    st->done = 0;
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

// ---- one Newton pass -----------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) mf_newton_kernel(const float* __restrict__ tau, long long n,
                                                           MFState* st, Partial* part)
{
    if (st->done) return;
    float a_hi, a_lo;
    split_rate(st->A, a_hi, a_lo);
    KahanF32 s0;
    float s0c = 0.f, s1 = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float t = tau[i];
        float e, c;
        exp_neg(t, a_hi, a_lo, e, c);
        s0.add(e);
        s0c += c;
        s1 = fmaf(t, e, s1);
    }
    __shared__ double sh[3][32];
    double v[3] = {(double)s0.value(), (double)s0c, (double)s1};
    block_sum<3>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = Partial{v[0], v[1], v[2], 0, 0};
    if (!last_block(&st->ticket)) return;
    if (threadIdx.x != 0) return;
    double S0 = 0.0, S0c = 0.0, S1 = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
        S0 += part[b].s0;
        S0c += part[b].s0c;
        S1 += part[b].s1;
    }
    st->ticket = 0;
    const double nn = (double)n;
    const double g = (S0 + S0c) / nn - st->Ft;
    const double gp = -S1 / nn;
    const double A = st->A;
    st->g = g;
    st->iter += 1;
    if (fabs(g) <= st->tol) {
        st->status = LYA_OK;
        st->done = 1;
        return;
    }
    if (g > 0.0) st->lo = A; else st->hi = A;
    double An = gp < 0.0 ? A - g / gp : NAN;
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

// ---- F = exp(-A tau) ---------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) mf_flux_kernel(const float* __restrict__ tau, long long n,
                                                         const MFState* st, float* __restrict__ F)
{
    if (st->status != LYA_OK) return;
    float a_hi, a_lo;
    split_rate(st->A, a_hi, a_lo);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float e, c;
        exp_neg(tau[i], a_hi, a_lo, e, c);
        F[i] = e + c;
    }
}

// ---- flux statistics -----------------------------------------------------------------
struct StatsOut {
    double m1, m2;                // sums of (F - 0.5) and (F - 0.5)^2
    unsigned long long pdf[21];
    unsigned int ticket;
};

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

__global__ void __launch_bounds__(kThreads) stats_kernel(const float* __restrict__ F, long long n,
                                                       StatsOut* out, double* part)
{
    __shared__ unsigned int hist[21];
    for (int k = threadIdx.x; k < 21; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    KahanF32 m1, m2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float f = F[i];
        const float d = f - 0.5f;
        m1.add(d);
        m2.add(d * d);
        atomicAdd(&hist[pdf_bin(f)], 1u);
    }
    __shared__ double sh[2][32];
    double v[2] = {(double)m1.value(), (double)m2.value()};
    block_sum<2>(v, sh);
    __syncthreads();
    for (int k = threadIdx.x; k < 21; k += blockDim.x)
        if (hist[k]) atomicAdd(&out->pdf[k], (unsigned long long)hist[k]);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = v[0];
        part[2 * blockIdx.x + 1] = v[1];
    }
    if (!last_block(&out->ticket)) return;
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    out->m1 = a;
    out->m2 = b;
    out->ticket = 0;
}

// ---- field validation ---------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) field_check_kernel(const float* __restrict__ rho,
                                                             const float* __restrict__ v,
                                                             const float* __restrict__ T, long long n,
                                                             FieldCheck* out)
{
    unsigned long long br = 0, bv = 0, bt = 0;
    float tmax = 0.f, rmax = 0.f, rmin = INFINITY;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float r = rho[i], u = v[i];
        const bool rok = r >= 0.f && isfinite(r);
        br += !rok;
        bv += !(isfinite(u) && fabsf(u) < 2.99792458e5f);
        if (rok && r > 0.f) {
            rmax = fmaxf(rmax, r);
            rmin = fminf(rmin, r);
        }
        if (T) {
            const float t = T[i];
            const bool ok = isfinite(t) && (t > 0.f || !(r > 0.f));
            bt += !ok;
            if (ok && r > 0.f) tmax = fmaxf(tmax, t);
        }
    }
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
    const long long cap = 8LL * sm_count();
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

int sm_count()
{
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

size_t max_dynamic_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

cudaError_t launch_field_check(const float* rho, const float* vpec, const float* temp, int64_t n,
                               FieldCheck* d_out, cudaStream_t stream)
{
    FieldCheck init{};
    init.rho_minpos_bits = 0x7f800000u;     // +inf
    cudaError_t e = cudaMemcpyAsync(d_out, &init, sizeof(FieldCheck), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // init is a stack value
    if (e != cudaSuccess || n == 0) return e;
    field_check_kernel<<<grid_for(n), kThreads, 0, stream>>>(rho, vpec, temp, n, d_out);
    count_launch();
    return cudaGetLastError();
}

#define LYA_TRY(call)                                   \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) { err = _e; goto done; } \
    } while (0)

lya_status mean_flux_solve(const float* tau, int64_t n, double target, double tol, int max_iter,
                           double* A_out, float* flux_out, cudaStream_t stream)
{
    const int grid = grid_for(n);
    MFState* st = nullptr;
    Partial* part = nullptr;
    MFState h{};
    cudaError_t err = cudaSuccess;
    lya_status result = LYA_OK;
    h.Ft = target;
    h.tol = tol;
    h.n = n;
    h.max_iter = max_iter;
    h.status = LYA_ENOCONV;
    LYA_TRY(cudaMallocAsync((void**)&st, sizeof(MFState), stream));
    LYA_TRY(cudaMallocAsync((void**)&part, sizeof(Partial) * grid, stream));
    LYA_TRY(cudaMemcpyAsync(st, &h, sizeof(MFState), cudaMemcpyHostToDevice, stream));
    mf_init_kernel<<<grid, kThreads, 0, stream>>>(tau, n, st, part);
    count_launch();
    LYA_TRY(cudaGetLastError());
    // Newton typically converges in 3-6 passes: launch them in batches and
    // read the state back once per batch.
    for (int launched = 0; launched < max_iter;) {
        const int batch = launched == 0 ? 6 : 4;
        for (int b = 0; b < batch && launched < max_iter; ++b, ++launched) {
            mf_newton_kernel<<<grid, kThreads, 0, stream>>>(tau, n, st, part);
            count_launch();
            LYA_TRY(cudaGetLastError());
        }
        LYA_TRY(cudaMemcpyAsync(&h, st, sizeof(MFState), cudaMemcpyDeviceToHost, stream));
        LYA_TRY(cudaStreamSynchronize(stream));
        if (h.done) break;
    }
    if (!h.done) {
        result = LYA_ENOCONV;
    } else {
        result = (lya_status)h.status;
    }
    if (result == LYA_OK) {
        *A_out = h.A;
        if (flux_out) {
            mf_flux_kernel<<<grid, kThreads, 0, stream>>>(tau, n, st, flux_out);
            count_launch();
            LYA_TRY(cudaGetLastError());
        }
    }
done:
    if (st) cudaFreeAsync(st, stream);
    if (part) cudaFreeAsync(part, stream);
    if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA;
    cudaError_t e2 = cudaStreamSynchronize(stream);
    if (e2 != cudaSuccess) return LYA_ECUDA;
    return result;
}

lya_status flux_stats_run(const float* flux, int64_t n, lya_flux_stats_t* out, cudaStream_t stream)
{
    const int grid = grid_for(n);
    StatsOut* d = nullptr;
    double* part = nullptr;
    StatsOut h{};
    cudaError_t err = cudaSuccess;
    LYA_TRY(cudaMallocAsync((void**)&d, sizeof(StatsOut), stream));
    LYA_TRY(cudaMallocAsync((void**)&part, sizeof(double) * 2 * grid, stream));
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
// For callers that cannot allocate device memory: code running while a CUDA
// graph is being captured into a pool they do not own, plug-ins whose host
// application forbids allocation after start-up, or callers on a memory
// budget that is already fully handed out.  The Newton state and the per-CTA
// partials live in a fixed file-scope device array instead of stream-ordered
// allocations.  The array is kNoAllocScratchBytes (64 KiB) on every GPU that
// loads the library and stays there until the process exits; it fits the
// state plus kNoAllocMaxBlocks partials, so the reduction grid is capped at
// kNoAllocMaxBlocks CTAs (the grid-stride loops still cover any n).
//
// Every call shares the one array and rewrites the whole state it reads (the
// state is copied in from the host at the start of each call, and every
// partial is written before it is read), so nothing is left over from a
// previous call.  Two calls whose work overlaps on the GPU (different streams,
// or different host threads on one device) race on the array.
namespace lya {
namespace {

constexpr size_t kNoAllocScratchBytes = 64 * 1024;
constexpr int kNoAllocMaxBlocks = 1024;
constexpr size_t kNoAllocStateBytes = 256;      // MFState, padded to the array's alignment
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
    cudaError_t err = noalloc_scratch(&scratch);
    if (err != cudaSuccess) return LYA_ECUDA;
    const int grid = grid_for(n) < kNoAllocMaxBlocks ? grid_for(n) : kNoAllocMaxBlocks;
    if (kNoAllocStateBytes + (size_t)grid * sizeof(Partial) > kNoAllocScratchBytes) return LYA_EINVAL;
    MFState* st = static_cast<MFState*>(scratch);
    Partial* part = reinterpret_cast<Partial*>(static_cast<unsigned char*>(scratch) + kNoAllocStateBytes);
    MFState h{};
    h.Ft = target;
    h.tol = tol;
    h.n = n;
    h.max_iter = max_iter;
    h.status = LYA_ENOCONV;
    lya_status result = LYA_OK;
    err = cudaMemcpyAsync(st, &h, sizeof(MFState), cudaMemcpyHostToDevice, stream);
    if (err != cudaSuccess) return LYA_ECUDA;
    mf_init_kernel<<<grid, kThreads, 0, stream>>>(tau, n, st, part);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return LYA_ECUDA;
    for (int launched = 0; launched < max_iter;) {
        const int batch = launched == 0 ? 6 : 4;
        for (int b = 0; b < batch && launched < max_iter; ++b, ++launched) {
            mf_newton_kernel<<<grid, kThreads, 0, stream>>>(tau, n, st, part);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) return LYA_ECUDA;
        }
        err = cudaMemcpyAsync(&h, st, sizeof(MFState), cudaMemcpyDeviceToHost, stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
        if (err != cudaSuccess) return LYA_ECUDA;
        if (h.done) break;
    }
    result = h.done ? (lya_status)h.status : LYA_ENOCONV;
    if (result == LYA_OK) {
        *A_out = h.A;
        if (flux_out) {
            mf_flux_kernel<<<grid, kThreads, 0, stream>>>(tau, n, st, flux_out);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) return LYA_ECUDA;
            if (cudaStreamSynchronize(stream) != cudaSuccess) return LYA_ECUDA;
        }
    }
    return result;
}

}  // namespace lya
