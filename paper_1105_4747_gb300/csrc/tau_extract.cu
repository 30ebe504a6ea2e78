// tau_extract.cu -- optical depth along skewers (Eq. 4-6), sm_103a.
//
// One CTA owns one skewer.  The work per skewer is:
//   1. histogram of target pixels: source j lands in bin t_j = j + s_j (mod N)
//      with s_j = rint(v_j/du), the nearest pixel of u_j = v_H(j) + v_pec(j);
//   2. block scan -> bin starts, then a scatter of per-source records
//      {a_j, c_j r_j, w_j, j} into shared memory (a counting sort by target),
//      and a per-bin insertion sort on j so the order inside a bin -- and
//      with it the summation order -- does not depend on atomic timing;
//   3. for each output pixel i, the windowed pair sum over the sources whose
//      bins lie within W pixels of i (W = the skewer's largest
//      ceil((nsigma b_j + |r_j|)/du)), periodic over the skewer.
//
// Velocity differences are formed in a local frame: with s_j integer and
// r_j = v_j - s_j du (a double-float du keeps r_j exact to ~1 ulp), the
// Gaussian argument is c_j ((i - t_j) du - r_j) with an exact integer pixel
// offset, so FP32 never subtracts two velocities of size ~1e5 km/s.
//
// Per source (FP32, MUFU):  T_j = stored or T0 min(rho_j, pivot)^(gamma-1)
//   w_j = rho_j^2 (T_j/1e4)^-1.2          (n_HI / b of Eq. 4 and Eq. 6 up to K)
//   c_j = sqrt(log2 e) / b_j,  a_j = c_j du,   so exp(-(d/b)^2) = 2^-(c d)^2.
// Per pair: x = fma(m, a_j, -c_j r_j); tau += w_j * ex2(-x*x).
#include <cfloat>
#include <cstdint>

#include "lya_device.cuh"
#include "lya_internal.h"

namespace lya {
namespace {

constexpr float kLog2_1e4 = 13.287712379549449f;   // log2(1e4)

template <int PREC> struct Prec;

template <> struct Prec<LYA_PREC_F32_COMPENSATED> {
    using Rec = float4;
    using Acc = KahanF32;
    __device__ static void add(Acc& a, float x) { a.add(x); }
    __device__ static float value(const Acc& a) { return a.value(); }
};

struct NaiveF32 { float s = 0.f; };
template <> struct Prec<LYA_PREC_F32_NAIVE> {
    using Rec = float4;
    using Acc = NaiveF32;
    __device__ static void add(Acc& a, float x) { a.s = __fadd_rn(a.s, x); }
    __device__ static float value(const Acc& a) { return a.s; }
};

struct PlainF64 { double s = 0.0; };
template <> struct Prec<LYA_PREC_F64> {
    using Rec = double4_32a;
    using Acc = PlainF64;
    __device__ static void add(Acc& a, double x) { a.s += x; }
    __device__ static double value(const Acc& a) { return a.s; }
};

__device__ __forceinline__ int wrap_pixel(int64_t x, int N)
{
    int64_t r = x % N;
    return (int)(r < 0 ? r + N : r);
}

// ---- per-source preparation -------------------------------------------------
struct SrcF32 { float a, bb, w; int t, h; };

__device__ __forceinline__ float target_shift_f32(float v, const TauLaunch& L)
{
    return rintf(v * L.inv_du);
}

__device__ __forceinline__ SrcF32 prep_f32(const TauLaunch& L, float rho, float v, float T, int j)
{
    SrcF32 s;
    if (L.t_mode != 0) T = L.T0 * ex2(L.gm1 * lg2(fminf(rho, L.pivot)));
    const float lt = lg2(T) - kLog2_1e4;                 // log2(T / 1e4 K)
    s.w = rho * rho * ex2(-1.2f * lt);                   // rho^2 (T/1e4)^-0.7 / (T/1e4)^0.5
    const float c = L.c_coef * ex2(-0.5f * lt);          // sqrt(log2 e) / b
    const float sf = target_shift_f32(v, L);
    float r = fmaf(-sf, L.du_hi, v);                     // exact product inside the fma
    r = fmaf(-sf, L.du_lo, r);
    s.t = wrap_pixel((int64_t)j + (int64_t)sf, L.n_pix);
    s.a = c * L.du_hi;
    s.bb = c * r;
    // |m du - r| <= nsigma b needs |m| <= (nsigma b + |r|)/du, and nsigma b/du =
    // h_coef/a; the 1e-5 margin covers the approximate reciprocal
    const float hx = (L.h_coef * rcp_approx(s.a) + fabsf(r) * L.inv_du) * 1.00001f;
    s.h = min((int)fminf(hx, (float)L.n_pix), L.w_max);
    return s;
}

struct SrcF64 { double a, bb, w; int t, h; };

__device__ __forceinline__ SrcF64 prep_f64(const TauLaunch& L, float rho_f, float v_f, float T_f, int j)
{
    SrcF64 s;
    const double rho = rho_f, v = v_f;
    double T = T_f;
    if (L.t_mode != 0) T = L.T0_d * pow(fmin(rho, L.pivot_d), L.gm1_d);
    const double tt = T * 1e-4;
    s.w = rho * rho * pow(tt, -1.2);
    const double c = L.c_coef_d / sqrt(tt);
    const double sf = rint(v * L.inv_du_d);
    const double r = v - sf * L.du_d;
    s.t = wrap_pixel((int64_t)j + (int64_t)sf, L.n_pix);
    s.a = c * L.du_d;
    s.bb = c * r;
    const double hx = (L.h_coef_d / s.a + fabs(r) * L.inv_du_d) * (1.0 + 1e-12);
    s.h = min((int)fmin(hx, (double)L.n_pix), L.w_max);
    return s;
}

// ---- the pair sum over one contiguous run of sorted sources -------------------
template <int PREC>
__device__ __forceinline__ void pair_segment(const typename Prec<PREC>::Rec* __restrict__ rec,
                                             int k0, int k1, float fi, typename Prec<PREC>::Acc& acc)
{
    for (int k = k0; k < k1; ++k) {
        const float4 r = rec[k];                 // {a, c r, w, t}
        const float m = fi - r.w;                // exact: integers below 2^24
        const float x = fmaf(m, r.x, -r.y);
        const float e = ex2(-(x * x));
        Prec<PREC>::add(acc, r.z * e);
    }
}

template <>
__device__ __forceinline__ void pair_segment<LYA_PREC_F64>(const double4_32a* __restrict__ rec,
                                                           int k0, int k1, float fi, PlainF64& acc)
{
    const double di = fi;
    for (int k = k0; k < k1; ++k) {
        const double4_32a r = rec[k];
        const double x = (di - r.w) * r.x - r.y;
        acc.s += r.z * exp2(-(x * x));
    }
}

template <int PREC>
__global__ void __launch_bounds__(512) tau_kernel(const TauLaunch L)
{
    using Rec = typename Prec<PREC>::Rec;
    using Acc = typename Prec<PREC>::Acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int warp_tot[33];
    __shared__ int s_hmax;

    const int N = L.n_pix;
    const int tid = threadIdx.x, nt = blockDim.x;
    Rec* rec = reinterpret_cast<Rec*>(smem_raw);
    int* bin = reinterpret_cast<int*>(smem_raw + sizeof(Rec) * (size_t)N);   // N + 1 ints

    const int64_t row = blockIdx.x;
    const int64_t sk = L.ids ? L.ids[row] : row;
    float* out = L.tau_out + row * (int64_t)N;
    if (sk < 0 || sk >= L.n_skewers) {
        for (int i = tid; i < N; i += nt) out[i] = 0.f;
        if (tid == 0) atomicOr(L.err, 1);
        return;
    }
    const float* __restrict__ rho = L.rho + sk * (int64_t)N;
    const float* __restrict__ vpec = L.vpec + sk * (int64_t)N;
    const float* __restrict__ temp = L.temp ? L.temp + sk * (int64_t)N : nullptr;

    // 1. zero the bins; histogram of target pixels
    for (int k = tid; k <= N; k += nt) bin[k] = 0;
    if (tid == 0) s_hmax = 0;
    __syncthreads();
    for (int j = tid; j < N; j += nt) {
        const float r = rho[j];
        if (r > 0.f) {
            const float v = vpec[j];
            int t;
            if (PREC == LYA_PREC_F64) t = wrap_pixel((int64_t)j + (int64_t)rint((double)v * L.inv_du_d), N);
            else t = wrap_pixel((int64_t)j + (int64_t)target_shift_f32(v, L), N);
            atomicAdd(&bin[t + 1], 1);
        }
    }
    __syncthreads();

    // 2. bin[t+1] = start(t); scatter records, bin[t+1] ends at start(t+1)
    const int nsrc = block_exclusive_scan(bin + 1, N, warp_tot);
    int hmax = 0;
    for (int j = tid; j < N; j += nt) {
        const float r = rho[j];
        if (!(r > 0.f)) continue;
        const float v = vpec[j];
        const float T = temp ? temp[j] : 0.f;
        if constexpr (PREC == LYA_PREC_F64) {
            const SrcF64 s = prep_f64(L, r, v, T, j);
            const int pos = atomicAdd(&bin[s.t + 1], 1);
            if (pos >= N) { atomicOr(L.err, 2); continue; }   // input changed under the kernel
            rec[pos] = make_double4_32a(s.a, s.bb, s.w, (double)j);
            hmax = max(hmax, s.h);
        } else {
            const SrcF32 s = prep_f32(L, r, v, T, j);
            const int pos = atomicAdd(&bin[s.t + 1], 1);
            if (pos >= N) { atomicOr(L.err, 2); continue; }   // input changed under the kernel
            rec[pos] = make_float4(s.a, s.bb, s.w, (float)j);
            hmax = max(hmax, s.h);
        }
    }
    atomicMax(&s_hmax, hmax);
    __syncthreads();

    // 3. deterministic order inside each bin (by source pixel), then key := target
    for (int t = tid; t < N; t += nt) {
        const int b0 = bin[t], b1 = bin[t + 1];
        for (int k = b0 + 1; k < b1; ++k) {
            const Rec x = rec[k];
            int q = k - 1;
            while (q >= b0 && rec[q].w > x.w) { rec[q + 1] = rec[q]; --q; }
            rec[q + 1] = x;
        }
        for (int k = b0; k < b1; ++k) rec[k].w = (float)t;
    }
    __syncthreads();

    // 4. windowed periodic pair sum
    const int W = min(s_hmax, (N - 1) / 2);
    const float K = L.K;
    for (int i = tid; i < N; i += nt) {
        Acc acc;
        const float fi = (float)i;
        const int lo = i - W, hi = i + W;
        if (lo < 0) {
            pair_segment<PREC>(rec, bin[lo + N], nsrc, fi + (float)N, acc);
            pair_segment<PREC>(rec, 0, bin[hi + 1], fi, acc);
        } else if (hi >= N) {
            pair_segment<PREC>(rec, bin[lo], nsrc, fi, acc);
            pair_segment<PREC>(rec, 0, bin[hi - N + 1], fi - (float)N, acc);
        } else {
            pair_segment<PREC>(rec, bin[lo], bin[hi + 1], fi, acc);
        }
        if constexpr (PREC == LYA_PREC_F64) out[i] = (float)(L.K_d * Prec<PREC>::value(acc));
        else out[i] = K * Prec<PREC>::value(acc);
    }
}

// ---- adaptive-window kernel -------------------------------------------------------
//
// Each source j covers the output pixels |i - t_j| <= h_j.  Instead of one
// window for the whole skewer, every output pixel i gets the tightest run of
// target bins [L_i, R_i] that still contains every source covering it:
//   L_i = first bin t with max_{t' <= t}(t' + h_t') >= i   (prefix max of right reach)
//   R_i = last  bin t with min_{t' >= t}(t' - h_t') <= i   (suffix min of left reach)
// computed on bins extended by w_max on both sides so the periodic wrap is
// explicit.  The sources in [L_i, R_i] are a superset of the pairs with
// |v_H(i) - u_j| <= nsigma b_j; outside the neighbourhood of the broadest
// lines the run is ~2 h + 1 sources long.
//
// Shared memory: records (N) | bin starts (N+1) | aux (N ints: packed
// target/half-width while sorting, then L_i and R_i as int16) | reach (N + 2 w_max).
constexpr int kReachLow = -(1 << 28);
constexpr int kReachHigh = 1 << 28;

template <int PREC, int MAXQ>
__global__ void __launch_bounds__(512) tau_env_kernel(const TauLaunch L)
{
    using Rec = typename Prec<PREC>::Rec;
    using Acc = typename Prec<PREC>::Acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int warp_tot[33];

    const int N = L.n_pix;
    const int Wd = L.w_max;
    const int NE = N + 2 * Wd;
    const int tid = threadIdx.x, nt = blockDim.x;
    Rec* rec = reinterpret_cast<Rec*>(smem_raw);
    int* bin = reinterpret_cast<int*>(smem_raw + sizeof(Rec) * (size_t)N);   // N + 1
    int* aux = bin + (N + 1);                                                 // N
    int* reach = aux + N;                                                     // NE
    short* Lb = reinterpret_cast<short*>(aux);
    short* Rb = Lb + N;

    const int64_t row = blockIdx.x;
    const int64_t sk = L.ids ? L.ids[row] : row;
    float* out = L.tau_out + row * (int64_t)N;
    if (sk < 0 || sk >= L.n_skewers) {
        for (int i = tid; i < N; i += nt) out[i] = 0.f;
        if (tid == 0) atomicOr(L.err, 1);
        return;
    }
    const float* __restrict__ rho = L.rho + sk * (int64_t)N;
    const float* __restrict__ vpec = L.vpec + sk * (int64_t)N;
    const float* __restrict__ temp = L.temp ? L.temp + sk * (int64_t)N : nullptr;

    // 1. inputs into registers (coalesced), histogram of target pixels
    float r_[MAXQ], v_[MAXQ], T_[MAXQ];
    int t_[MAXQ];
    for (int k = tid; k <= N; k += nt) bin[k] = 0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        const int j = tid + q * nt;
        r_[q] = 0.f;
        if (j < N) {
            r_[q] = rho[j];
            v_[q] = vpec[j];
            T_[q] = temp ? temp[j] : 0.f;
            if (r_[q] > 0.f) {
                if constexpr (PREC == LYA_PREC_F64)
                    t_[q] = wrap_pixel((int64_t)j + (int64_t)rint((double)v_[q] * L.inv_du_d), N);
                else
                    t_[q] = wrap_pixel((int64_t)j + (int64_t)target_shift_f32(v_[q], L), N);
                atomicAdd(&bin[t_[q] + 1], 1);
            }
        }
    }
    __syncthreads();

    // 2. bin starts; scatter records {a, c r, w, j} and (target, half-width)
    const int nsrc = block_exclusive_scan(bin + 1, N, warp_tot);
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        const int j = tid + q * nt;
        if (j >= N || !(r_[q] > 0.f)) continue;
        int pos, t, h;
        if constexpr (PREC == LYA_PREC_F64) {
            const SrcF64 s = prep_f64(L, r_[q], v_[q], T_[q], j);
            t = s.t; h = s.h;
            pos = atomicAdd(&bin[t + 1], 1);
            if (pos >= N) { atomicOr(L.err, 2); continue; }
            rec[pos] = make_double4_32a(s.a, s.bb, s.w, (double)j);
        } else {
            const SrcF32 s = prep_f32(L, r_[q], v_[q], T_[q], j);
            t = s.t; h = s.h;
            pos = atomicAdd(&bin[t + 1], 1);
            if (pos >= N) { atomicOr(L.err, 2); continue; }
            rec[pos] = make_float4(s.a, s.bb, s.w, (float)j);
        }
        aux[pos] = (t << 16) | h;
    }
    for (int e = tid; e < NE; e += nt) reach[e] = kReachLow;
    __syncthreads();

    // 3. order inside each bin by source pixel j: rank by counting (parallel,
    //    deterministic), then write back with the key replaced by the target
    Rec rr[MAXQ];
    int np[MAXQ], th[MAXQ];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        const int k = tid + q * nt;
        np[q] = -1;
        if (k < nsrc) {
            rr[q] = rec[k];
            th[q] = aux[k];
            const int t = th[q] >> 16;
            const int b0 = bin[t], b1 = bin[t + 1];
            int rank = 0;
            if (b1 - b0 > 1)
                for (int k2 = b0; k2 < b1; ++k2) rank += rec[k2].w < rr[q].w;
            np[q] = b0 + rank;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        if (np[q] < 0) continue;
        const int t = th[q] >> 16, h = th[q] & 0xffff;
        rr[q].w = (float)t;
        rec[np[q]] = rr[q];
        atomicMax(&reach[t + Wd], t + h);
        if (t >= N - Wd) atomicMax(&reach[t - N + Wd], t - N + h);
        if (t < Wd) atomicMax(&reach[t + N + Wd], t + N + h);
    }
    __syncthreads();

    // 4. L_i from the prefix max of the right reach
    block_prefix_max(reach, NE, warp_tot, kReachLow);
    for (int i = tid; i < N; i += nt) Lb[i] = (short)(i + 1);
    __syncthreads();
    for (int e = tid; e < NE; e += nt) {
        const int prev = e ? reach[e - 1] : kReachLow;
        const int lo = max(prev + 1, 0), hi = min(reach[e], N - 1);
        for (int i = lo; i <= hi; ++i) Lb[i] = (short)(e - Wd);
    }
    __syncthreads();
    for (int e = tid; e < NE; e += nt) reach[e] = kReachHigh;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        if (np[q] < 0) continue;
        const int t = th[q] >> 16, h = th[q] & 0xffff;
        atomicMin(&reach[t + Wd], t - h);
        if (t >= N - Wd) atomicMin(&reach[t - N + Wd], t - N - h);
        if (t < Wd) atomicMin(&reach[t + N + Wd], t + N - h);
    }
    __syncthreads();

    // 5. R_i from the suffix min of the left reach
    block_suffix_min(reach, NE, warp_tot, kReachHigh);
    for (int i = tid; i < N; i += nt) Rb[i] = (short)(i - 1);
    __syncthreads();
    for (int e = tid; e < NE; e += nt) {
        const int next = e + 1 < NE ? reach[e + 1] : kReachHigh;
        const int lo = max(reach[e], 0), hi = min(next - 1, N - 1);
        for (int i = lo; i <= hi; ++i) Rb[i] = (short)(e - Wd);
    }
    __syncthreads();

    // 6. pair sums over [L_i, R_i], split where the run crosses the periodic seam
    for (int i = tid; i < N; i += nt) {
        Acc acc;
        const float fi = (float)i;
        const int lx = Lb[i], rx = Rb[i];
        if (lx <= rx) {
            if (lx < 0) {
                const int u1 = min(rx, -1);
                pair_segment<PREC>(rec, bin[lx + N], bin[u1 + N + 1], fi + (float)N, acc);
            }
            const int a0 = max(lx, 0), a1 = min(rx, N - 1);
            if (a0 <= a1) pair_segment<PREC>(rec, bin[a0], bin[a1 + 1], fi, acc);
            if (rx >= N) {
                const int u0 = max(lx, N) - N;
                pair_segment<PREC>(rec, bin[u0], bin[rx - N + 1], fi - (float)N, acc);
            }
        }
        if constexpr (PREC == LYA_PREC_F64) out[i] = (float)(L.K_d * Prec<PREC>::value(acc));
        else out[i] = L.K * Prec<PREC>::value(acc);
    }
}

int block_threads(int n_pix)
{
    if (n_pix >= 2048) return 512;
    if (n_pix >= 512) return 256;
    return 128;
}

}  // namespace

static size_t rec_bytes(int precision)
{
    return precision == LYA_PREC_F64 ? sizeof(double4_32a) : sizeof(float4);
}

// Adaptive-window layout: records, bin starts, aux, reach.
static size_t env_smem_bytes(int n_pix, int w_max, int precision)
{
    return rec_bytes(precision) * (size_t)n_pix + sizeof(int) * (size_t)(n_pix + 1) +
           sizeof(int) * (size_t)n_pix + sizeof(int) * (size_t)(n_pix + 2 * w_max);
}

// Whole-skewer-window layout: records, bin starts.
static size_t global_smem_bytes(int n_pix, int precision)
{
    return rec_bytes(precision) * (size_t)n_pix + sizeof(int) * (size_t)(n_pix + 1);
}

static bool use_env(int n_pix, int w_max, int precision)
{
    return n_pix <= 4096 && env_smem_bytes(n_pix, w_max, precision) <= max_dynamic_smem();
}

size_t tau_smem_bytes(int n_pix, int w_max, int precision)
{
    return use_env(n_pix, w_max, precision) ? env_smem_bytes(n_pix, w_max, precision)
                                            : global_smem_bytes(n_pix, precision);
}

template <typename K>
static cudaError_t launch_kernel(K kernel, const TauLaunch& L, size_t smem, cudaStream_t stream)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    if (L.n_rows == 0) return cudaSuccess;
    kernel<<<(unsigned)L.n_rows, block_threads(L.n_pix), smem, stream>>>(L);
    count_launch();
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_prec(const TauLaunch& L, cudaStream_t stream)
{
    if (!use_env(L.n_pix, L.w_max, PREC))
        return launch_kernel(tau_kernel<PREC>, L, global_smem_bytes(L.n_pix, PREC), stream);
    const size_t smem = env_smem_bytes(L.n_pix, L.w_max, PREC);
    const int q = (L.n_pix + block_threads(L.n_pix) - 1) / block_threads(L.n_pix);
    if (q <= 4) return launch_kernel(tau_env_kernel<PREC, 4>, L, smem, stream);
    return launch_kernel(tau_env_kernel<PREC, 8>, L, smem, stream);
}

cudaError_t launch_tau(const TauLaunch& L, int precision, cudaStream_t stream)
{
    switch (precision) {
    case LYA_PREC_F32_COMPENSATED: return launch_prec<LYA_PREC_F32_COMPENSATED>(L, stream);
    case LYA_PREC_F32_NAIVE: return launch_prec<LYA_PREC_F32_NAIVE>(L, stream);
    case LYA_PREC_F64: return launch_prec<LYA_PREC_F64>(L, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lya
