// tau_extract.cu -- optical depth along skewers (Eq. 4-6), sm_103a.
//
// Three kernels:
//   * tau_tile_kernel (FP32, the product path): one CTA per skewer (1,024
//     threads above 4,096 pixels, else 512 or fewer); sources counting-sorted
//     by target pixel; each eight-pixel tile finds the run of sources whose
//     reach covers it; four lanes share a tile (two lanes of four pixels
//     where the runs are long), taken in order of run length, and sum the
//     run (compensated or plain);
//   * tau_serve_kernel (the serving loop): the same per-skewer body run by
//     1 to 8 warp groups of a persistent 1024-thread CTA over a work list;
//   * tau_kernel (FP64 comparator): one CTA per skewer; sources
//     counting-sorted by target pixel, then each output pixel sums the
//     sources of the bins within the skewer's widest reach.
//
// Source j lands at the target pixel t_j = j + s_j (mod N), s_j = rint(v_j/du),
// the pixel nearest u_j = v_H(j) + v_pec(j).  Velocity differences are formed
// in a local frame: with s_j integer and r_j = v_j - s_j du (a double-float du
// keeps r_j exact to ~1 ulp), the Gaussian argument is c_j (m du - r_j) with
// an exact integer pixel offset m, so FP32 never subtracts two velocities of
// size ~1e5 km/s.
//
// Per source (FP32, MUFU):  T_j = stored or T0 min(rho_j, pivot)^(gamma-1)
//   w_j = rho_j^2 (T_j/1e4)^-1.2          (n_HI / b of Eq. 4 and Eq. 6 up to K)
//   c_j = sqrt(log2 e) / b_j,  a_j = c_j du,   so exp(-(d/b)^2) = 2^-(c d)^2.
// Per pair: x = fma(m, a_j, -c_j r_j); tau += ex2(lw_j - x*x), lw_j = log2 w_j
// (the pixel-averaged profile: w_j times a difference of two erfc).
#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "lya_device.cuh"
#include "lya_internal.h"
#include "serve_internal.h"

// LYA_CHECKED builds (a stand-in for a memory checker): every shared-memory
// index of the tile gather is checked before use, and a failed check sets
// bit 2 (value 4) of the launch's error word instead of trapping.
#ifdef LYA_CHECKED
#define LYA_BOUND(cond)                       \
    do {                                      \
        if (!(cond)) atomicOr(L.err, 4);      \
    } while (0)
#else
#define LYA_BOUND(cond) \
    do {                \
    } while (0)
#endif

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

// x mod N in [0, N) for |x| < 2^30 (the host bounds |v_pec|/du below 2^22);
// one wrap either way is a compare and an add, farther ones a division.
__device__ __forceinline__ int wrap_pixel(int x, int N)
{
    if (x < 0) x += N;
    else if (x >= N) x -= N;
    if ((unsigned)x >= (unsigned)N) {
        x %= N;
        if (x < 0) x += N;
    }
    return x;
}

// ---- per-source preparation -------------------------------------------------
// lw = log2 of the source's weight rho^2 (T/1e4)^-0.7 / (T/1e4)^0.5 (n_HI / b
// of Eq. 4 and 6 up to the constant K): the pair term w 2^-x^2 is then one
// exponential 2^(lw - x^2), its argument one FFMA.
struct SrcF32 { float a, bb, lw; int t, h; };

// The source's shift in whole pixels, round(v / du), as a float and an int
// (|v| / du < 2^22, which the host checks).
__device__ __forceinline__ float target_shift_f32(float v, const TauLaunch& L, int& isf)
{
    return round_to_int(v * L.inv_du, isf);
}

__device__ __forceinline__ SrcF32 prep_f32(const TauLaunch& L, float rho, float v, float T, int j)
{
    SrcF32 s;
    const float lr = lg2(rho);                           // log2 rho
    // log2(T / 1e4 K): stored, or Eq. 5 in log form, T0 min(rho, pivot)^(gamma-1)
    const float lt = L.t_mode != 0 ? fmaf(L.gm1, fminf(lr, L.lpivot), L.lT0) : lg2(T) - kLog2_1e4;
    s.lw = fmaf(-1.2f, lt, 2.f * lr);
    const float c = L.c_coef * ex2(-0.5f * lt);          // sqrt(log2 e) / b
    int isf;
    const float sf = target_shift_f32(v, L, isf);
    float r = fmaf(-sf, L.du_hi, v);                     // exact product inside the fma
    r = fmaf(-sf, L.du_lo, r);
    s.t = wrap_pixel(j + isf, L.n_pix);
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
    s.t = wrap_pixel(j + (int)sf, L.n_pix);
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
            if (PREC == LYA_PREC_F64) t = wrap_pixel(j + (int)rint((double)v * L.inv_du_d), N);
            else {
                int isf;
                (void)target_shift_f32(v, L, isf);
                t = wrap_pixel(j + isf, N);
            }
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
            rec[pos] = make_float4(s.a, s.bb, ex2(s.lw), (float)j);
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

// ---- tile kernel (FP32) -----------------------------------------------------------
//
// Sources are counting-sorted by target pixel into shared memory.  Source j
// covers the pixels |i - t_j| <= h_j, h_j = floor((nsigma b_j + |r_j|)/du).
// The output pixels are cut into tiles of kTile consecutive pixels; a tile's
// candidate sources are the sorted run of target bins [L, R] with
//   L = first bin t whose widest source reaches the first pixel of the tile
//       (t + h_t >= lo, h_t the widest reach in bin t)
//   R = last bin t whose widest source reaches the last pixel (t - h_t <= hi).
// The run holds every source covering the tile and, away from the broadest
// lines, little else.  Two ways to find L and R:
//   * local (window bound w_max <= kLocalReach): a per-bin widest-reach array
//     filled with shared-memory atomics; each tile scans at most the skewer's
//     widest reach hs to either side of it, four bins per 16-byte read;
//   * otherwise: the prefix max of the right reach and the suffix min of the
//     left reach, over bins extended by w_max on both sides so the periodic
//     wrap is explicit; both are monotone and a binary search over
//     [lo, hi + 2 w_max] of the extended bins finds L and R.
// With local runs the records of bins [N - hs, N) are also copied in front of
// the sorted records (target t - N) and those of bins [0, hs) behind them
// (t + N), so that every tile's run, across the seam or not, is one range of
// the record array, stored beside the tile order (when the copies fit the
// reserved ext_capacity records; else the run is split at the seam).  A tile
// whose run would span more than the whole skewer (a box so small that a
// line's window reaches past half of it) takes every source once instead, at
// the image nearest each pixel (wrap_segment).
//
// Load balance: the tiles are counting-sorted by candidate count, largest
// first, and handed to the threads in that order (reversed on alternate
// rounds), so the lanes of a warp walk lists of nearly equal length.  Four
// lanes share a tile and each owns two adjacent pixels: a candidate record is
// read once from shared memory and evaluated for both (one MUFU ex2 each).
// Where the runs average kLongRun candidates or more, two lanes share a tile
// with four pixels each.  tau is gathered in shared memory and written to HBM
// in order at the end.
//
// Accumulation per pixel: the terms of eight consecutive candidates (four
// where a lane takes four pixels) are added plainly, then folded into a Kahan
// sum (compensated variant); or every term is added plainly (naive variant).
//
// Shared memory: records (N + ext_capacity rounded up to 4) | bin counts
// (4 + N rounded up to 4; the leading zero makes bin starts and ends one
// array) | reach (N + 2 w_max; later tau) | tile runs L, R, the tile order and
// the ordered tiles' record ranges (int16).
//
// Each CTA of the standalone kernel also asks L2 for the inputs of the row one
// wave of CTAs later (a bulk prefetch), so its loads wait on L2, not HBM.
constexpr int kTile = 8;
constexpr int kLanesPerTile = 4;                 // each lane: kTile / kLanesPerTile = 2 pixels
constexpr int kTileKeys = 256;                   // tile-order histogram (counts >= 255 share a key; 8 per lane of one warp)
constexpr int kReachLow = -(1 << 28);
constexpr int kReachHigh = 1 << 28;
constexpr int kEmptyRun = 30000;                 // L of a tile no source reaches (L > R)
constexpr int kWrapTile = 8192;                  // tile-order flag: the run spans more than the skewer (NT <= 1024)
constexpr float kSqrtLn2 = 0.83255461115769775f;
constexpr float kHalfSqrtPi = 0.88622692545275801f;

__host__ __device__ __forceinline__ int round_up4(int n) { return (n + 3) & ~3; }

constexpr int kLocalReach = 64;                  // window bound up to which tiles search their runs locally
constexpr unsigned kStageSpins = 1u << 22;       // polls of the staged inputs' mbarrier before giving up

// Records past the seam copied to the ends of the record array (local
// searches only), so that every tile's candidates are one contiguous run:
// room for four sources per bin within w_max + 4 of either end.
__host__ __device__ __forceinline__ int ext_capacity(int w_max)
{
    return w_max <= kLocalReach ? 4 * (2 * w_max + 8) : 0;
}

// FP32 tile gather: records (with the seam copies) | bin starts | reach |
// tile runs, tile order and the ordered tiles' record ranges.
__host__ __device__ inline size_t tile_smem_bytes(int n_pix, int w_max)
{
    const int nt = (n_pix + kTile - 1) / kTile;
    return sizeof(float4) * (size_t)round_up4(n_pix + ext_capacity(w_max)) +
           sizeof(int) * (size_t)(4 + round_up4(n_pix)) + sizeof(int) * (size_t)(n_pix + 2 * w_max) +
           5 * sizeof(short) * (size_t)nt;
}

// One warp group of the serving kernel: its tile arrays, then 40 ints of scan
// scratch and the tile-order histogram.
constexpr int kGroupScanInts = 40;
constexpr int kRunTotal = 34;                    // scan scratch slot: the skewer's summed tile runs
constexpr int kSkewerReach = 35;                 // scan scratch slot: the skewer's widest reach h
constexpr int kSeamStarts = 36;                  // scan scratch slots 36, 37: bin starts at N - h and h
constexpr int kLongRun = 256;                    // mean run per tile from which a lane takes four pixels
__host__ __device__ inline size_t group_smem_bytes(int n_pix, int w_max)
{
    return (tile_smem_bytes(n_pix, w_max) + 15) / 16 * 16 + sizeof(int) * (kGroupScanInts + kTileKeys);
}

// Index of the source held in register slot q: vector loads give a thread
// four consecutive sources per group, scalar loads one source per stride.
__device__ __forceinline__ int src_index(int q, bool vec, int tid, int nt)
{
    return vec ? 4 * (tid + (q >> 2) * nt) + (q & 3) : tid + q * nt;
}

// The sorted-source pieces of extended bins [lx, rx], split where the run
// crosses the periodic seam: f(k0, k1, shift) for up to three pieces with
// frame shifts +N, 0, -N.
template <typename F>
__device__ __forceinline__ void for_tile_run(const int* bin, int N, int lx, int rx, F&& f)
{
    if (lx > rx) return;
    if (lx < 0) f(bin[lx + N], bin[min(rx, -1) + N + 1], (float)N);
    const int a0 = max(lx, 0), a1 = min(rx, N - 1);
    if (a0 <= a1) f(bin[a0], bin[a1 + 1], 0.f);
    if (rx >= N) f(bin[max(lx, N) - N], bin[rx - N + 1], -(float)N);
}

// Binary searches over a non-decreasing int array v on [a, b]: the first
// index with v >= x (b + 1 if none), the last with v <= x (a - 1 if none).
__device__ __forceinline__ int first_at_least(const int* v, int a, int b, int x)
{
    int lo = a, hi = b + 1;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (v[m] >= x) hi = m; else lo = m + 1;
    }
    return lo;
}
__device__ __forceinline__ int last_at_most(const int* v, int a, int b, int x)
{
    int lo = a, hi = b + 1;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (v[m] > x) hi = m; else lo = m + 1;
    }
    return lo - 1;
}

// Local candidate runs.  hm[t] is the widest reach of the sources in bin t
// (-1: empty).  The first bin t in [lo - hs, lo) whose sources reach pixel
// lo (t + hm[t] >= lo), else lo; the last bin t in (hi, hi + hs] whose
// sources reach hi (t - hm[t] <= hi), else hi.  Bins past the seam are read
// at their periodic image.  With N a multiple of 4 the bins are read four at
// a time (16-byte aligned groups).
__device__ __forceinline__ int local_run_left(const int* hm, int N, int lo, int hs, bool vec)
{
    if (vec) {
        for (int g = (lo - hs) & ~3; g < lo; g += 4) {
            const int4 q = *reinterpret_cast<const int4*>(hm + (g < 0 ? g + N : g));
            const int t0 = max(g, lo - hs);
            if (g >= t0 && g + q.x >= lo) return g;
            if (g + 1 >= t0 && g + 1 < lo && g + 1 + q.y >= lo) return g + 1;
            if (g + 2 >= t0 && g + 2 < lo && g + 2 + q.z >= lo) return g + 2;
            if (g + 3 >= t0 && g + 3 < lo && g + 3 + q.w >= lo) return g + 3;
        }
        return lo;
    }
    for (int t = lo - hs; t < lo; ++t)
        if (t + hm[t < 0 ? t + N : t] >= lo) return t;
    return lo;
}
__device__ __forceinline__ int local_run_right(const int* hm, int N, int hi, int hs, bool vec)
{
    if (vec) {
        for (int g = (hi + hs) & ~3; g + 3 > hi; g -= 4) {
            const int4 q = *reinterpret_cast<const int4*>(hm + (g >= N ? g - N : g));
            const int t1 = hi + hs;
            if (g + 3 <= t1 && g + 3 > hi && g + 3 - q.w <= hi) return g + 3;
            if (g + 2 <= t1 && g + 2 > hi && g + 2 - q.z <= hi) return g + 2;
            if (g + 1 <= t1 && g + 1 > hi && g + 1 - q.y <= hi) return g + 1;
            if (g <= t1 && g > hi && g - q.x <= hi) return g;
        }
        return hi;
    }
    for (int t = hi + hs; t > hi; --t)
        if (t - hm[t >= N ? t - N : t] <= hi) return t;
    return hi;
}

__device__ __forceinline__ void kahan_fold(float& S, float& C, float P)
{
    const float y = __fsub_rn(P, C);
    const float t = __fadd_rn(S, y);
    C = __fsub_rn(__fsub_rn(t, S), y);
    S = t;
}

// erfc(x) for x >= 0 in FP32 (the pixel-averaged profile): t = 1/(1 + 0.4 x)
// and erfc(x) = t 2^(P(t) - x^2 log2 e), P a degree-6 polynomial fitted by
// least squares on Chebyshev nodes of t (erfc_fit.py beside this file): within
// ~3e-6 of erfc for x < 4 and ~7e-6 out to x = 9, where the rounding of
// x^2 log2 e sets it; two MUFU and eight FMA-pipe operations.  Below 2^-126
// the result flushes to zero.
__device__ __forceinline__ float erfc_pos(float x)
{
    const float t = rcp_approx(fmaf(0.4f, x, 1.f));
    float p = 0x1.61e06ap-2f;
    p = fmaf(p, t, -0x1.15daap+0f);
    p = fmaf(p, t, 0x1.c0d2bap-1f);
    p = fmaf(p, t, -0x1.d295c4p-4f);
    p = fmaf(p, t, 0x1.624c58p-1f);
    p = fmaf(p, t, 0x1.6ea9f6p+0f);
    p = fmaf(p, t, -0x1.12d6acp+1f);
    return t * ex2(fmaf(-x * 1.44269504f, x, p));
}

// erfc of either sign: erfc(-x) = 2 - erfc(x).
__device__ __forceinline__ float erfc_any(float x)
{
    return x >= 0.f ? erfc_pos(x) : 2.f - erfc_pos(-x);
}

// The pixel-cell average of exp(-y^2) over [y - hw, y + hw], times 2 hw / sqrt(pi):
// erf(y + hw) - erf(y - hw), written with erfc of |y| so the far wings do not
// cancel.
__device__ __forceinline__ float cell_erf(float y, float hw)
{
    const float ay = fabsf(y);
    return erfc_any(ay - hw) - erfc_pos(ay + hw);
}

// The same for the cell between edges a < b from Ea = erfc(|a|), Eb =
// erfc(|b|), so that adjacent cells share their common edge's erfc: a cell
// right of 0 is Ea - Eb, left of 0 Eb - Ea, across 0 2 - Ea - Eb.
__device__ __forceinline__ float cell_from_edges(float a, float b, float Ea, float Eb)
{
    return a >= 0.f ? Ea - Eb : (b <= 0.f ? Eb - Ea : (2.f - Ea) - Eb);
}

// Two adjacent pixels fo, fo + 1 (in the run's frame) against candidates [k0, k1).
// Records {a, c r, lw, t} (sampled profile: term 2^(lw - x^2)); AVG: records
// hold the averaged-profile constants {du/b, r/b, w sqrt(pi) b/2du, t}.
template <bool COMP, bool AVG, int FOLD = 8>
__device__ __forceinline__ void pair2_segment(const float4* __restrict__ rec, int k0, int k1, float fo,
                                              float (&S)[2], float (&C)[2])
{
    auto terms = [&](const float4& r, float& t0, float& t1) {
        const float x0 = fmaf(fo - r.w, r.x, -r.y);                  // r = {a, c r, w, t}
        const float x1 = x0 + r.x;
        if constexpr (AVG) {
            // the two cells' three edges, each erfc once
            const float e0 = fmaf(-0.5f, r.x, x0), e1 = fmaf(0.5f, r.x, x0), e2 = fmaf(1.5f, r.x, x0);
            const float E0 = erfc_pos(fabsf(e0)), E1 = erfc_pos(fabsf(e1)), E2 = erfc_pos(fabsf(e2));
            t0 = r.z * cell_from_edges(e0, e1, E0, E1);
            t1 = r.z * cell_from_edges(e1, e2, E1, E2);
        } else {
            t0 = ex2(fmaf(-x0, x0, r.z));                             // r.z = lw
            t1 = ex2(fmaf(-x1, x1, r.z));
        }
    };
    int k = k0;
    if constexpr (COMP && !AVG) {
        // blocks of FOLD (8 or 4) candidates, read four at a time, their terms
        // summed plainly and the block sums folded into the Kahan sums; then a
        // block of four, then the last one to three
        for (; FOLD == 8 && k + 8 <= k1; k += 8) {
            float Q0, Q1;
            {
                const float4 r0 = rec[k], r1 = rec[k + 1], r2 = rec[k + 2], r3 = rec[k + 3];
                float a0, a1, b0, b1, c0, c1, d0, d1;
                terms(r0, a0, a1);
                terms(r1, b0, b1);
                terms(r2, c0, c1);
                terms(r3, d0, d1);
                Q0 = (a0 + b0) + (c0 + d0);
                Q1 = (a1 + b1) + (c1 + d1);
            }
            {
                const float4 r0 = rec[k + 4], r1 = rec[k + 5], r2 = rec[k + 6], r3 = rec[k + 7];
                float a0, a1, b0, b1, c0, c1, d0, d1;
                terms(r0, a0, a1);
                terms(r1, b0, b1);
                terms(r2, c0, c1);
                terms(r3, d0, d1);
                Q0 += (a0 + b0) + (c0 + d0);
                Q1 += (a1 + b1) + (c1 + d1);
            }
            kahan_fold(S[0], C[0], Q0);
            kahan_fold(S[1], C[1], Q1);
        }
        for (; k + 4 <= k1; k += 4) {
            const float4 r0 = rec[k], r1 = rec[k + 1], r2 = rec[k + 2], r3 = rec[k + 3];
            float a0, a1, b0, b1, c0, c1, d0, d1;
            terms(r0, a0, a1);
            terms(r1, b0, b1);
            terms(r2, c0, c1);
            terms(r3, d0, d1);
            kahan_fold(S[0], C[0], (a0 + b0) + (c0 + d0));
            kahan_fold(S[1], C[1], (a1 + b1) + (c1 + d1));
        }
        if (k < k1) {
            // one to three left: a pair, then a single, without a loop
            float P0, P1;
            if (k + 2 <= k1) {
                const float4 r0 = rec[k], r1 = rec[k + 1];
                float a0, a1, b0, b1;
                terms(r0, a0, a1);
                terms(r1, b0, b1);
                P0 = a0 + b0;
                P1 = a1 + b1;
                k += 2;
            } else {
                P0 = 0.f;
                P1 = 0.f;
            }
            if (k < k1) {
                float a0, a1;
                terms(rec[k], a0, a1);
                P0 += a0;
                P1 += a1;
            }
            kahan_fold(S[0], C[0], P0);
            kahan_fold(S[1], C[1], P1);
        }
    } else if constexpr (COMP) {
        while (k < k1) {
            float P0 = 0.f, P1 = 0.f;
            const int kk = min(k + 4, k1);
            for (; k < kk; ++k) {
                float t0, t1;
                terms(rec[k], t0, t1);
                P0 += t0;
                P1 += t1;
            }
            kahan_fold(S[0], C[0], P0);                      // Kahan folds of the block sums
            kahan_fold(S[1], C[1], P1);
        }
    } else {
#pragma unroll 2
        for (; k < k1; ++k) {
            float t0, t1;
            terms(rec[k], t0, t1);
            S[0] += t0;
            S[1] += t1;
        }
    }
}

// 2^y for y <= 0 on the FMA pipe: Cody-Waite split y = n + f (n the nearest
// integer, by the 1.5 * 2^23 shifter; |f| <= 1/2), 2^f by a degree-5
// polynomial fitted by least squares on Chebyshev nodes of [-1/2, 1/2]
// (coefficients from exp2_poly_fit.py beside this file), 2^n written into the
// exponent field.  Relative error ~2.3e-7; y is clamped at -126, so terms far
// outside a line's window come out as 2^-126 of its weight instead of 0.
__device__ __forceinline__ float exp2_poly(float y)
{
    y = fmaxf(y, -126.f);
    const float shifter = 0x1.8p23f;
    const float t = y + shifter;
    const int n = __float_as_int(t) - __float_as_int(shifter);
    const float f = y - (t - shifter);
    float p = 0x1.5f48c8p-10f;
    p = fmaf(p, f, 0x1.3d107cp-7f);
    p = fmaf(p, f, 0x1.c6aeccp-5f);
    p = fmaf(p, f, 0x1.ebf906p-3f);
    p = fmaf(p, f, 0x1.62e43p-1f);
    p = fmaf(p, f, 0x1.000002p+0f);
    return p * __int_as_float((n << 23) + 0x3f800000);
}

// Largest a = du sqrt(log2 e)/b for which the Gaussian recurrence is used: three
// steps then move x by at most 1.5, so a chain that starts below 2^-126 (|x| >
// 11.2) cannot reach a term above 2^-94 of the line's peak, below the window's
// own cut.
constexpr float kRecMaxA = 0.5f;

// Four adjacent pixels fo .. fo + 3 against candidates [k0, k1) (long runs:
// a record read from shared memory serves four pixels).  EXP selects how the
// four exponentials 2^-x_m^2, x_m = x_0 + m a, are formed:
//   LYA_EXP_MUFU        four MUFU ex2 of lw - x_m^2 (records carry lw);
//   LYA_EXP_RECURRENCE  the Gaussian recurrence of fast Gaussian gridding
//                       (Greengard & Lee 2004): E_{m+1} = E_m Q_m,
//                       Q_{m+1} = Q_m R with Q_0 = 2^-a(2 x_0 + a), R = 2^-2a^2:
//                       three MUFU and two FMUL per further pixel (lines with
//                       a <= kRecMaxA; wider pixels take the MUFU form);
//   LYA_EXP_POLY_SPLIT  three MUFU and one exp2_poly on the FMA pipe.
// (the last two take records with the linear weight w = 2^lw)
template <bool COMP, bool AVG, int EXP>
__device__ __forceinline__ void pair4_segment(const float4* __restrict__ rec, int k0, int k1, float fo,
                                              float (&S)[4], float (&C)[4])
{
    auto terms = [&](const float4& r, float (&t)[4]) {
        const float x0 = fmaf(fo - r.w, r.x, -r.y);                  // r = {a, c r, w, t}
        if constexpr (AVG) {
            // the four cells' five edges, each erfc once
            float e[5], E[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                e[m] = fmaf((float)m - 0.5f, r.x, x0);
                E[m] = erfc_pos(fabsf(e[m]));
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) t[m] = r.z * cell_from_edges(e[m], e[m + 1], E[m], E[m + 1]);
        } else if constexpr (EXP == LYA_EXP_RECURRENCE) {
            if (r.x <= kRecMaxA) {
                float E = ex2(-(x0 * x0));
                float Q = ex2(fminf(-r.x * fmaf(2.f, x0, r.x), 126.f));
                const float R = ex2(-2.f * r.x * r.x);
                t[0] = r.z * E;
#pragma unroll
                for (int m = 1; m < 4; ++m) {
                    E *= Q;
                    Q *= R;
                    t[m] = r.z * E;
                }
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float x = fmaf((float)m, r.x, x0);
                    t[m] = r.z * ex2(-(x * x));
                }
            }
        } else if constexpr (EXP == LYA_EXP_MUFU) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float x = fmaf((float)m, r.x, x0);
                t[m] = ex2(fmaf(-x, x, r.z));                         // r.z = lw
            }
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float x = fmaf((float)m, r.x, x0);
                t[m] = r.z * ((EXP == LYA_EXP_POLY_SPLIT && m == 3) ? exp2_poly(-(x * x)) : ex2(-(x * x)));
            }
        }
    };
    int k = k0;
    if constexpr (AVG) {
        // the cell averages keep fewer terms in flight (four erfc each)
        while (k < k1) {
            float P[4] = {0.f, 0.f, 0.f, 0.f};
            const int kk = COMP ? min(k + 4, k1) : k1;
            for (; k < kk; ++k) {
                float t[4];
                terms(rec[k], t);
#pragma unroll
                for (int m = 0; m < 4; ++m) P[m] += t[m];
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if constexpr (COMP) kahan_fold(S[m], C[m], P[m]);
                else S[m] += P[m];
            }
        }
    } else if constexpr (COMP) {
        // blocks of four candidates, read together and summed plainly, then
        // folded into the Kahan sums; the last block may be short
        for (; k + 4 <= k1; k += 4) {
            const float4 r0 = rec[k], r1 = rec[k + 1], r2 = rec[k + 2], r3 = rec[k + 3];
            float t0[4], t1[4], t2[4], t3[4];
            terms(r0, t0);
            terms(r1, t1);
            terms(r2, t2);
            terms(r3, t3);
#pragma unroll
            for (int m = 0; m < 4; ++m) kahan_fold(S[m], C[m], (t0[m] + t1[m]) + (t2[m] + t3[m]));
        }
        if (k < k1) {
            float P[4] = {0.f, 0.f, 0.f, 0.f};
            for (; k < k1; ++k) {
                float t[4];
                terms(rec[k], t);
#pragma unroll
                for (int m = 0; m < 4; ++m) P[m] += t[m];
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) kahan_fold(S[m], C[m], P[m]);
        }
    } else {
        for (; k < k1; ++k) {
            float t[4];
            terms(rec[k], t);
#pragma unroll
            for (int m = 0; m < 4; ++m) S[m] += t[m];
        }
    }
}

// A tile whose candidate run would span more than the whole skewer (boxes so
// small that a line's window reaches past half the box): every source once,
// records [k0, k1) with targets in [0, N), at the periodic image nearest each
// pixel (velocity difference in [-V/2, V/2), as Eq. 6 is read), NPX pixels
// fo .. fo + NPX - 1.  Slow, and met only in such boxes.
template <bool COMP, bool AVG, int NPX, bool LOGW>
__device__ __forceinline__ void wrap_segment(const float4* __restrict__ rec, int k0, int k1, float fo, float Nf,
                                          float (&S)[NPX], float (&C)[NPX])
{
    for (int k = k0; k < k1; ++k) {
        const float4 r = rec[k];                                    // r = {a, c r, w, t}
#pragma unroll
        for (int m = 0; m < NPX; ++m) {
            const float mi = (fo + (float)m) - r.w;                  // exact: integers
            float x = fmaf(mi, r.x, -r.y);
            if (x >= 0.5f * Nf * r.x) x = fmaf(mi - Nf, r.x, -r.y);
            else if (x < -0.5f * Nf * r.x) x = fmaf(mi + Nf, r.x, -r.y);
            const float t = AVG ? r.z * cell_erf(x, 0.5f * r.x)
                                : (LOGW ? ex2(fmaf(-x, x, r.z)) : r.z * ex2(-(x * x)));
            if constexpr (COMP) kahan_fold(S[m], C[m], t);
            else S[m] += t;
        }
    }
}

// A lane's finished pixels o .. o + NPX - 1 of tau, written straight to HBM
// (no staging in shared memory): one 8- or 16-byte streaming store where the
// row allows it (al: the row pointer is aligned to NPX floats).
template <int NPX>
__device__ __forceinline__ void store_pixels(float* out, int o, int N, bool al, const float (&t)[NPX])
{
    if (al && o + NPX <= N) {
        if constexpr (NPX == 4)
            __stcs(reinterpret_cast<float4*>(out + o), make_float4(t[0], t[1], t[2], t[3]));
        else
            __stcs(reinterpret_cast<float2*>(out + o), make_float2(t[0], t[1]));
        return;
    }
#pragma unroll
    for (int m = 0; m < NPX; ++m)
        if (o + m < N) out[o + m] = t[m];
}

// Step 7 with two lanes per tile, four pixels each, over the tiles in order.
template <bool COMP, bool AVG, int EXP>
__device__ __forceinline__ void tiles_by_four(const float4* __restrict__ rec, const int* bin, const short* Lt,
                                              const short* Rt, const short* order, const short* ok0,
                                              const short* ok1, bool ext, int N, int NT, float K,
                                              float* out, int tid, int nt, int base, int nsrc)
{
    const bool al16 = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    const int half = tid & 1, ng = nt / 2, grp = tid / 2;
    for (int round = 0; round * ng < NT; ++round) {
        const int i = round * ng + ((round & 1) ? ng - 1 - grp : grp);
        if (i >= NT) continue;
        const int ot = order[i];
        const int tile = ot & (kWrapTile - 1);
        const int o = kTile * tile + 4 * half;
        float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
        if (ot & kWrapTile) {
            wrap_segment<COMP, AVG, 4, !AVG && EXP == LYA_EXP_MUFU>(rec, base, base + nsrc, (float)o, (float)N, S, C);
        } else if (ext) {
            pair4_segment<COMP, AVG, EXP>(rec, ok0[i], ok1[i], (float)o, S, C);
        } else {
            for_tile_run(bin, N, Lt[tile], Rt[tile], [&](int k0, int k1, float shift) {
                pair4_segment<COMP, AVG, EXP>(rec, k0, k1, (float)o + shift, S, C);
            });
        }
        float t[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) t[m] = K * (COMP ? __fsub_rn(S[m], C[m]) : S[m]);
        store_pixels<4>(out, o, N, al16, t);
    }
}

// One skewer by one group of threads (the whole block, or a run of warps of
// it): rho/vpec/temp are the skewer's input rows, out its tau row.  smem
// holds the group's tile_smem_bytes(N, w_max) bytes (16-byte aligned);
// warp_tot (kGroupScanInts ints) and tile_hist (kTileKeys ints, 16-byte aligned) are the
// group's own shared scratch.  N <= MAXQ * g.nt.
// FOLD: candidates per Kahan fold in the two-pixel loop (8, or 4 where registers
// are scarcer: the serving kernel and the four-sources-per-thread tile kernel).
// STAGE: the skewer's inputs arrive by three 1D bulk copies (the TMA engine)
// into the record area, issued by the group's first thread and counted on
// the mbarrier *bar; needs N % 4 == 0 and 16-byte aligned rows.  Otherwise
// every thread loads its sources with 16-byte (or scalar) loads.
template <bool COMP, int MAXQ, bool AVG = false, bool ALT_EXP = false, int FOLD = 8, bool STAGE = false>
__device__ __forceinline__ void tile_skewer(const TauLaunch& L, const float* __restrict__ rho,
                                            const float* __restrict__ vpec, const float* __restrict__ temp,
                                            float* out, unsigned char* smem, int* warp_tot, int* tile_hist,
                                            const Group& g, unsigned long long* bar = nullptr)
{
    const int N = L.n_pix;
    const int Wd = L.w_max;
    const int NE = N + 2 * Wd;
    const int NT = (N + kTile - 1) / kTile;
    const int tid = g.tid, nt = g.nt;
    const int Cx = ext_capacity(Wd);
    float4* rec = reinterpret_cast<float4*>(smem);               // N + Cx (padded to 4)
    int* cnt = reinterpret_cast<int*>(rec + round_up4(N + Cx)) + 4;   // N (padded to 4), cnt[-1] = 0
    int* bin = cnt - 1;                                          // after the scatter: bin[t] = start(t),
                                                                 // bin[t + 1] = end(t)
    int* reach = cnt + round_up4(N);                         // NE
    short* Lt = reinterpret_cast<short*>(reach + NE);        // NT
    short* Rt = Lt + NT;                                     // NT
    short* order = Rt + NT;                                  // NT: tiles by candidate count
    short* ok0 = order + NT;                                 // NT: record run of order[i] (seam copies)
    short* ok1 = ok0 + NT;

    // 1. every input load issued up front (float4 when rows are 16-byte aligned)
    const bool vec = (N & 3) == 0;
    const int rec_cap = round_up4(N + Cx);                  // records the shared memory holds
    LYA_BOUND(N <= MAXQ * nt && NT <= kWrapTile);
    float r_[MAXQ], v_[MAXQ], T_[MAXQ];
    float* s_rho = reinterpret_cast<float*>(rec);           // staged inputs (STAGE), 12 N bytes
    float* s_v = s_rho + N;
    float* s_T = s_v + N;
    if constexpr (STAGE) {
        if (tid == 0) {
            mbar_init(bar, 1);
            const unsigned bytes = 4u * (unsigned)N;
            mbar_expect_tx(bar, (temp ? 3u : 2u) * bytes);
            bulk_copy_g2s(s_rho, rho, bytes, bar);
            bulk_copy_g2s(s_v, vpec, bytes, bar);
            if (temp) bulk_copy_g2s(s_T, temp, bytes, bar);
        }
    } else if (vec) {
#pragma unroll
        for (int u4 = 0; u4 < MAXQ / 4; ++u4) {
            const int grp = tid + u4 * nt;
            if (4 * grp < N) {
                const float4 a = __ldcs(reinterpret_cast<const float4*>(rho) + grp);
                const float4 b = __ldcs(reinterpret_cast<const float4*>(vpec) + grp);
                const float4 c = temp ? __ldcs(reinterpret_cast<const float4*>(temp) + grp)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                r_[4 * u4] = a.x; r_[4 * u4 + 1] = a.y; r_[4 * u4 + 2] = a.z; r_[4 * u4 + 3] = a.w;
                v_[4 * u4] = b.x; v_[4 * u4 + 1] = b.y; v_[4 * u4 + 2] = b.z; v_[4 * u4 + 3] = b.w;
                T_[4 * u4] = c.x; T_[4 * u4 + 1] = c.y; T_[4 * u4 + 2] = c.z; T_[4 * u4 + 3] = c.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) r_[4 * u4 + u] = 0.f;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < MAXQ; ++q) {
            const int j = tid + q * nt;
            r_[q] = j < N ? __ldcs(rho + j) : 0.f;
            v_[q] = j < N ? __ldcs(vpec + j) : 0.f;
            T_[q] = (j < N && temp) ? __ldcs(temp + j) : 0.f;
        }
    }
    // local: every tile finds its run by looking at most the skewer's widest
    // reach to either side in a per-bin widest-reach array (-1: empty bin);
    // otherwise the runs come from block-wide envelope scans
    const bool local = Wd <= kLocalReach;
    if (vec) {
        // cnt[-4 .. N) and reach[0 .. N) are 16-byte aligned runs of whole int4s
        for (int k = tid; k < N / 4 + 1; k += nt) reinterpret_cast<int4*>(cnt - 4)[k] = make_int4(0, 0, 0, 0);
    } else {
        for (int k = tid - 4; k < N; k += nt) cnt[k] = 0;
    }
    if (local && vec) {
        for (int e = tid; e < N / 4; e += nt) reinterpret_cast<int4*>(reach)[e] = make_int4(-1, -1, -1, -1);
    } else if (local) {
        for (int e = tid; e < N; e += nt) reach[e] = -1;
    } else {
        for (int e = tid; e < NE; e += nt) reach[e] = kReachLow;
    }
    for (int k = tid; k < kTileKeys / 4; k += nt) reinterpret_cast<int4*>(tile_hist)[k] = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        warp_tot[kRunTotal] = 0;
        warp_tot[kSkewerReach] = 0;
    }
    g.sync();                       // (also: the mbarrier is initialised before anyone waits on it)
    if constexpr (STAGE) {
        if (!mbar_wait(bar, 0, kStageSpins)) {
            // the copies did not land in time: flag it (bit 3) and wait once
            // more, bounded, so none is still in flight when the CTA moves on
            if ((tid & 31) == 0) atomicOr(L.err, 8);
            mbar_wait(bar, 0, kStageSpins);
        }
#pragma unroll
        for (int u4 = 0; u4 < MAXQ / 4; ++u4) {
            const int grp = tid + u4 * nt;
            if (4 * grp < N) {
                const float4 a = reinterpret_cast<const float4*>(s_rho)[grp];
                const float4 b = reinterpret_cast<const float4*>(s_v)[grp];
                const float4 c = temp ? reinterpret_cast<const float4*>(s_T)[grp] : make_float4(0.f, 0.f, 0.f, 0.f);
                r_[4 * u4] = a.x; r_[4 * u4 + 1] = a.y; r_[4 * u4 + 2] = a.z; r_[4 * u4 + 3] = a.w;
                v_[4 * u4] = b.x; v_[4 * u4 + 1] = b.y; v_[4 * u4 + 2] = b.z; v_[4 * u4 + 3] = b.w;
                T_[4 * u4] = c.x; T_[4 * u4 + 1] = c.y; T_[4 * u4 + 2] = c.z; T_[4 * u4 + 3] = c.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) r_[4 * u4 + u] = 0.f;
            }
        }
    }

    // 2. per-source constants (kept in registers) and the histogram of target
    //    pixels; th_ packs (target << 16) | reach, -1 = no source
    float a_[MAXQ], bb_[MAXQ], w_[MAXQ];                 // w_: lw, or the linear weight (see below)
    int th_[MAXQ];
    int hsk = 0;
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        const int j = src_index(q, vec, tid, nt);
        th_[q] = -1;
        if (j < N && r_[q] > 0.f) {
            SrcF32 s = prep_f32(L, r_[q], v_[q], T_[q], j);
            if constexpr (AVG) {
                // cell average: y = d/b = x sqrt(ln 2), half-width du/2b, weight
                // w sqrt(pi) b / 2du; the window grows by the half cell
                s.a *= kSqrtLn2;
                s.bb *= kSqrtLn2;
                s.lw = ex2(s.lw) * (kHalfSqrtPi / s.a);
                s.h = min(s.h + 1, L.w_max);
            } else if (ALT_EXP && L.exp_method != LYA_EXP_MUFU) {
                s.lw = ex2(s.lw);                    // the other exponential forms take w itself
            }
            a_[q] = s.a;
            bb_[q] = s.bb;
            w_[q] = s.lw;
            th_[q] = (s.t << 16) | s.h;
            LYA_BOUND(s.t >= 0 && s.t < N && s.h >= 0 && s.h <= Wd);
            atomicAdd(&cnt[s.t], 1);
            if (local) {
                atomicMax(&reach[s.t], s.h);
                hsk = max(hsk, s.h);
            }
        }
    }
    if (local) {
        hsk = __reduce_max_sync(0xffffffffu, hsk);
        if ((tid & 31) == 0 && hsk > 0) atomicMax(&warp_tot[kSkewerReach], hsk);
    }
    g.sync();

    // 3. bin starts; scatter the records {a, c r, w, t} and every source's
    //    right reach t + h (three periodic images).  With local searches the
    //    sources of bins [N - hs, N) are later copied in front of the records
    //    (t - N) and those of bins [0, hs) behind them (t + N), so the
    //    records start at P = the number of the former: ext (when the copies
    //    fit the reserved Cx records)
    const int hs = local ? warp_tot[kSkewerReach] : 0;
    const int nsrc = block_exclusive_scan(cnt, N, warp_tot, g, hs > 0 ? N - hs : -1, hs > 0 ? hs : -1,
                                          warp_tot + kSeamStarts);
    const int P = hs > 0 ? nsrc - warp_tot[kSeamStarts] : 0;
    const int npost = hs > 0 ? warp_tot[kSeamStarts + 1] : 0;
    const bool ext = local && P + npost <= Cx;
    const int base = ext ? P : 0;
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        if (th_[q] < 0) continue;
        const int t = th_[q] >> 16, h = th_[q] & 0xffff;
        const int pos = atomicAdd(&cnt[t], 1);
        if (pos >= N) { atomicOr(L.err, 2); th_[q] = -1; continue; }   // input changed under the kernel
        LYA_BOUND(base + pos >= 0 && base + pos < rec_cap);
        rec[base + pos] = make_float4(a_[q], bb_[q], w_[q], (float)t);
        if (local) continue;
        LYA_BOUND(t >= 0 && t + Wd < NE);
        atomicMax(&reach[t + Wd], t + h);
        if (t >= N - Wd) atomicMax(&reach[t - N + Wd], t - N + h);
        if (t < Wd) atomicMax(&reach[t + N + Wd], t + N + h);
    }
    g.sync();
    if (!local) {
        // 4. first candidate bin of every tile: search the prefix max of the right reach
        block_prefix_max(reach, NE, warp_tot, kReachLow, g);       // ends with a barrier
        for (int tile = tid; tile < NT; tile += nt) {
            const int lo = kTile * tile, hi = min(lo + kTile - 1, N - 1);
            const int e = first_at_least(reach, lo, min(hi + 2 * Wd, NE - 1), lo);
            Lt[tile] = (short)(e <= min(hi + 2 * Wd, NE - 1) ? e - Wd : kEmptyRun);
        }
        g.sync();
        for (int e = tid; e < NE; e += nt) reach[e] = kReachHigh;
        g.sync();
#pragma unroll
        for (int q = 0; q < MAXQ; ++q) {
            if (th_[q] < 0) continue;
            const int t = th_[q] >> 16, h = th_[q] & 0xffff;
            atomicMin(&reach[t + Wd], t - h);
            if (t >= N - Wd) atomicMin(&reach[t - N + Wd], t - N - h);
            if (t < Wd) atomicMin(&reach[t + N + Wd], t + N - h);
        }
        g.sync();

        // 5. last candidate bin of every tile: search the suffix min of the left reach
        block_suffix_min(reach, NE, warp_tot, kReachHigh, g);      // ends with a barrier
        for (int tile = tid; tile < NT; tile += nt) {
            const int lo = kTile * tile, hi = min(lo + kTile - 1, N - 1);
            const int e = last_at_most(reach, lo, min(hi + 2 * Wd, NE - 1), hi);
            Rt[tile] = (short)(e >= lo ? e - Wd : -kEmptyRun);
        }
        g.sync();
    }

    // 6. tiles ordered by candidate count, largest first (counting sort)
    constexpr int kMaxTilesPerThread = (MAXQ + kTile - 1) / kTile;   // NT <= MAXQ nt / kTile
    int tkey[kMaxTilesPerThread], trank[kMaxTilesPerThread], kk0[kMaxTilesPerThread], kk1[kMaxTilesPerThread];
    bool wrap[kMaxTilesPerThread];
    int runs = 0;
#pragma unroll
    for (int u = 0; u < kMaxTilesPerThread; ++u) {
        const int tile = tid + u * nt;
        tkey[u] = -1;
        if (tile < NT) {
            int lx, rx;
            if (local) {
                // first bin at most hs left of the tile whose widest source
                // reaches it, last bin at most hs right of it likewise (bins
                // past the seam are read at their periodic image)
                const int lo = kTile * tile, hi = min(lo + kTile - 1, N - 1);
                LYA_BOUND(hs <= Wd && lo - hs > -N && hi + hs < 2 * N);
                lx = local_run_left(reach, N, lo, hs, vec);
                rx = local_run_right(reach, N, hi, hs, vec);
                if (!ext) {
                    Lt[tile] = (short)lx;
                    Rt[tile] = (short)rx;
                }
            } else {
                lx = Lt[tile];
                rx = Rt[tile];
            }
            int c = 0;
            wrap[u] = rx - lx + 1 > N;        // the run would hold a source twice: every source once instead
            if (wrap[u]) {
                c = nsrc;
            } else if (ext) {
                // the run as one range of the record array with its copies
                LYA_BOUND(lx >= -N && lx < N && rx >= 0 && rx < 2 * N);
                kk0[u] = lx >= 0 ? base + bin[lx] : bin[lx + N] - (nsrc - P);
                kk1[u] = rx < N ? base + bin[rx + 1] : base + nsrc + bin[rx - N + 1];
                c = kk1[u] - kk0[u];
                LYA_BOUND(kk0[u] >= 0 && kk0[u] <= kk1[u] && kk1[u] <= base + nsrc + npost &&
                          base + nsrc + npost <= rec_cap && kk1[u] < 32768);
            } else {
                for_tile_run(bin, N, lx, rx, [&](int k0, int k1, float) { c += k1 - k0; });
            }
            tkey[u] = kTileKeys - 1 - min(c, kTileKeys - 1);
            trank[u] = atomicAdd(&tile_hist[tkey[u]], 1);    // its rank among the tiles of its key
            runs += c;
        }
    }
    if (runs) atomicAdd(&warp_tot[kRunTotal], runs);
    if (ext) {
        // the seam copies: bins [N - hs, N) in front as t - N, bins [0, hs) behind as t + N
        for (int e = tid; e < P + npost; e += nt) {
            LYA_BOUND(base + nsrc + npost <= rec_cap && nsrc - P >= 0);
            if (e < P) {
                float4 r = rec[base + nsrc - P + e];
                r.w -= (float)N;
                rec[e] = r;
            } else {
                float4 r = rec[base + e - P];
                r.w += (float)N;
                rec[base + nsrc + e - P] = r;
            }
        }
    }
    g.sync();
    if (tid < 32) {
        // exclusive scan of the kTileKeys counts by the first warp, eight per lane
        int4* h4 = reinterpret_cast<int4*>(tile_hist) + 2 * tid;
        const int4 x = h4[0], y = h4[1];
        const int loc = (x.x + x.y + x.z + x.w) + (y.x + y.y + y.z + y.w);
        int run = warp_inclusive_scan(loc) - loc;
        int4 ox, oy;
        ox.x = run; run += x.x; ox.y = run; run += x.y; ox.z = run; run += x.z; ox.w = run; run += x.w;
        oy.x = run; run += y.x; oy.y = run; run += y.y; oy.z = run; run += y.z; oy.w = run;
        h4[0] = ox;
        h4[1] = oy;
    }
    g.sync();
#pragma unroll
    for (int u = 0; u < kMaxTilesPerThread; ++u) {
        if (tkey[u] < 0) continue;
        LYA_BOUND(tkey[u] < kTileKeys);
        const int pos = tile_hist[tkey[u]] + trank[u];     // the key's first slot + the rank
        LYA_BOUND(pos >= 0 && pos < NT);
        order[pos] = (short)((tid + u * nt) | (wrap[u] ? kWrapTile : 0));
        if (ext && !wrap[u]) {
            ok0[pos] = (short)kk0[u];
            ok1[pos] = (short)kk1[u];
        }
    }
    g.sync();

    // 7. lane groups walk the tiles in that order (reversed on alternate
    //    rounds, so every warp's total work evens out); each lane owns two
    //    adjacent pixels, or four where the runs are long, and writes them
    //    to HBM itself (store_pixels: no staging, no final barrier)
    const float K = L.K;
    if (ALT_EXP && L.exp_method != LYA_EXP_MUFU) {
        if constexpr (ALT_EXP && !AVG) {
            if (L.exp_method == LYA_EXP_RECURRENCE)
                tiles_by_four<COMP, false, LYA_EXP_RECURRENCE>(rec, bin, Lt, Rt, order, ok0, ok1, ext, N, NT, K,
                                                               out, tid, nt, base, nsrc);
            else
                tiles_by_four<COMP, false, LYA_EXP_POLY_SPLIT>(rec, bin, Lt, Rt, order, ok0, ok1, ext, N, NT, K,
                                                               out, tid, nt, base, nsrc);
        }
    } else if (warp_tot[kRunTotal] >= kLongRun * NT) {
        tiles_by_four<COMP, AVG, LYA_EXP_MUFU>(rec, bin, Lt, Rt, order, ok0, ok1, ext, N, NT, K, out, tid, nt, base,
                                               nsrc);
    } else {
    const bool al8 = (reinterpret_cast<uintptr_t>(out) & 7) == 0;
    const int lane_q = tid & (kLanesPerTile - 1);
    const int npairs = nt / kLanesPerTile, pair = tid / kLanesPerTile;
    for (int round = 0; round * npairs < NT; ++round) {
        const int i = round * npairs + ((round & 1) ? npairs - 1 - pair : pair);
        if (i >= NT) continue;
        const int ot = order[i];
        int k0 = 0, k1 = 0;
        if (ext && !(ot & kWrapTile)) {
            k0 = ok0[i];
            k1 = ok1[i];
        }
        const int tile = ot & (kWrapTile - 1);
        const int o = kTile * tile + 2 * lane_q;
        LYA_BOUND(tile < NT && (!ext || (ot & kWrapTile) || (ok0[i] >= 0 && ok0[i] <= ok1[i] && ok1[i] <= rec_cap)));
        LYA_BOUND(ext || (ot & kWrapTile) || Lt[tile] > Rt[tile] || (Lt[tile] >= -Wd && Rt[tile] < N + Wd));
        float S[2] = {0.f, 0.f}, C[2] = {0.f, 0.f};
        if (ot & kWrapTile) {
            wrap_segment<COMP, AVG, 2, !AVG>(rec, base, base + nsrc, (float)o, (float)N, S, C);
        } else if (ext) {
            pair2_segment<COMP, AVG, FOLD>(rec, k0, k1, (float)o, S, C);
        } else {
            for_tile_run(bin, N, Lt[tile], Rt[tile], [&](int k0, int k1, float shift) {
                pair2_segment<COMP, AVG, FOLD>(rec, k0, k1, (float)o + shift, S, C);
            });
        }
        const float t[2] = {K * (COMP ? __fsub_rn(S[0], C[0]) : S[0]), K * (COMP ? __fsub_rn(S[1], C[1]) : S[1])};
        store_pixels<2>(out, o, N, al8, t);
    }
    }
}

template <bool COMP, int MAXQ, bool AVG, int NTB, bool STAGE>
__global__ void __launch_bounds__(NTB, NTB == 384 ? 5 : (NTB >= 1024 ? 1 : 2)) tau_tile_kernel(const TauLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int warp_tot[kGroupScanInts];
    __shared__ __align__(16) int tile_hist[kTileKeys];
    __shared__ __align__(8) unsigned long long stage_bar;
    const int64_t row = blockIdx.x;
    const int64_t sk = L.ids ? L.ids[row] : row;
    const int N = L.n_pix;
    float* out = L.tau_out + row * (int64_t)N;
    if (sk < 0 || sk >= L.n_skewers) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) out[i] = 0.f;
        if (threadIdx.x == 0) atomicOr(L.err, 1);
        return;
    }
    if (threadIdx.x == 0 && L.pf_ahead > 0 && row + L.pf_ahead < L.n_rows) {
        // the row a CTA about one wave later extracts, into L2: its loads then
        // wait on L2 rather than HBM
        const int64_t pr = row + L.pf_ahead;
        const int64_t psk = L.ids ? L.ids[pr] : pr;
        const unsigned bytes = 4u * (unsigned)N;
        if (psk >= 0 && psk < L.n_skewers && (bytes & 15u) == 0) {
            const float* rows[3] = {L.rho + psk * (int64_t)N, L.vpec + psk * (int64_t)N,
                                    L.temp ? L.temp + psk * (int64_t)N : nullptr};
            for (const float* q : rows)
                if (q && (reinterpret_cast<uintptr_t>(q) & 15) == 0) prefetch_l2(q, bytes);
        }
    }
    tile_skewer<COMP, MAXQ, AVG, true, (MAXQ >= 8 ? 8 : 4), STAGE>(
        L, L.rho + sk * (int64_t)N, L.vpec + sk * (int64_t)N, L.temp ? L.temp + sk * (int64_t)N : nullptr, out,
        smem_raw, warp_tot, tile_hist, whole_block(), &stage_bar);
}


// ---- serving: one persistent kernel over a step's work list ---------------------
//
// One 1024-thread CTA per SM takes tasks from the step's list in order (an
// atomic counter; the list is sorted longest first).  A task is up to
// 1 << shift skewers of one request; the CTA splits into that many warp
// groups of 1024 >> shift threads, each with its own named barrier and its
// own slice of shared memory, and each group extracts one skewer with the
// same tile gather as tau_tile_kernel (compensated sums).  The request's
// constants are copied to shared memory once per task.
__global__ void __launch_bounds__(serve::kTauThreads, 1) tau_serve_kernel(unsigned char* __restrict__ step)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the task and its request's constants live in shared memory, so that
    // little but the step pointer stays in registers across the skewer body
    __shared__ TauLaunch Ls;
    __shared__ serve::TauTask Ts;
    __shared__ long long s_src[1 << serve::kMaxShift], s_out[1 << serve::kMaxShift];
    __shared__ int s_more;
    for (;;) {
        if (threadIdx.x == 0) {
            serve::StepHeader* hdr = reinterpret_cast<serve::StepHeader*>(step);
            const int t = (int)atomicAdd(&hdr->task_next, 1u);
            s_more = t < hdr->n_tasks;
            if (s_more) {
                Ts = serve::step_table<serve::TauTask>(step, hdr->off_tasks)[t];
                const serve::TauItem* items = serve::step_table<serve::TauItem>(step, hdr->off_items);
                for (int k = 0; k < Ts.n_items; ++k) {
                    s_src[k] = items[Ts.first_item + k].src_row;
                    s_out[k] = items[Ts.first_item + k].out_row;
                }
            }
        }
        __syncthreads();
        if (!s_more) break;
        {
            const serve::StepHeader* hdr = reinterpret_cast<const serve::StepHeader*>(step);
            const int* src = reinterpret_cast<const int*>(serve::step_table<TauLaunch>(step, hdr->off_slots) + Ts.slot);
            int* dst = reinterpret_cast<int*>(&Ls);
            for (int k = threadIdx.x; k < (int)(sizeof(TauLaunch) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
        }
        __syncthreads();
        const int gnt = serve::kTauThreads >> Ts.shift;
        const int gi = (int)threadIdx.x / gnt;
        if (gi < Ts.n_items) {
            const Group g{(int)threadIdx.x - gi * gnt, gnt, Ts.shift == 0 ? 0 : 1 + gi};
            const int N = Ls.n_pix;
            unsigned char* base = smem_raw + (size_t)gi * group_smem_bytes(N, Ls.w_max);
            int* warp_tot = reinterpret_cast<int*>(base + (tile_smem_bytes(N, Ls.w_max) + 15) / 16 * 16);
            int* tile_hist = warp_tot + kGroupScanInts;
            const long long src = s_src[gi];
            float* out = Ls.tau_out + s_out[gi] * (int64_t)N;
            if (src < 0 || src >= Ls.n_skewers) {
                for (int i = g.tid; i < N; i += g.nt) out[i] = 0.f;
                if (g.tid == 0) atomicOr(Ls.err, 1);
            } else {
                const float* rho = Ls.rho + src * (int64_t)N;
                const float* vpec = Ls.vpec + src * (int64_t)N;
                const float* temp = Ls.temp ? Ls.temp + src * (int64_t)N : nullptr;
                tile_skewer<true, serve::kTauMaxQ, false, false, 4>(Ls, rho, vpec, temp, out, base, warp_tot,
                                                                    tile_hist, g);
            }
        }
        __syncthreads();
    }
}

int block_threads(int n_pix)
{
    if (n_pix > 4096) return 1024;
    if (n_pix >= 2048) return 512;
    if (n_pix >= 512) return 256;
    return 128;
}

}  // namespace

// FP64 comparator (whole-skewer-window gather): records | bin starts.
static size_t global_smem_bytes(int n_pix)
{
    return sizeof(double4_32a) * (size_t)n_pix + sizeof(int) * (size_t)(n_pix + 1);
}


size_t tau_smem_bytes(int n_pix, int w_max, int precision)
{
    if (precision == LYA_PREC_F64) return global_smem_bytes(n_pix);
    return tile_smem_bytes(n_pix, w_max);
}

// Per kernel and device: the dynamic shared memory it has been allowed, and
// the resident CTAs of the device for the last (threads, shared memory) asked
// for, so that repeated launches skip the attribute and occupancy queries.
struct LaunchInfo {
    const void* fn;
    int dev;
    size_t smem_allowed;
    int nt;
    size_t smem;
    int64_t resident;
};
static std::mutex g_launch_mu;
static LaunchInfo g_launch_info[64];
static int g_launch_n = 0;

template <typename K>
static cudaError_t launch_kernel(K kernel, const TauLaunch& L0, size_t smem, int nt, cudaStream_t stream,
                                 bool prefetch = false)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const void* fn = reinterpret_cast<const void*>(kernel);
    int64_t resident = -1;
    {
        std::lock_guard<std::mutex> lk(g_launch_mu);
        LaunchInfo* li = nullptr;
        for (int i = 0; i < g_launch_n; ++i)
            if (g_launch_info[i].fn == fn && g_launch_info[i].dev == dev) li = &g_launch_info[i];
        if (!li || li->smem_allowed < smem) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (e != cudaSuccess) return e;
            if (!li && g_launch_n < 64) {
                li = &g_launch_info[g_launch_n++];
                *li = LaunchInfo{fn, dev, 0, 0, 0, -1};
            }
            if (li) li->smem_allowed = smem;
        }
        if (prefetch) {
            // one wave ahead: the CTAs resident on the whole device at once
            if (li && li->nt == nt && li->smem == smem && li->resident >= 0) {
                resident = li->resident;
            } else {
                int sms = 0, per_sm = 0;
                if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, smem) == cudaSuccess)
                    resident = (int64_t)sms * per_sm;
                (void)cudaGetLastError();
                if (li && resident >= 0) {
                    li->nt = nt;
                    li->smem = smem;
                    li->resident = resident;
                }
            }
        }
    }
    if (L0.n_rows == 0) return cudaSuccess;
    TauLaunch L = L0;
    L.pf_ahead = resident > 0 ? resident : 0;
    kernel<<<(unsigned)L.n_rows, nt, smem, stream>>>(L);
    count_launch();
    return cudaGetLastError();
}

// Inputs staged by bulk copies for rows of 2,048 pixels or more (n_pix % 4 ==
// 0: rows 16-byte aligned, since fields are); measured on GB300 on 16,384 x
// 4,096 px: 0.953 ms staged against 0.958 ms with vector loads, and on
// 262,144 rows of 1,536 px 5.10 ms staged against 4.87 ms, hence the
// threshold.  LYA_TILE_STAGE=0/1 in the environment forces either
// (diagnostics).
static bool stage_inputs(const TauLaunch& L)
{
    const char* env = std::getenv("LYA_TILE_STAGE");
    if ((L.n_pix & 3) != 0) return false;
    if (env && (env[0] == '0' || env[0] == '1')) return env[0] == '1';
    return L.n_pix >= 2048;
}

template <bool COMP, bool AVG, bool STAGE>
static cudaError_t launch_tile_staged(const TauLaunch& L, cudaStream_t stream)
{
    const size_t smem = tile_smem_bytes(L.n_pix, L.w_max);
    const int nt = block_threads(L.n_pix);                   // N <= 8 nt (n_pix <= 8192)
    const int q = (L.n_pix + nt - 1) / nt;
    // rows of 1,025-1,536 px (the 1536^3 grid): 384 threads with four sources
    // each, five CTAs per SM at 32 registers (measured on 262,144 grid rows:
    // 5.29 ms against 5.56 ms with 256 threads of eight sources, four CTAs
    // per SM at 64 registers)
    if constexpr (!AVG) {
        if (L.n_pix > 1024 && L.n_pix <= 1536)
            return launch_kernel(tau_tile_kernel<COMP, 4, AVG, 384, STAGE>, L, smem, 384, stream, true);
    }
    if (nt > 512) return launch_kernel(tau_tile_kernel<COMP, 8, AVG, 1024, STAGE>, L, smem, nt, stream, true);
    if (q <= 4) return launch_kernel(tau_tile_kernel<COMP, 4, AVG, 512, STAGE>, L, smem, nt, stream, true);
    return launch_kernel(tau_tile_kernel<COMP, 8, AVG, 512, STAGE>, L, smem, nt, stream, true);
}

template <bool COMP, bool AVG>
static cudaError_t launch_tile_profile(const TauLaunch& L, cudaStream_t stream)
{
    return stage_inputs(L) ? launch_tile_staged<COMP, AVG, true>(L, stream)
                           : launch_tile_staged<COMP, AVG, false>(L, stream);
}

template <bool COMP>
static cudaError_t launch_tile(const TauLaunch& L, cudaStream_t stream)
{
    return L.profile == LYA_PROFILE_AVERAGED ? launch_tile_profile<COMP, true>(L, stream)
                                             : launch_tile_profile<COMP, false>(L, stream);
}

cudaError_t launch_tau(const TauLaunch& L, int precision, cudaStream_t stream)
{
    switch (precision) {
    case LYA_PREC_F32_COMPENSATED: return launch_tile<true>(L, stream);
    case LYA_PREC_F32_NAIVE: return launch_tile<false>(L, stream);
    case LYA_PREC_F64:
        return launch_kernel(tau_kernel<LYA_PREC_F64>, L, global_smem_bytes(L.n_pix),
                             std::min(block_threads(L.n_pix), 512), stream);
    default: return cudaErrorInvalidValue;
    }
}


namespace serve {

size_t serve_group_smem(int n_pix, int w_max) { return group_smem_bytes(n_pix, w_max); }

cudaError_t serve_tau_prepare(size_t* dyn_smem)
{
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, tau_serve_kernel);
    if (e != cudaSuccess) return e;
    const size_t dyn = max_dynamic_smem() - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(tau_serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tau_serve_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess) *dyn_smem = dyn;
    return e;
}

cudaError_t serve_tau_launch(const unsigned char* d_step, size_t dyn_smem, int grid, cudaStream_t stream)
{
    tau_serve_kernel<<<grid, kTauThreads, dyn_smem, stream>>>(const_cast<unsigned char*>(d_step));
    return cudaGetLastError();
}

}  // namespace serve

}  // namespace lya
