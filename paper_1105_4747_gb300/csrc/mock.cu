// mock.cu -- mock spectra (Sec. 4) and the line-of-sight flux power spectrum
// (Sec. 5.3) on sm_103a.
//
// mock_kernel: one CTA per skewer.  The input cells the output reads, with a
// periodic halo of the profile's half-width, are staged in shared memory; the
// instrument profile is a discrete convolution with normalised Gaussian
// weights (computed once per call in FP64 by mock_weights_kernel), evaluated
// only on those cells; output pixel k of width B takes the cell-overlap mean
// of the convolved cells (cell edges in FP64, fractions and sums in FP32); noise
// of sigma 1/(S/N) comes from Philox4x32-10 (Salmon et al. 2011) keyed by the
// seed and countered by (output pixel, skewer row), by Box-Muller on two
// 24-bit uniforms.
//
// flux_ps_kernel: persistent CTAs over pairs of skewers.  Two real skewers
// ride in one complex FFT (a + i b) of length N = 2^p 3^q, a Stockham
// autosort decimation-in-frequency transform in shared memory (radix 3, then
// radix 2 passes, twiddles from a per-CTA table); the two spectra are separated by
// conjugate symmetry and |X|^2 is summed per CTA, then once per CTA into the
// FP64 totals.
#include <cmath>
#include <cstdint>

#include "lya_device.cuh"
#include "lya_internal.h"
#include "mean_flux_device.cuh"
#include "fft_device.cuh"

namespace lya {
namespace {

using namespace mfd;
using namespace fftd;

constexpr int kMockThreads = 256;
constexpr int kPsThreads = 512;

// ---- instrument profile weights (FP64, normalised) -----------------------------------
__global__ void __launch_bounds__(kMockThreads) mock_weights_kernel(int W, double du_over_sigma, float* w)
{
    __shared__ double sh[1][32];
    double s[1] = {0.0};
    for (int m = -W + (int)threadIdx.x; m <= W; m += blockDim.x) {
        const double x = m * du_over_sigma;
        s[0] += exp(-0.5 * x * x);
    }
    block_sum<1>(s, sh);
    __shared__ double total;
    if (threadIdx.x == 0) total = s[0];
    __syncthreads();
    for (int m = -W + (int)threadIdx.x; m <= W; m += blockDim.x) {
        const double x = m * du_over_sigma;
        w[m + W] = (float)(exp(-0.5 * x * x) / total);
    }
}

struct MockLaunch {
    const float* flux;
    float* out;
    long long n_skewers;
    int N, M, W;                 // input pixels, output pixels, profile half-width (0: none)
    int i_lo, n_cells;           // the input cells the output reads: i_lo .. i_lo + n_cells - 1 (periodic)
    const float* w;              // 2W + 1 weights
    double ratio;                // output pixel width / input pixel width
    float noise;                 // sigma of the noise (0: none)
    unsigned long long seed;
    long long row0;              // noise counter of row 0
};

// Shared memory: the cells i_lo - W .. i_lo + n_cells - 1 + W of the skewer
// (periodic copies, so the profile needs no wrap test), the convolved cells,
// the weights.
__global__ void __launch_bounds__(kMockThreads) mock_kernel(const MockLaunch L)
{
    extern __shared__ __align__(16) float sm[];
    const int N = L.N, W = L.W, nc = L.n_cells;
    const int n_ext = nc + 2 * W;
    float* ext = sm;                                  // n_ext
    float* conv = W > 0 ? sm + n_ext : sm;            // nc (the cells themselves without a profile)
    float* w = sm + (W > 0 ? n_ext + nc : n_ext);     // 2W + 1
    const long long row = blockIdx.x;
    const float* F = L.flux + row * (long long)N;
    int src = (L.i_lo - W) % N;
    if (src < 0) src += N;
    for (int c = threadIdx.x; c < n_ext; c += blockDim.x) {
        int i = src + c;
        while (i >= N) i -= N;
        ext[c] = __ldcs(F + i);
    }
    for (int m = threadIdx.x; m < 2 * W + 1 && W > 0; m += blockDim.x) w[m] = L.w[m];
    __syncthreads();

    // instrument profile: conv[c] = sum_m w[m] ext[c + m]
    if (W > 0) {
        const int taps = 2 * W + 1;
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const float* x = ext + c;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int m = 0;
            for (; m + 3 < taps; m += 4) {
                a0 = fmaf(w[m], x[m], a0);
                a1 = fmaf(w[m + 1], x[m + 1], a1);
                a2 = fmaf(w[m + 2], x[m + 2], a2);
                a3 = fmaf(w[m + 3], x[m + 3], a3);
            }
            for (; m < taps; ++m) a0 = fmaf(w[m], x[m], a0);
            conv[c] = (a0 + a1) + (a2 + a3);
        }
        __syncthreads();
    }

    // resampling: output pixel k spans cells [a, b) (cell units relative to
    // i_lo), edges in FP64, the overlap fractions and sums in FP32; then noise
    float* out = L.out + row * (long long)L.M;
    const double r = L.ratio;
    for (int k = threadIdx.x; k < L.M; k += blockDim.x) {
        const double a = fma((double)k - 0.5, r, 0.5 - L.i_lo), b = fma((double)k + 0.5, r, 0.5 - L.i_lo);
        const int ia = max((int)floor(a), 0), ib = min((int)ceil(b) - 1, L.n_cells - 1);
        float acc;
        if (ia == ib) {
            acc = (float)(b - a) * conv[ia];
        } else {
            acc = (float)((double)(ia + 1) - a) * conv[ia];
            for (int i = ia + 1; i < ib; ++i) acc += conv[i];
            acc = fmaf((float)(b - (double)ib), conv[ib], acc);
        }
        float y = (float)(acc / r);
        if (L.noise > 0.f) y = fmaf(L.noise, normal_deviate(L.seed, k, L.row0 + row), y);
        out[k] = y;
    }
}

// ---- 1D flux power spectrum ---------------------------------------------------------
struct PsLaunch {
    const float* flux;
    long long n_skewers;
    int N;
    const double* sum;           // device: sum of every F value
    double* power;               // device: N/2 + 1 totals of |X_n|^2 (n_skewers summed)
};

__global__ void __launch_bounds__(kThreads) ps_sum_kernel(const float* __restrict__ F, long long n, double* out,
                                                        double* part, unsigned int* ticket)
{
    KahanF32 s;
    stream_f32(F, n, [&](long long, float f) { s.add(f); });
    __shared__ double sh[1][32];
    double v[1] = {(double)s.value()};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
    if (!last_block(ticket)) return;
    double t[1] = {0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t[0] += part[b];
    block_sum<1>(t, sh);
    if (threadIdx.x == 0) {
        *out = t[0];
        *ticket = 0;
    }
}

__global__ void __launch_bounds__(kPsThreads) flux_ps_kernel(const PsLaunch L)
{
    extern __shared__ __align__(16) float2 buf[];
    const int N = L.N, H = N / 2 + 1;
    float2* X = buf;
    float2* Y = buf + N;
    float2* T = buf + 2 * N;                                   // N twiddles
    float* acc = reinterpret_cast<float*>(buf + 3 * N);        // H partial powers
    for (int n = threadIdx.x; n < H; n += blockDim.x) acc[n] = 0.f;
    fft_twiddles(T, N);
    const float inv_mean = (float)((double)L.n_skewers * N / *L.sum);
    const long long pairs = (L.n_skewers + 1) / 2;
    for (long long pr = blockIdx.x; pr < pairs; pr += gridDim.x) {
        const long long ra = 2 * pr, rb = 2 * pr + 1;
        const float* Fa = L.flux + ra * (long long)N;
        const float* Fb = rb < L.n_skewers ? L.flux + rb * (long long)N : nullptr;
        __syncthreads();                                       // the previous pair is done with X, Y
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const float da = fmaf(__ldcs(Fa + i), inv_mean, -1.f);
            const float db = Fb ? fmaf(__ldcs(Fb + i), inv_mean, -1.f) : 0.f;
            X[i] = make_float2(da, db);
        }
        __syncthreads();
        const float2* src = fft_stockham(X, Y, T, N);
        // Z = A + i B: A_n = (Z_n + conj Z_{N-n}) / 2, B_n = (Z_n - conj Z_{N-n}) / 2i
        for (int k = threadIdx.x; k < H; k += blockDim.x) {
            const float2 z = src[k], zc = src[k == 0 ? 0 : N - k];
            const float ar = 0.5f * (z.x + zc.x), ai = 0.5f * (z.y - zc.y);
            const float br = 0.5f * (z.y + zc.y), bi = -0.5f * (z.x - zc.x);
            acc[k] += ar * ar + ai * ai + (Fb ? br * br + bi * bi : 0.f);
        }
    }
    __syncthreads();
    for (int n = threadIdx.x; n < H; n += blockDim.x)
        if (acc[n] != 0.f) atomicAdd(L.power + n, (double)acc[n]);
}

}  // namespace

// ---- host side -----------------------------------------------------------------------
// The input cells output pixels 0 .. M-1 read (cell units, i_lo may be
// negative), with one spare cell on each side so that rounding of the FP64
// edges on the device can never index outside them.
static void mock_cells(int M, double ratio, int* i_lo, int* n_cells)
{
    const int lo = (int)std::floor(0.5 - 0.5 * ratio) - 1;
    const int hi = (int)std::ceil((M - 0.5) * ratio + 0.5);
    *i_lo = lo;
    *n_cells = hi - lo + 1;
}

size_t mock_smem_bytes(int n_pix, int n_out, double ratio, int W)
{
    int lo, nc;
    mock_cells(n_out, ratio, &lo, &nc);
    (void)n_pix;
    const size_t n_ext = (size_t)nc + 2 * (size_t)W;
    return sizeof(float) * (n_ext + (W > 0 ? (size_t)nc + 2 * (size_t)W + 1 : 0));
}

lya_status mock_spectra_run(const float* flux, int64_t n_skewers, int n_pix, int n_out, int W, double du_over_sigma,
                            double ratio, double noise, uint64_t seed, int64_t row0, float* out, cudaStream_t stream)
{
    float* w = nullptr;
    cudaError_t e = cudaSuccess;
    if (W > 0) {
        e = scratch_malloc((void**)&w, sizeof(float) * (2 * W + 1), stream);
        if (e == cudaSuccess) {
            mock_weights_kernel<<<1, kMockThreads, 0, stream>>>(W, du_over_sigma, w);
            count_launch();
            e = cudaGetLastError();
        }
    }
    int i_lo, n_cells;
    mock_cells(n_out, ratio, &i_lo, &n_cells);
    const size_t smem = mock_smem_bytes(n_pix, n_out, ratio, W);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mock_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && n_skewers > 0) {
        MockLaunch L{flux, out, (long long)n_skewers, n_pix, n_out, W, i_lo, n_cells, w, ratio, (float)noise, seed,
                     (long long)row0};
        mock_kernel<<<(unsigned)n_skewers, kMockThreads, smem, stream>>>(L);
        count_launch();
        e = cudaGetLastError();
    }
    if (w) cudaFreeAsync(w, stream);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA;
    return LYA_OK;
}

size_t flux_ps_smem_bytes(int n_pix) { return sizeof(float2) * 3 * (size_t)n_pix + sizeof(float) * (n_pix / 2 + 1); }

lya_status flux_power_run(const float* flux, int64_t n_skewers, int n_pix, double* sums_out /* host: N/2+1 */,
                          double* mean_out, cudaStream_t stream)
{
    const long long n = (long long)n_skewers * n_pix;
    const int H = n_pix / 2 + 1;
    const int grid_sum = (int)std::min<long long>((n + kThreads - 1) / kThreads, 8LL * sm_count());
    double* d = nullptr;       // [0] sum of F, [1..H] power totals, then partials
    unsigned int* ticket = nullptr;
    cudaError_t e = scratch_malloc((void**)&d, sizeof(double) * (1 + H + grid_sum), stream);
    if (e == cudaSuccess) e = scratch_malloc((void**)&ticket, sizeof(unsigned int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(double) * (1 + H), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess) {
        ps_sum_kernel<<<grid_sum, kThreads, 0, stream>>>(flux, n, d, d + 1 + H, ticket);
        count_launch();
        e = cudaGetLastError();
    }
    const size_t smem = flux_ps_smem_bytes(n_pix);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flux_ps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flux_ps_kernel, kPsThreads, smem);
        const long long pairs = (n_skewers + 1) / 2;
        const int grid = (int)std::min<long long>(pairs, (long long)std::max(per_sm, 1) * sm_count());
        if (e == cudaSuccess) {
            PsLaunch L{flux, (long long)n_skewers, n_pix, d, d + 1};
            flux_ps_kernel<<<grid, kPsThreads, smem, stream>>>(L);
            count_launch();
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums_out, d + 1, sizeof(double) * H, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mean_out, d, sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (d) cudaFreeAsync(d, stream);
    if (ticket) cudaFreeAsync(ticket, stream);
    const cudaError_t e2 = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA;
    *mean_out /= (double)n;
    return LYA_OK;
}

}  // namespace lya
