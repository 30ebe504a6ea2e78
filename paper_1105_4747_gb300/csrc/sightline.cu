// sightline.cu -- lines of sight generated in Fourier space on the device
// (Sec. 2.1-2.2), sm_103a.
//
// For skewer id s of a field with seed S and N = 2^a 3^b pixels over a
// periodic box L, modes n = 1 .. N/2 - 1 (k_n = 2 pi n / L) get
//   D_n = (N/2) sqrt(P_n) conj(g_n),  P_n ~ k_n^-1 exp(-(k_n/k_J)^2), sum P_n = sigma^2,
// with g_n = a + i b (a, b standard normal: Box-Muller on Philox4x32-10 words
// of counter (n, s) under key S), the Eq. 3 velocity V_n = i aH D_n / k_n and
// the Eq. 1 gas smoothing D_n / (1 + k_n^2 / k_F^2) of the density.  Both real
// fields come from one complex inverse transform of Z_n = D_n + i V_n (with
// the Hermitian halves filled in): delta = Re z, v = c Im z, where V enters
// divided by c, the ratio of the two fields' ensemble rms, so that the
// rounding of the much larger velocity does not swamp the density.  The
// density is returned as the lognormal 1 + delta = exp(delta - sigma_b^2 / 2).
//
// sightline_modes_kernel (one CTA) tabulates the per-mode factors in FP64;
// sightline_kernel runs persistent CTAs (one twiddle table each) over the
// skewers, each transform in shared memory.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "fft_device.cuh"
#include "lya_device.cuh"
#include "lya_internal.h"
#include "mean_flux_device.cuh"

namespace lya {
namespace {

using namespace mfd;
using namespace fftd;

constexpr int kGenThreads = 512;

// table[n - 1] = {(N/2) sqrt(P_n), Eq. 1 factor, aH / (c k_n)};
// out[0] = sigma_b^2, out[1] = c = rms(v) / rms(delta_b) over the ensemble.
__global__ void __launch_bounds__(kThreads) sightline_modes_kernel(int N, double box, double k_j, double sigma,
                                                                 double k_f, double aH, float* table,
                                                                 double* out)
{
    const int H = N / 2 - 1;
    __shared__ double sh[3][32];
    double s[3] = {0.0, 0.0, 0.0};
    for (int n = 1 + threadIdx.x; n <= H; n += blockDim.x) {
        const double k = 2.0 * 3.14159265358979323846 * n / box;
        const double p = exp(-(k / k_j) * (k / k_j)) / k;
        const double f = k_f > 0.0 ? 1.0 / (1.0 + (k / k_f) * (k / k_f)) : 1.0;
        s[0] += p;
        s[1] += p * f * f;
        s[2] += p * (aH / k) * (aH / k);
    }
    block_sum<3>(s, sh);
    __shared__ double norm, c;
    if (threadIdx.x == 0) {
        norm = sigma * sigma / s[0];
        c = s[1] > 0.0 && s[2] > 0.0 ? sqrt(s[2] / s[1]) : 1.0;
        out[0] = s[1] * norm;
        out[1] = c;
    }
    __syncthreads();
    for (int n = 1 + threadIdx.x; n <= H; n += blockDim.x) {
        const double k = 2.0 * 3.14159265358979323846 * n / box;
        const double p = exp(-(k / k_j) * (k / k_j)) / k * norm;
        table[3 * (n - 1)] = (float)(0.5 * N * sqrt(p));
        table[3 * (n - 1) + 1] = (float)(k_f > 0.0 ? 1.0 / (1.0 + (k / k_f) * (k / k_f)) : 1.0);
        table[3 * (n - 1) + 2] = (float)(aH / (c * k));
    }
}

struct GenLaunch {
    int N;
    long long n_rows;
    unsigned long long seed;
    long long first_id;
    const float* table;
    const double* consts;        // {sigma_b^2, c}
    float* rho;
    float* vpec;
};

__global__ void __launch_bounds__(kGenThreads) sightline_kernel(const GenLaunch G)
{
    extern __shared__ __align__(16) float2 zbuf[];
    const int N = G.N, H = N / 2;
    float2* X = zbuf;
    float2* Y = zbuf + N;
    float2* T = zbuf + 2 * N;                                           // twiddles, once per CTA
    fft_twiddles(T, N);
    const float inv_n = 1.f / (float)N;
    const float half_var = (float)(0.5 * G.consts[0]);
    const float v_scale = (float)(G.consts[1]) * inv_n;
    for (long long row = blockIdx.x; row < G.n_rows; row += gridDim.x) {
        const unsigned long long id = (unsigned long long)(G.first_id + row);
        __syncthreads();                                                // T ready; X free again
        // conj(Z) for the forward transform: Z_n = D_n + i V_n and Z_{N-n} = conj D_n + i conj V_n
        for (int n = threadIdx.x; n <= H; n += blockDim.x) {
            if (n == 0 || n == H) {
                X[n] = make_float2(0.f, 0.f);
                continue;
            }
            const float2 g = normal_pair(philox4x32_10(
                U4{(unsigned int)n, (unsigned int)id, (unsigned int)(id >> 32), 0u}, (unsigned int)G.seed,
                (unsigned int)(G.seed >> 32)));
            const float* t = G.table + 3 * (n - 1);
            const float2 D = make_float2(t[0] * g.x, -t[0] * g.y);      // (N/2) sqrt(P) conj(g)
            const float2 Db = make_float2(t[1] * D.x, t[1] * D.y);      // Eq. 1
            const float2 V = make_float2(-t[2] * D.y, t[2] * D.x);      // Eq. 3: i (aH/k) D / c
            const float2 Zn = make_float2(Db.x - V.y, Db.y + V.x);      // Db + i V
            const float2 Zm = make_float2(Db.x + V.y, -Db.y + V.x);     // conj(Db) + i conj(V)
            X[n] = make_float2(Zn.x, -Zn.y);
            X[N - n] = make_float2(Zm.x, -Zm.y);
        }
        __syncthreads();
        const float2* W = fft_stockham(X, Y, T, N);                     // fft(conj Z) = N conj(z)
        float* rho = G.rho + row * (long long)N;
        float* v = G.vpec + row * (long long)N;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            const float2 w = W[j];
            rho[j] = expf(fmaf(w.x, inv_n, -half_var));
            v[j] = -w.y * v_scale;
        }
    }
}

}  // namespace

size_t sightline_smem_bytes(int n_pix) { return sizeof(float2) * 3 * (size_t)n_pix; }

lya_status sightlines_run(int n_pix, double box, double k_j, double sigma, double k_f, double aH, uint64_t seed,
                          int64_t first_id, int64_t n_ids, float* rho, float* vpec, cudaStream_t stream)
{
    const int H = n_pix / 2 - 1;
    float* table = nullptr;
    double* consts = nullptr;
    cudaError_t e = scratch_malloc((void**)&table, sizeof(float) * 3 * (size_t)(H > 0 ? H : 1), stream);
    if (e == cudaSuccess) e = scratch_malloc((void**)&consts, 2 * sizeof(double), stream);
    if (e == cudaSuccess) {
        sightline_modes_kernel<<<1, kThreads, 0, stream>>>(n_pix, box, k_j, sigma, k_f, aH, table, consts);
        count_launch();
        e = cudaGetLastError();
    }
    const size_t smem = sightline_smem_bytes(n_pix);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sightline_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sightline_kernel, kGenThreads, smem);
    if (e == cudaSuccess && n_ids > 0) {
        const int grid = (int)std::min<long long>(n_ids, (long long)std::max(per_sm, 1) * sm_count());
        GenLaunch G{n_pix, (long long)n_ids, seed, (long long)first_id, table, consts, rho, vpec};
        sightline_kernel<<<grid, kGenThreads, smem, stream>>>(G);
        count_launch();
        e = cudaGetLastError();
    }
    if (table) cudaFreeAsync(table, stream);
    if (consts) cudaFreeAsync(consts, stream);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA;
    return LYA_OK;
}

}  // namespace lya
