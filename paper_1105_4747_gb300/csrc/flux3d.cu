// flux3d.cu -- 3D flux power spectrum of a set of lines of sight with the
// Eq. 7 reconstruction, sm_103a.
//
// Lines of sight run along z through a periodic cube; each sits at a cell of
// an n x n transverse grid.  The box field delta_F (0 off the lines) is
// transformed in two stages: a 1D transform along each line (persistent CTAs,
// two real lines per complex Stockham transform, as for the 1D flux power),
// whose modes k_z = 0 .. N/2 are scattered into N/2 + 1 transverse planes of
// n x n complex values; then one CTA per plane runs the 2D transform in
// shared memory (batched rows, then batched columns) and folds every mode's
// |G|^2, less the Eq. 7 terms P_1D(k_z) P_2D,w and P_N, into the spherical
// shells [b, b + 1) k_f that plane can reach (an exact integer square root
// picks the shell).  The modes are visited in order of mx^2 + my^2, so a
// thread's run of modes stays in one or two shells and adds to the shared
// sums only when its shell changes; the shared sums go once per shell into
// the FP64 totals.
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

constexpr int kLosThreads = 512;
constexpr int kPlaneThreads = 256;

__global__ void __launch_bounds__(kThreads) f3_sum_kernel(const float* __restrict__ F, long long n, double* out,
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

struct LosLaunch {
    const float* flux;
    const int* cell;          // n_los transverse cell indices ix * n + iy
    long long n_los;
    int N, cells;             // pixels per line, n * n
    const double* sum;        // sum of every F value
    float2* planes;           // [N/2 + 1][n * n]
    double* p1d;              // [N/2 + 1] sums over lines of |D|^2
};

// 1D transforms of the lines' delta_F, scattered into the k_z planes.
__global__ void __launch_bounds__(kLosThreads) f3_los_kernel(const LosLaunch L)
{
    extern __shared__ __align__(16) float2 buf[];
    const int N = L.N, H = N / 2 + 1;
    float2* X = buf;
    float2* Y = buf + N;
    float2* T = buf + 2 * N;
    float* acc = reinterpret_cast<float*>(buf + 3 * N);
    for (int n = threadIdx.x; n < H; n += blockDim.x) acc[n] = 0.f;
    fft_twiddles(T, N);
    const float inv_mean = (float)((double)L.n_los * N / *L.sum);
    const long long pairs = (L.n_los + 1) / 2;
    for (long long pr = blockIdx.x; pr < pairs; pr += gridDim.x) {
        const long long ra = 2 * pr, rb = 2 * pr + 1;
        const bool two = rb < L.n_los;
        const float* Fa = L.flux + ra * (long long)N;
        const float* Fb = two ? L.flux + rb * (long long)N : nullptr;
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            X[i] = make_float2(fmaf(__ldcs(Fa + i), inv_mean, -1.f), two ? fmaf(__ldcs(Fb + i), inv_mean, -1.f) : 0.f);
        __syncthreads();
        const float2* Z = fft_stockham(X, Y, T, N);
        const int ca = L.cell[ra], cb = two ? L.cell[rb] : 0;
        for (int k = threadIdx.x; k < H; k += blockDim.x) {
            const float2 z = Z[k], zc = Z[k == 0 ? 0 : N - k];
            const float2 A = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
            float2* pa = L.planes + (long long)k * L.cells + ca;
            atomicAdd(&pa->x, A.x);
            atomicAdd(&pa->y, A.y);
            float a2 = A.x * A.x + A.y * A.y;
            if (two) {
                const float2 B = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
                float2* pb = L.planes + (long long)k * L.cells + cb;
                atomicAdd(&pb->x, B.x);
                atomicAdd(&pb->y, B.y);
                a2 += B.x * B.x + B.y * B.y;
            }
            acc[k] += a2;
        }
    }
    __syncthreads();
    for (int n = threadIdx.x; n < H; n += blockDim.x)
        if (acc[n] != 0.f) atomicAdd(L.p1d + n, (double)acc[n]);
}

struct PlaneLaunch {
    const float2* planes;
    const short* order;       // the n^2 transverse modes sorted by mx^2 + my^2
    int n, N;                 // transverse side, pixels per line
    const double* p1d;        // sums of |D|^2 over lines
    double box_norm;          // V / M^2
    double alias;             // (L / N^2) / n_los * P_2D,w: multiplies p1d sums
    double noise;             // P_N
    double* shells;           // [n_shells][4]: sum P_true, sum P_box, sum |m|, modes
    int n_shells;
};

__device__ __forceinline__ int isqrt_exact(int m2)
{
    int b = (int)sqrtf((float)m2);
    while ((b + 1) * (b + 1) <= m2) ++b;
    while (b * b > m2) --b;
    return b;
}

// fftfreq order: index i of n -> signed mode number
__device__ __forceinline__ int mode_number(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

// The n^2 transverse modes sorted by mx^2 + my^2 (a counting sort in one CTA):
// for any k_z the shell index is non-decreasing along this order.
__global__ void __launch_bounds__(kPlaneThreads) f3_order_kernel(int n, short* order)
{
    extern __shared__ int keys[];                      // 2 (n/2)^2 + 2 counters
    const int K = 2 * (n / 2) * (n / 2) + 1;
    __shared__ int warp_tot[33];
    for (int k = threadIdx.x; k < K; k += blockDim.x) keys[k] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        const int mx = mode_number(i / n, n), my = mode_number(i % n, n);
        atomicAdd(&keys[mx * mx + my * my], 1);
    }
    __syncthreads();
    block_exclusive_scan(keys, K, warp_tot);
    // stable within a key by mode index: one thread places every mode
    if (threadIdx.x == 0)
        for (int i = 0; i < n * n; ++i) {
            const int mx = mode_number(i / n, n), my = mode_number(i % n, n);
            order[keys[mx * mx + my * my]++] = (short)i;
        }
}

// One k_z plane: 2D transform, Eq. 7, shells.
__global__ void __launch_bounds__(kPlaneThreads) f3_plane_kernel(const PlaneLaunch P)
{
    extern __shared__ __align__(16) float2 pbuf[];
    const int n = P.n, cells = n * n;
    const int kz = blockIdx.x;
    float2* X = pbuf;
    float2* Y = pbuf + cells;
    float2* T = pbuf + 2 * cells;
    // shells this plane reaches: kz .. floor(sqrt(kz^2 + 2 (n/2)^2))
    const int b0 = kz;
    const int nb = isqrt_exact(kz * kz + 2 * (n / 2) * (n / 2)) - b0 + 1;
    float* sacc = reinterpret_cast<float*>(pbuf + 2 * cells + n);       // [nb][4]
    for (int i = threadIdx.x; i < 4 * nb; i += blockDim.x) sacc[i] = 0.f;
    fft_twiddles(T, n);
    const float2* src = P.planes + (long long)kz * cells;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) X[i] = src[i];
    __syncthreads();
    float2* R = fft_stockham_batched(X, Y, T, n, n, n, 1);              // rows
    float2* O = R == X ? Y : X;
    float2* G = fft_stockham_batched(R, O, T, n, n, 1, n);              // columns
    const float mult = (kz == 0 || 2 * kz == P.N) ? 1.f : 2.f;
    const double sub = P.alias * P.p1d[kz] + P.noise;
    // each thread takes a contiguous run of the sorted modes, where the shell
    // changes rarely, and adds to the shared sums only when it does
    const int per = (cells + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(cells, lo + per);
    int cur = -1;
    float s_t = 0.f, s_b = 0.f, s_k = 0.f, s_n = 0.f;
    for (int j = lo; j < hi; ++j) {
        const int i = P.order[j];
        const int mx = mode_number(i / n, n), my = mode_number(i % n, n);
        const int m2 = mx * mx + my * my + kz * kz;
        if (m2 == 0) continue;
        const int b = isqrt_exact(m2) - b0;
        if (b != cur) {
            if (cur >= 0) {
                atomicAdd(&sacc[4 * cur], s_t);
                atomicAdd(&sacc[4 * cur + 1], s_b);
                atomicAdd(&sacc[4 * cur + 2], s_k);
                atomicAdd(&sacc[4 * cur + 3], s_n);
            }
            cur = b;
            s_t = s_b = s_k = s_n = 0.f;
        }
        const float2 g = G[i];
        const double pbox = P.box_norm * ((double)g.x * g.x + (double)g.y * g.y);
        s_t += mult * (float)(pbox - sub);
        s_b += mult * (float)pbox;
        s_k += mult * sqrtf((float)m2);
        s_n += mult;
    }
    if (cur >= 0) {
        atomicAdd(&sacc[4 * cur], s_t);
        atomicAdd(&sacc[4 * cur + 1], s_b);
        atomicAdd(&sacc[4 * cur + 2], s_k);
        atomicAdd(&sacc[4 * cur + 3], s_n);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * nb; i += blockDim.x) {
        const int b = b0 + i / 4;
        if (b < P.n_shells && sacc[i] != 0.f) atomicAdd(P.shells + 4 * b + (i & 3), (double)sacc[i]);
    }
}

}  // namespace

size_t flux3d_los_smem_bytes(int n_pix) { return sizeof(float2) * 3 * (size_t)n_pix + sizeof(float) * (n_pix / 2 + 1); }

size_t flux3d_plane_smem_bytes(int n_perp, int n_pix)
{
    // the widest shell range a plane reaches: floor(sqrt(2 (n/2)^2)) + 1
    const int nb = (int)std::floor(std::sqrt(2.0 * (n_perp / 2) * (n_perp / 2))) + 2;
    (void)n_pix;
    return sizeof(float2) * (2 * (size_t)n_perp * n_perp + n_perp) + sizeof(float) * 4 * (size_t)nb;
}

int flux3d_shells(int n_perp, int n_pix)
{
    const long long m2 = 2LL * (n_perp / 2) * (n_perp / 2) + (long long)(n_pix / 2) * (n_pix / 2);
    long long b = (long long)std::sqrt((double)m2);
    while ((b + 1) * (b + 1) <= m2) ++b;
    while (b * b > m2) --b;
    return (int)b + 1;
}

lya_status flux_power_3d_run(const float* flux, const int* cells_host, int64_t n_los, int n_pix, int n_perp,
                             double box, double noise_sigma, double* shells_out /* host [n_shells][4] */,
                             int n_shells, cudaStream_t stream)
{
    const long long npx = (long long)n_los * n_pix;
    const int H = n_pix / 2 + 1, cells = n_perp * n_perp;
    const int grid_sum = (int)std::min<long long>((npx + kThreads - 1) / kThreads, 8LL * sm_count());
    double* d = nullptr;            // [0] sum of F, [1 .. H] p1d, then shells (4 n_shells), then partials
    unsigned int* ticket = nullptr;
    int* cell = nullptr;
    float2* planes = nullptr;
    const size_t nd = 1 + (size_t)H + 4 * (size_t)n_shells + grid_sum;
    cudaError_t e = scratch_malloc((void**)&d, sizeof(double) * nd, stream);
    if (e == cudaSuccess) e = scratch_malloc((void**)&ticket, sizeof(unsigned int), stream);
    if (e == cudaSuccess) e = scratch_malloc((void**)&cell, sizeof(int) * (size_t)n_los, stream);
    if (e == cudaSuccess) e = scratch_malloc((void**)&planes, sizeof(float2) * (size_t)H * cells, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(double) * (1 + H + 4 * (size_t)n_shells), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(planes, 0, sizeof(float2) * (size_t)H * cells, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cell, cells_host, sizeof(int) * (size_t)n_los, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
        f3_sum_kernel<<<grid_sum, kThreads, 0, stream>>>(flux, npx, d, d + 1 + H + 4 * n_shells, ticket);
        count_launch();
        e = cudaGetLastError();
    }
    const size_t smem_los = flux3d_los_smem_bytes(n_pix);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f3_los_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_los);
    if (e == cudaSuccess) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f3_los_kernel, kLosThreads, smem_los);
        const long long pairs = (n_los + 1) / 2;
        const int grid = (int)std::min<long long>(pairs, (long long)std::max(per_sm, 1) * sm_count());
        if (e == cudaSuccess) {
            LosLaunch L{flux, cell, (long long)n_los, n_pix, cells, d, planes, d + 1};
            f3_los_kernel<<<grid, kLosThreads, smem_los, stream>>>(L);
            count_launch();
            e = cudaGetLastError();
        }
    }
    short* order = nullptr;
    if (e == cudaSuccess) e = scratch_malloc((void**)&order, sizeof(short) * (size_t)cells, stream);
    if (e == cudaSuccess) {
        const size_t smem_keys = sizeof(int) * (2 * (size_t)(n_perp / 2) * (n_perp / 2) + 2);
        f3_order_kernel<<<1, kPlaneThreads, smem_keys, stream>>>(n_perp, order);
        count_launch();
        e = cudaGetLastError();
    }
    const size_t smem_plane = flux3d_plane_smem_bytes(n_perp, n_pix);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f3_plane_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plane);
    if (e == cudaSuccess) {
        const double M = (double)cells * n_pix;
        const double p2d = box * box * (double)n_los / ((double)cells * cells);     // white level of the weights
        PlaneLaunch P{planes, order, n_perp, n_pix, d + 1, box * box * box / (M * M),
                      box / ((double)n_pix * n_pix) / (double)n_los * p2d,
                      box / n_pix * noise_sigma * noise_sigma * p2d, d + 1 + H, n_shells};
        f3_plane_kernel<<<H, kPlaneThreads, smem_plane, stream>>>(P);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(shells_out, d + 1 + H, sizeof(double) * 4 * (size_t)n_shells, cudaMemcpyDeviceToHost, stream);
    if (d) cudaFreeAsync(d, stream);
    if (ticket) cudaFreeAsync(ticket, stream);
    if (cell) cudaFreeAsync(cell, stream);
    if (planes) cudaFreeAsync(planes, stream);
    if (order) cudaFreeAsync(order, stream);
    const cudaError_t e2 = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LYA_ENOMEM : LYA_ECUDA;
    return LYA_OK;
}

}  // namespace lya
