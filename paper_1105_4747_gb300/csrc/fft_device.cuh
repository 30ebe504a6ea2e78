// fft_device.cuh -- device pieces shared by the mock-spectrum, power-spectrum
// and sightline kernels: the Philox4x32-10 counter-based generator (Salmon et
// al. 2011) with Box-Muller deviates, and a shared-memory Stockham FFT.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lya {
namespace fftd {

// ---- Philox4x32-10 ------------------------------------------------------------------
struct U4 { unsigned int x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, unsigned int k0, unsigned int k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned int lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned int lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// A standard normal deviate for (column, row): Box-Muller on the first two
// words, uniforms (w >> 8 + 1/2) 2^-24 (exact in FP32).
__device__ __forceinline__ float normal_deviate(unsigned long long seed, long long col, long long row)
{
    const U4 r = philox4x32_10(U4{(unsigned int)col, (unsigned int)row, (unsigned int)((unsigned long long)row >> 32), 0u},
                               (unsigned int)seed, (unsigned int)(seed >> 32));
    const float u1 = ((float)(r.x >> 8) + 0.5f) * 5.9604644775390625e-8f;   // 2^-24
    const float u2 = ((float)(r.y >> 8) + 0.5f) * 5.9604644775390625e-8f;
    return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// A pair of independent standard normal deviates from the first two Philox
// words (Box-Muller, uniforms (w >> 8 + 1/2) 2^-24).
__device__ __forceinline__ float2 normal_pair(U4 r)
{
    const float u1 = ((float)(r.x >> 8) + 0.5f) * 5.9604644775390625e-8f;
    const float u2 = ((float)(r.y >> 8) + 0.5f) * 5.9604644775390625e-8f;
    const float m = sqrtf(-2.f * logf(u1));
    float s, c;
    sincospif(2.f * u2, &s, &c);
    return make_float2(m * c, m * s);
}

// ---- Stockham FFT in shared memory --------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// T[j] = exp(-2 pi i j / N), j = 0 .. N-1, filled by the whole block (the
// caller synchronises before use).
__device__ inline void fft_twiddles(float2* T, int N)
{
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        float s, c;
        sincospif(-2.f * (float)j / (float)N, &s, &c);
        T[j] = make_float2(c, s);
    }
}

// t = p s + q for t < 2^16: the float quotient is within 1/s of the true one,
// so one correction either way makes it exact.
__device__ __forceinline__ void divmod_small(int t, int s, float inv_s, int& p, int& q)
{
    p = (int)((float)t * inv_s);
    q = t - p * s;
    if (q >= s) { ++p; q -= s; }
    if (q < 0) { --p; q += s; }
}

// One Stockham pass of radix R on length-N data: x -> y, n the current
// sub-length, s the current stride (n s = N); the twiddle of butterfly p,
// output k is exp(-2 pi i p k / n) = T[p k s] (p k < n).
template <int R>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ x, float2* __restrict__ y,
                                              const float2* __restrict__ T, int N, int n, int s)
{
    const int m = n / R;
    const float inv_s = 1.f / (float)s;
    for (int t = threadIdx.x; t < N / R; t += blockDim.x) {
        int p, q;
        divmod_small(t, s, inv_s, p, q);
        float2 a[R];
#pragma unroll
        for (int j = 0; j < R; ++j) a[j] = x[q + s * (p + j * m)];
        float2 c[R];
        if constexpr (R == 2) {
            c[0] = make_float2(a[0].x + a[1].x, a[0].y + a[1].y);
            c[1] = make_float2(a[0].x - a[1].x, a[0].y - a[1].y);
        } else {
            // w3 = exp(-2 pi i / 3) = (-1/2, -sqrt(3)/2)
            const float h = 0.86602540378443865f;
            const float2 s12 = make_float2(a[1].x + a[2].x, a[1].y + a[2].y);
            const float2 d12 = make_float2(a[1].x - a[2].x, a[1].y - a[2].y);
            c[0] = make_float2(a[0].x + s12.x, a[0].y + s12.y);
            const float2 mid = make_float2(a[0].x - 0.5f * s12.x, a[0].y - 0.5f * s12.y);
            // -i h d12 = (h d12.y, -h d12.x)
            c[1] = make_float2(mid.x + h * d12.y, mid.y - h * d12.x);
            c[2] = make_float2(mid.x - h * d12.y, mid.y + h * d12.x);
        }
        y[q + s * (R * p)] = c[0];
#pragma unroll
        for (int k = 1; k < R; ++k) y[q + s * (R * p + k)] = cmul(c[k], T[p * k * s]);
    }
}

// Forward transform X_n = sum_j x_j exp(-2 pi i j n / N) of x (in X) for
// N = 2^a 3^b <= 2^16, ping-ponging between X and Y: radix-3 passes, then
// radix-2; T from fft_twiddles.  Returns the buffer that holds the result;
// called by the whole block, ends with a barrier.
__device__ inline float2* fft_stockham(float2* X, float2* Y, const float2* T, int N)
{
    float2* src = X;
    float2* dst = Y;
    int n = N, s = 1;
    while (n % 3 == 0) {
        stockham_pass<3>(src, dst, T, N, n, s);
        __syncthreads();
        n /= 3;
        s *= 3;
        float2* t = src; src = dst; dst = t;
    }
    while (n > 1) {
        stockham_pass<2>(src, dst, T, N, n, s);
        __syncthreads();
        n /= 2;
        s *= 2;
        float2* t = src; src = dst; dst = t;
    }
    return src;
}


// Batched, strided form for 2D transforms in shared memory: B transforms of
// length Nf, transform b's element i at b * bs + i * es (rows: bs = Nf, es = 1;
// columns: bs = 1, es = Nf).  T holds the Nf twiddles.
template <int R>
__device__ __forceinline__ void stockham_pass_batched(const float2* __restrict__ x, float2* __restrict__ y,
                                                      const float2* __restrict__ T, int Nf, int n, int s, int B,
                                                      int bs, int es)
{
    const int m = n / R, per = Nf / R;
    const float inv_s = 1.f / (float)s, inv_per = 1.f / (float)per, inv_b = 1.f / (float)B;
    for (int t = threadIdx.x; t < B * per; t += blockDim.x) {
        // consecutive threads walk the unit-stride direction: along a
        // transform when es = 1, across transforms when bs = 1 (so a warp's
        // accesses never stride by a whole row)
        int b, tt, p, q;
        if (es == 1) divmod_small(t, per, inv_per, b, tt);
        else divmod_small(t, B, inv_b, tt, b);
        divmod_small(tt, s, inv_s, p, q);
        const int base = b * bs;
        float2 a[R];
#pragma unroll
        for (int j = 0; j < R; ++j) a[j] = x[base + es * (q + s * (p + j * m))];
        float2 c[R];
        if constexpr (R == 2) {
            c[0] = make_float2(a[0].x + a[1].x, a[0].y + a[1].y);
            c[1] = make_float2(a[0].x - a[1].x, a[0].y - a[1].y);
        } else {
            const float h = 0.86602540378443865f;
            const float2 s12 = make_float2(a[1].x + a[2].x, a[1].y + a[2].y);
            const float2 d12 = make_float2(a[1].x - a[2].x, a[1].y - a[2].y);
            c[0] = make_float2(a[0].x + s12.x, a[0].y + s12.y);
            const float2 mid = make_float2(a[0].x - 0.5f * s12.x, a[0].y - 0.5f * s12.y);
            c[1] = make_float2(mid.x + h * d12.y, mid.y - h * d12.x);
            c[2] = make_float2(mid.x - h * d12.y, mid.y + h * d12.x);
        }
        y[base + es * (q + s * (R * p))] = c[0];
#pragma unroll
        for (int k = 1; k < R; ++k) y[base + es * (q + s * (R * p + k))] = cmul(c[k], T[p * k * s]);
    }
}

// B strided transforms of length Nf = 2^a 3^b (B Nf <= 2^16), ping-ponging
// between X and Y; returns the buffer holding the result.  Ends with a barrier.
__device__ inline float2* fft_stockham_batched(float2* X, float2* Y, const float2* T, int Nf, int B, int bs, int es)
{
    float2* src = X;
    float2* dst = Y;
    int n = Nf, s = 1;
    while (n % 3 == 0) {
        stockham_pass_batched<3>(src, dst, T, Nf, n, s, B, bs, es);
        __syncthreads();
        n /= 3;
        s *= 3;
        float2* t = src; src = dst; dst = t;
    }
    while (n > 1) {
        stockham_pass_batched<2>(src, dst, T, Nf, n, s, B, bs, es);
        __syncthreads();
        n /= 2;
        s *= 2;
        float2* t = src; src = dst; dst = t;
    }
    return src;
}

}  // namespace fftd
}  // namespace lya
