// lya_internal.h -- host/device structures passed from the C-ABI layer to the
// kernel launchers.  Not part of the public ABI.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "lya.h"

namespace lya {
struct FieldCheck;
}

// A field: its description and device arrays (owned or borrowed).
struct lya_field_s {
    lya_field_desc desc;
    float* rho = nullptr;
    float* vpec = nullptr;
    float* temp = nullptr;
    bool owned = false;
    int* d_err = nullptr;            // device error word of extract launches
    lya::FieldCheck* d_check = nullptr;
    float temp_max = 0.f;            // largest T where rho > 0 (stored-T fields)
    float rho_max = 0.f;             // largest rho
    float rho_minpos = 0.f;          // smallest rho > 0
    int device = 0;
    std::atomic<int> users{0};       // server requests not yet finished
    // chunked loads from host memory: the check runs on its own stream, each
    // piece once the host has seen its copies' event (created at the first load)
    cudaStream_t check_stream = nullptr;
    cudaEvent_t piece_ev[8] = {};
};

namespace lya {

// Everything the optical-depth kernel needs, precomputed in FP64 on the host
// and handed to the device in both FP32 and FP64 forms.
struct TauLaunch {
    const float* rho;
    const float* vpec;
    const float* temp;        // nullptr in power-law mode
    const int64_t* ids;       // nullptr: row r is skewer r
    int64_t n_rows;           // skewers to extract (grid size)
    int64_t n_skewers;        // skewers in the field (id bound)
    int64_t pf_ahead;         // tile kernel: CTA r prefetches row r + pf_ahead into L2 (0: none)
    int n_pix;
    float* tau_out;           // [n_rows][n_pix]
    int* err;                 // device error word: bit 0 = skewer id out of range, bit 1 = input
                              // changed under the kernel, bit 2 = failed bounds check (LYA_CHECKED)
    int w_max;                // bound on every source's window half-width, pixels (<= (n_pix-1)/2)

    int t_mode;               // 0 stored T, 1 power law (Eq. 5)
    int profile;              // LYA_PROFILE_SAMPLED (Eq. 6) or LYA_PROFILE_AVERAGED
    int exp_method;           // LYA_EXP_*
    // FP32 forms
    float du_hi, du_lo;       // pixel velocity width as a double-float (km/s)
    float inv_du;             // 1/du
    float c_coef;             // sqrt(log2 e) / b(1e4 K), s/km
    float h_coef;             // nsigma * sqrt(log2 e): window half-width = h_coef / a
    float K;                  // Eq. 6 prefactor times Eq. 4 constants (see api)
    float T0, gm1, pivot;     // power law: T = T0 min(rho, pivot)^gm1
    float lT0;                // log2(T0 / 1e4 K)
    float lpivot;             // log2(pivot) (+inf: no pivot)
    float lK;                 // log2(K)
    // FP64 forms (the FP64 comparator kernel)
    double du_d, inv_du_d, c_coef_d, h_coef_d, K_d, T0_d, gm1_d, pivot_d;
};

// Validate extraction parameters against a field and fill the field- and
// parameter-dependent members of *out (everything but ids, n_rows, tau_out).
lya_status make_tau_launch(lya_field f, const lya_extract_params* p, TauLaunch* out);

// Launch the optical-depth kernel for the requested precision.
cudaError_t launch_tau(const TauLaunch& L, int precision, cudaStream_t stream);



// Shared-memory bytes the optical-depth kernel needs for n_pix pixels and a
// window bound w_max (the kernel variant is chosen by what fits).
size_t tau_smem_bytes(int n_pix, int w_max, int precision);

// Maximum dynamic shared memory a block may opt into on this device.
size_t max_dynamic_smem();

// Mean-flux root-find (Sec. 2.3) over n device values of tau; writes A to
// *A_out and, if flux_out is not null, F = exp(-A tau).  Returns a lya_status.
// With stats_out, the final flux pass also gathers the statistics of F
// (Sec. 2.3, 5.2) into *stats_out.
lya_status mean_flux_solve(const float* tau, int64_t n, double target, double tol,
                           int max_iter, double* A_out, float* flux_out,
                           cudaStream_t stream, lya_flux_stats_t* stats_out = nullptr);

// The same root-find with its scratch in a fixed device array (no allocation).
lya_status mean_flux_solve_noalloc(const float* tau, int64_t n, double target, double tol,
                                   int max_iter, double* A_out, float* flux_out,
                                   cudaStream_t stream);

// Per-device shares of a root-find split over devices: tau moments (sum,
// zeros, invalid), the sums at a given A, and F at a given A.
lya_status tau_moments_run(const float* tau, int64_t n, double* out3, cudaStream_t stream);
lya_status mean_flux_sums_run(const float* tau, int64_t n, double A, double* out3, cudaStream_t stream);
lya_status flux_at_run(const float* tau, int64_t n, double A, float* flux, cudaStream_t stream);

// The split root-find's host steps (lya_mean_flux_start / _step) and its
// whole driver with an all-reduce callback (lya_rescale_mean_flux_sharded).
lya_status mean_flux_start(const double totals[4], double target, double tol, int max_iter,
                           lya_mean_flux_iter* it);
lya_status mean_flux_step(lya_mean_flux_iter* it, const double sums[3]);
lya_status mean_flux_sharded(const float* tau, int64_t n, double target, double tol, int max_iter,
                             lya_allreduce_fn allreduce, void* user, double* A_out, int* iters_out, float* flux_out,
                             cudaStream_t stream);

// Flux statistics (Sec. 2.3, 5.2) over n device flux values.
lya_status flux_stats_run(const float* flux, int64_t n, lya_flux_stats_t* out,
                          cudaStream_t stream);

// Mock spectra (Sec. 4): instrument profile of half-width W pixels (0: none,
// sigma = du / du_over_sigma), resampling to pixels ratio times wider, n_out
// output pixels, noise sigma (0: none) from Philox keyed by seed, rows
// counted from row0.
lya_status mock_spectra_run(const float* flux, int64_t n_skewers, int n_pix, int n_out, int W,
                            double du_over_sigma, double ratio, double noise, uint64_t seed,
                            int64_t row0, float* out, cudaStream_t stream);
size_t mock_smem_bytes(int n_pix, int n_out, double ratio, int W);

// Line-of-sight flux power (Sec. 5.3): sums over skewers of |X_n|^2 of
// delta_F = F/<F> - 1, n = 0..N/2 (host), and <F>.  n_pix = 2^a 3^b.
lya_status flux_power_run(const float* flux, int64_t n_skewers, int n_pix, double* sums_out,
                          double* mean_out, cudaStream_t stream);
size_t flux_ps_smem_bytes(int n_pix);

// Lines of sight generated in Fourier space (Sec. 2.1-2.2): rows
// first_id .. first_id + n_ids - 1 of a field; n_pix = 2^a 3^b, a >= 1.
lya_status sightlines_run(int n_pix, double box, double k_j, double sigma, double k_f, double aH,
                          uint64_t seed, int64_t first_id, int64_t n_ids, float* rho, float* vpec,
                          cudaStream_t stream);
size_t sightline_smem_bytes(int n_pix);

// 3D flux power of lines of sight on an n_perp^2 transverse grid with the
// Eq. 7 reconstruction: per shell {sum P_true, sum P_box, sum |m|, modes}.
lya_status flux_power_3d_run(const float* flux, const int* cells_host, int64_t n_los, int n_pix, int n_perp,
                             double box, double noise_sigma, double* shells_out, int n_shells,
                             cudaStream_t stream);
size_t flux3d_los_smem_bytes(int n_pix);
size_t flux3d_plane_smem_bytes(int n_perp, int n_pix);
int flux3d_shells(int n_perp, int n_pix);

// Field validation: counts out-of-domain values and finds the largest T.
struct FieldCheck {
    unsigned long long bad_rho, bad_vpec, bad_temp;
    unsigned int temp_max_bits;      // largest T where rho > 0 (float bits)
    unsigned int rho_max_bits;       // largest rho (float bits)
    unsigned int rho_minpos_bits;    // smallest rho > 0 (float bits; 0x7f800000 if none)
};
cudaError_t launch_field_check(const float* rho, const float* vpec, const float* temp,
                               int64_t n, FieldCheck* d_out, cudaStream_t stream);
// The same in parts: set the totals empty, then check any number of ranges
// into them (atomics), e.g. each piece of a chunked load as it lands.
cudaError_t launch_field_check_init(FieldCheck* d_out, cudaStream_t stream);
cudaError_t launch_field_check_range(const float* rho, const float* vpec, const float* temp,
                                     int64_t n, FieldCheck* d_out, cudaStream_t stream);

// Count one kernel launch (lya_kernel_launches).
void count_launch(int n = 1);
uint64_t launches_so_far();

// Number of SMs of the current device (cached).
int sm_count();

// Stream-ordered scratch for the library's per-call buffers (root-find state
// and partials, statistics, transforms), from a memory pool the library owns
// on the current device, created at first use with its release threshold at
// the maximum: its memory stays mapped between calls instead of going back
// at every synchronise (the default pool's behaviour, which made each call
// map its buffers again).  Freed with cudaFreeAsync like any pool block.
cudaError_t scratch_malloc(void** p, size_t bytes, cudaStream_t stream);

// That pool on the current device (created if needed), or nullptr.
cudaMemPool_t scratch_pool();

}  // namespace lya
