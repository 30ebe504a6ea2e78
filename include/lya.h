/*
 * lya.h -- C ABI of the GB300 Lyman-alpha optical-depth library (liblya.so).
 *
 * The library extracts H I optical depth along skewers through a gridded
 * density / velocity / temperature field and turns it into transmitted flux,
 * following the semi-analytic method of Greig, Bolton & Wyithe (2011):
 *
 *   Eq. 5   T = T0 (1+delta)^(gamma-1), held at T(1+delta = 10) above the
 *           pivot (power-law mode), or T read per pixel (stored mode);
 *   Eq. 4   n_HI ~ (T/1e4)^-0.7 (1+delta)^2 (fluctuating Gunn-Peterson);
 *   Eq. 6   tau(i) = (c sigma_a dR / sqrt(pi)) sum_j n_HI(j)/b(j)
 *                    exp(-((v_H(i) - u(j))/b(j))^2),  b = sqrt(2 k T/m_H),
 *           u(j) = v_H(j) + v_pec(j), summed periodically along the skewer;
 *   Sec 2.3 F = exp(-A tau) with A solved so that <F> hits a target;
 *   Sec 5.2 flux statistics: <F>, Var F, tau_eff = -ln<F>, 21-bin PDF.
 *
 * Conventions shared by every entry point:
 *   - Arrays are FP32, row-major [n_skewers][n_pix]: one skewer is n_pix
 *     contiguous floats.  Velocities are km/s, temperatures K, lengths
 *     h^-1 Mpc (comoving).  "rho" is 1 + delta_b (density over the mean).
 *   - "Device" pointers are CUDA global-memory pointers on the current
 *     device; "host" pointers are ordinary (preferably pinned) memory.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are stream-ordered; a call that returns a host value (A, statistics)
 *     synchronises that stream before returning.
 *   - Every call returns a lya_status.  No C++ exception crosses the ABI.
 *     Arguments are validated on the host before any launch; an invalid
 *     argument returns LYA_EINVAL and launches nothing.
 *   - The caller owns every buffer it passes in; a field owns (or, when
 *     borrowed, references) its device arrays until lya_destroy_field.
 */
#ifndef LYA_H
#define LYA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LYA_OK = 0,
    LYA_EINVAL = -1,     /* bad argument, or a field value outside its domain */
    LYA_ENOMEM = -2,     /* a device allocation failed                        */
    LYA_ECUDA = -3,      /* a CUDA runtime call failed                        */
    LYA_ENOCONV = -4,    /* the mean-flux root-find did not converge / no root */
    LYA_ETIMEDOUT = -5,  /* a bounded device wait gave up                     */
    LYA_EBUDGET = -6,    /* a request does not fit the memory budget          */
    LYA_EDEVICE = -7,    /* no usable sm_103 device                           */
    LYA_EBUSY = -8       /* object in use (field held by a server request, or  */
                         /* a server call that needs an idle server)          */
} lya_status;

/* Opaque handle to a field resident in device memory. */
typedef struct lya_field_s* lya_field;

/* Geometry and cosmology of a field (defaults: the paper's cosmology, Sec. 2:
 * h = 0.72, Omega_m = 0.26, Omega_L = 0.74, Omega_b = 0.0444). */
typedef struct {
    double box;          /* comoving skewer length, h^-1 Mpc (> 0)            */
    double z;            /* redshift of the spectra (> -1)                     */
    double h, omega_m, omega_l, omega_b;
    double y_he;         /* helium mass fraction in nbar_H of Eq. 4 (0.24)     */
    int64_t n_skewers;   /* >= 1                                              */
    int64_t n_pix;       /* pixels per skewer, 16 <= n_pix <= 8192, even      */
    int has_temp;        /* 1: the field carries a temperature array          */
} lya_field_desc;

/* Source of the arrays passed to lya_create_field / lya_field_load. */
enum {
    LYA_SRC_HOST = 0,          /* host memory: copied to the device            */
    LYA_SRC_DEVICE_COPY = 1,   /* device memory: copied into field-owned memory */
    LYA_SRC_DEVICE_BORROW = 2  /* device memory: referenced, not copied; the
                                  caller keeps it alive and unchanged while the
                                  field exists (create only); each array must
                                  start on a 16-byte boundary (LYA_EINVAL
                                  otherwise)                                   */
};

/* Accumulation precision of the pair sum (Eq. 6). */
enum {
    LYA_PREC_F32_COMPENSATED = 0, /* FP32 pairs, compensated (Kahan) sum       */
    LYA_PREC_F32_NAIVE = 1,       /* FP32 pairs, plain FP32 sum                 */
    LYA_PREC_F64 = 2              /* FP64 throughout (comparator; n_pix <= 4096) */
};

/* Per-extraction physics (Eq. 4-6). */
typedef struct {
    int t_mode;          /* 0: stored T (field must have one); 1: Eq. 5 power law */
    double T0;           /* K, power-law mode                                  */
    double gamma;        /* power-law slope, power-law mode                    */
    double delta_pivot;  /* 1+delta above which T is constant (10; INFINITY = off) */
    double gamma12;      /* H I photo-ionisation rate / 1e-12 s^-1 (> 0)       */
    double nsigma;       /* pairs with |v_H(i)-u(j)| <= nsigma b(j) are summed (8) */
    int precision;       /* LYA_PREC_*                                         */
    int profile;         /* LYA_PROFILE_SAMPLED: Eq. 6 as written, each line's   */
                         /* Gaussian sampled at the pixel velocity v_H(i);     */
                         /* LYA_PROFILE_AVERAGED: the Gaussian averaged over   */
                         /* the pixel's velocity cell [v_H - du/2, v_H + du/2) */
                         /* (column density then conserved exactly for any     */
                         /* b/du; F32 precisions only)                          */
    int exp_method;      /* how the pair sum's exponentials exp(-(d/b)^2) of   */
                         /* Eq. 6 are evaluated (F32 precisions, sampled        */
                         /* profile; extraction only, not the serving loop):   */
                         /* LYA_EXP_MUFU: one MUFU ex2 per pair (default);     */
                         /* LYA_EXP_RECURRENCE: a lane takes four pixels of a  */
                         /* line from three exponentials by the Gaussian       */
                         /* recurrence (Greengard & Lee 2004), lines with      */
                         /* b >= 2.4 du; LYA_EXP_POLY_SPLIT: one in four       */
                         /* exponentials by an FMA-pipe polynomial.  All three */
                         /* meet the same tolerance; they differ in which      */
                         /* pipe does the work                                 */
} lya_extract_params;

enum { LYA_PROFILE_SAMPLED = 0, LYA_PROFILE_AVERAGED = 1 };
enum { LYA_EXP_MUFU = 0, LYA_EXP_RECURRENCE = 1, LYA_EXP_POLY_SPLIT = 2 };

typedef struct {
    double mean_flux;    /* <F>                                               */
    double var_flux;     /* population variance of F                          */
    double tau_eff;      /* -ln <F>                                           */
    int64_t pdf[21];     /* bin k counts (2k-1)/40 <= F < (2k+1)/40 (Sec. 5.2) */
    int64_t n;           /* number of values                                  */
} lya_flux_stats_t;

/*
 * Create a field of desc->n_skewers skewers x desc->n_pix pixels (Sec. 2.3:
 * the gridded density, peculiar velocity and temperature the spectra are
 * drawn from).  rho = 1+delta (>= 0, finite), vpec in km/s (finite), temp in
 * K (> 0 where rho > 0; NULL iff desc->has_temp == 0).  src is LYA_SRC_*.
 * The field validates every value once on the device and records the largest
 * temperature (it bounds the line width).  Returns LYA_EINVAL for a bad
 * descriptor or an out-of-domain value, LYA_ENOMEM if device memory runs out.
 */
lya_status lya_create_field(const lya_field_desc* desc, const float* rho,
                            const float* vpec, const float* temp, int src,
                            void* stream, lya_field* out);

/*
 * Overwrite the arrays of an owned field with new values of the same shape
 * (src = LYA_SRC_HOST or LYA_SRC_DEVICE_COPY), validating them as above.
 * Stream-ordered; synchronises the stream to read the validation result.
 */
lya_status lya_field_load(lya_field field, const float* rho, const float* vpec,
                          const float* temp, int src, void* stream);

/* Release a field (waits for work on the device to finish first). */
lya_status lya_destroy_field(lya_field field);

/*
 * Read and clear the field's device error word (set by lya_extract_skewers
 * when a skewer id is out of range; in a library built with -DLYA_CHECKED
 * also when a bounds check of the optical-depth kernel fails).  Synchronises
 * the stream; returns LYA_EINVAL if an extraction since the last call set it.
 */
lya_status lya_field_status(lya_field field, void* stream);

/* Shape of a field. */
lya_status lya_field_shape(lya_field field, int64_t* n_skewers, int64_t* n_pix);

/*
 * Optical depth along skewers (Eq. 4-6): tau_out[r][i] for the skewers
 * skewer_ids[r], r < n_ids (a DEVICE array of int64 in [0, n_skewers); NULL
 * means all skewers in order, with n_ids == n_skewers).  tau_out is a device
 * array of n_ids * n_pix floats, owned by the caller.  The sum is periodic
 * over the skewer (each source at the image nearest each pixel) and keeps
 * every pair with |v_H(i) - u(j)| <= nsigma b(j) (a superset of them is
 * allowed).  Out-of-range ids are not checked on the
 * host; the kernel writes zeros for them and returns LYA_EINVAL at the next
 * synchronising call on the field.
 */
lya_status lya_extract_skewers(lya_field field, const lya_extract_params* params,
                               const int64_t* skewer_ids, int64_t n_ids,
                               float* tau_out, void* stream);

/*
 * Mean-flux rescaling (Sec. 2.3): find A with <exp(-A tau)> = target over all
 * n device values tau (every pixel of every skewer, equally weighted).
 * A safeguarded Halley/Newton/bisection iteration on the device, started from
 * a sample of tau, with <exp(-A tau)> evaluated to ~1e-13 (double-float
 * exponentials, FP64 sums); it stops when |<exp(-A tau)> - target| <= tol, or
 * when its last Newton step is certified by Taylor's bound to land within
 * tol, or when the step stalls at FP64 resolution.  *A_out receives A (host).
 * If flux_out (device, n floats) is not NULL it receives F = exp(-A tau) in
 * FP32, within 6e-8 plus one rounding of exp(-A tau) at the returned A
 * (written by the last evaluation pass when its step moved A little enough,
 * else by a flux pass at the final A).  Returns LYA_EINVAL if target is not in (0,1),
 * tau holds a negative or non-finite value or all tau are 0; LYA_ENOCONV if
 * no A reaches the target (too many tau = 0) or max_iter is exhausted.
 * Synchronises the stream.
 */
lya_status lya_rescale_mean_flux(const float* tau, int64_t n, double target,
                                 double tol, int max_iter, double* A_out,
                                 float* flux_out, void* stream);

/*
 * lya_rescale_mean_flux without any device allocation.  The paper has no
 * counterpart: this is a deployment variant for callers that cannot call
 * cudaMalloc: plug-ins whose host application forbids allocation after
 * start-up, or a service whose device-memory budget is already handed out.
 * Arguments, results and errors are those of lya_rescale_mean_flux.
 *
 * Its scratch (the root-find state and one partial sum per CTA) is a fixed
 * 64 KiB device array inside the library, present on every GPU that loads
 * it until the process exits; the reduction therefore uses at most 1024
 * CTAs, which still covers any n.  The first call on a device looks up the
 * array's device address (once per device, with that device current).  At
 * the start of every call a kernel zeroes and sets the whole state, and every
 * CTA writes its partial before the last CTA reads them, so nothing carries
 * over from an earlier call; but all calls share the one array: calls whose
 * work overlaps on the GPU (other streams, other host threads on the same
 * device) race and must be serialised by the caller.  The call reads the
 * state back and synchronises the stream after every round of passes, so the
 * stream must not be capturing a CUDA graph.
 */
lya_status lya_rescale_mean_flux_noalloc(const float* tau, int64_t n, double target,
                                         double tol, int max_iter, double* A_out,
                                         float* flux_out, void* stream);

/*
 * lya_rescale_mean_flux followed by lya_flux_stats of the F it writes, with
 * the statistics gathered in the pass that writes F instead of a separate
 * read of F (Sec. 2.3, Sec. 5.2).  flux_out may be NULL (the statistics are
 * still those of exp(-A tau) in FP32).  Arguments, results and
 * errors are those of the two calls; stats_out must not be NULL.
 * Synchronises the stream.
 */
lya_status lya_rescale_mean_flux_stats(const float* tau, int64_t n, double target_mean_flux,
                                       double tol, int max_iter, double* A_out,
                                       float* flux_out, lya_flux_stats_t* stats_out,
                                       void* stream);

/*
 * Per-device shares of the mean-flux root-find (Sec. 2.3) when one request's
 * pixels are split over several devices or processes: each computes its
 * share, the shares are summed over all parts (an all-reduce of three
 * numbers) and stepped with lya_mean_flux_step below, then each part writes
 * its F with lya_flux_at (lya_rescale_mean_flux_sharded does all of it).
 *   lya_tau_moments:    out = { sum tau, number of tau == 0, number of
 *                       negative or non-finite tau } over n device values.
 *   lya_mean_flux_sums: out = { sum e, sum tau e, sum tau^2 e }, e = exp(-A tau):
 *                       sum e to ~1e-13 relative (double-float exponentials,
 *                       FP64 sums), the other two in compensated FP32 / FP64.
 *   lya_flux_at:        flux_out[i] = exp(-A tau[i]) (device, n floats).
 * The first two synchronise the stream; A must be finite and >= 0.
 */
lya_status lya_tau_moments(const float* tau, int64_t n, double out[3], void* stream);
lya_status lya_mean_flux_sums(const float* tau, int64_t n, double A, double out[3], void* stream);
lya_status lya_flux_at(const float* tau, int64_t n, double A, float* flux_out, void* stream);

/*
 * The Sec. 2.3 iteration for a request split over several parts, stepped on
 * the host from the parts' summed shares (no device work; every part holds
 * its own copy and takes the same steps from the same sums):
 *   lya_mean_flux_start: totals = { sum tau, number of tau == 0, number of
 *     invalid tau, number of values } over all parts (each part's
 *     lya_tau_moments and its n, summed); target in (0, 1), tol > 0,
 *     max_iter >= 1.  Starts Newton at the Jensen bound A0 = -ln(target)/<tau>
 *     (below the root).  LYA_EINVAL for an invalid value or all tau = 0,
 *     LYA_ENOCONV when no A reaches the target (too many tau = 0); the
 *     iteration is then already done with that status.
 *   lya_mean_flux_step: sums = { sum e, sum tau e, sum tau^2 e } at it->A over
 *     all parts (each part's lya_mean_flux_sums, summed), e = exp(-A tau).
 *     One safeguarded step (Halley, else Newton, else bisection inside the
 *     bracket).  The iteration ends (it->done, it->status = LYA_OK) when
 *     |<e> - target| <= tol at it->A, or when Taylor's bound certifies that
 *     the Newton step lands within tol (it->A is then that point and it->g
 *     the bound), or when the step stalls at FP64 resolution; it ends with
 *     LYA_ENOCONV after max_iter steps.  Returns it->status once done, else
 *     LYA_OK.
 */
typedef struct {
    double A;            /* current A (the final one once done)                  */
    double lo, hi;       /* bracket of the root                                  */
    double g;            /* last <e> - target, or the certified bound on |g|     */
    int iter, max_iter;  /* steps taken, step limit                              */
    int done;            /* 1 once the iteration has ended                       */
    lya_status status;   /* LYA_OK when converged; the error otherwise          */
    double target, tol, n;   /* target <F>, tolerance, values over all parts    */
} lya_mean_flux_iter;

lya_status lya_mean_flux_start(const double totals[4], double target, double tol, int max_iter,
                               lya_mean_flux_iter* it);
lya_status lya_mean_flux_step(lya_mean_flux_iter* it, const double sums[3]);

/*
 * The whole split root-find in one call per part (Sec. 2.3): every part calls
 * it with its own n device values tau (n may be 0), the same target, tol and
 * max_iter, and an all-reduce callback that replaces values[0 .. count) by
 * their sums over all parts (and returns 0; anything else ends the call with
 * LYA_ECUDA).  The library computes the shares, sums them with the callback
 * (one call of 4 values, then one of 3 values per step) and steps the
 * iteration as lya_mean_flux_step; *A_out (identical on every part) and
 * *iters_out (nullable) receive the result, flux_out (device, n floats,
 * nullable) this part's F = exp(-A tau).  Errors as lya_rescale_mean_flux.
 * Synchronises the stream.
 */
typedef int (*lya_allreduce_fn)(double* values, int count, void* user);
lya_status lya_rescale_mean_flux_sharded(const float* tau, int64_t n, double target, double tol, int max_iter,
                                         lya_allreduce_fn allreduce, void* user, double* A_out, int* iters_out,
                                         float* flux_out, void* stream);

/*
 * Flux statistics (Sec. 2.3, Sec. 5.2) over n device values F: mean,
 * population variance, tau_eff = -ln<F> and the 21-bin PDF with bin k holding
 * (2k-1)/40 <= F < (2k+1)/40 (clamped to [0, 20]); the bin decision is exact
 * for FP32 F.  Synchronises the stream.
 */
lya_status lya_flux_stats(const float* flux, int64_t n, lya_flux_stats_t* out,
                          void* stream);

/*
 * Pixel velocity width du (km/s) of a field's skewers: the Hubble-law width
 * H(z) L / (h (1 + z) N) of Sec. 2.3 (Eq. 6 text).
 */
lya_status lya_field_pixel_width(lya_field field, double* du_kms);

/*
 * Mock spectra (Sec. 4): the transmitted flux of each skewer processed to look
 * like an instrument's spectra.  The paper describes the steps in words; this
 * library reads them as:
 *   - instrument profile: periodic discrete convolution with the Gaussian
 *     exp(-(m du)^2 / 2 sigma^2), sigma = FWHM / (2 sqrt(2 ln 2)), over
 *     |m du| <= nsigma sigma, weights normalised to one (fwhm_kms = 0: none);
 *   - resampling: input pixel i is the cell [(i - 1/2) du, (i + 1/2) du) of the
 *     periodic skewer; output pixel k the cell [(k - 1/2) B, (k + 1/2) B),
 *     B = bin_kms (<= 0: du), valued by the cell-overlap mean;
 *   - path cut: floor(min(N du, max_kms) / B) output pixels (max_kms <= 0:
 *     the whole skewer), e.g. the Ly-alpha to Ly-beta path less 3000 km/s;
 *   - noise: (1/snr) g with g standard normal, Box-Muller on Philox4x32-10
 *     (Salmon et al. 2011) with key = seed and counter = (output pixel,
 *     row0 + skewer row, 0, 0) (snr = 0: none).
 * flux: device [n_skewers][n_pix]; out: device [n_skewers][n_out] with n_out
 * from lya_mock_shape.  LYA_EINVAL if 2W + 1 > n_pix for the profile's
 * half-width W pixels, or the skewer does not fit shared memory (n_pix up to
 * ~28,000).  Asynchronous on the stream.
 */
typedef struct {
    double fwhm_kms;     /* instrument FWHM, km/s (0: no profile)                 */
    double bin_kms;      /* output pixel width, km/s (<= 0: the input width)      */
    double snr;          /* S/N per output pixel (0: no noise)                    */
    double max_kms;      /* keep the first max_kms of each skewer (<= 0: all)     */
    double nsigma;       /* profile window half-width in sigma (e.g. 6)          */
    uint64_t seed;       /* noise key                                             */
    int64_t row0;        /* noise counter of the first skewer of the call         */
} lya_mock_params;

lya_status lya_mock_shape(int64_t n_pix, double du_kms, const lya_mock_params* params, int64_t* n_out);
lya_status lya_mock_spectra(const float* flux, int64_t n_skewers, int64_t n_pix, double du_kms,
                            const lya_mock_params* params, float* out, void* stream);

/*
 * Line-of-sight flux power spectrum (Sec. 5.3): with delta_F = F / <F> - 1
 * (<F> over every given pixel), P(k_n) = (du / N) |sum_j delta_j e^{-2 pi i j n / N}|^2
 * averaged over the skewers, k_n = 2 pi n / (N du) s/km, n = 0 .. N/2.
 * flux: device [n_skewers][n_pix] with n_pix = 2^a 3^b; k_out (nullable) and
 * power_out: host arrays of n_pix/2 + 1; mean_flux_out (nullable): <F>.
 * The transforms run in FP32 (two real skewers per complex transform); the
 * sums over skewers in FP64.  Synchronises the stream.
 */
lya_status lya_flux_power_1d(const float* flux, int64_t n_skewers, int64_t n_pix, double du_kms,
                             double* k_out, double* power_out, double* mean_flux_out, void* stream);

/*
 * Lines of sight generated in Fourier space on the device (Sec. 2.1-2.2),
 * one independent 1D realisation per skewer id: modes k_n = 2 pi n / box,
 * n = 1 .. N/2 - 1, with the 1D linear power P_n ~ k_n^-1 exp(-(k_n/k_j)^2)
 * normalised to sum_n P_n = sigma_delta^2; amplitudes (N/2) sqrt(P_n)
 * conj(g_n), g_n = a + i b with a, b standard normal (Box-Muller on
 * Philox4x32-10, key = seed, counter = (n, id)); the Eq. 3 velocity
 * i aH delta_n / k_n (f = 1); the Eq. 1 gas smoothing 1/(1 + k^2/k_f^2) of the
 * density (k_f = 0: none); and the lognormal 1 + delta = exp(delta_b -
 * sigma_b^2/2), sigma_b^2 = sum_n P_n/(1 + k_n^2/k_f^2)^2, in place of the
 * paper's rank-ordered mapping to a hydrodynamical simulation.  Rows
 * first_id .. first_id + n_ids - 1 are written to rho_out and vpec_out
 * (device, [n_ids][n_pix] each); any subset of ids reproduces the same rows.
 * n_pix = 2^a 3^b with a >= 1 (up to 9,216 by shared memory).  The transform
 * runs in FP32.  Asynchronous on the stream.
 */
typedef struct {
    double box;          /* comoving skewer length, h^-1 Mpc                      */
    double z, h, omega_m, omega_l;
    double k_j;          /* power cut-off scale, h Mpc^-1                        */
    double sigma_delta;  /* rms of the linear density contrast                   */
    double k_f;          /* Eq. 1 filtering scale, h Mpc^-1 (0: none)           */
    uint64_t seed;
} lya_sightline_desc;

lya_status lya_generate_sightlines(const lya_sightline_desc* desc, int64_t n_pix, int64_t first_id,
                                   int64_t n_ids, float* rho_out, float* vpec_out, void* stream);

/*
 * 3D flux power spectrum of a set of lines of sight, reconstructed with Eq. 7
 * and spherically averaged.  The lines run
 * along z through a periodic cube of side box (h^-1 Mpc); line i sits at
 * transverse cell cells[i] = ix * n_perp + iy (host array) of an n_perp x
 * n_perp grid.  With delta_F = F / <F> - 1:
 *   P_box(k)  = (V / M^2) |G_k|^2 of delta_F placed at the lines' cells (0
 *               elsewhere) on the n_perp^2 x n_pix grid, V = box^3, M cells;
 *   P_1D(k_z) = (box / n_pix^2) <|D(k_z)|^2> over the lines;
 *   P_2D,w    = box^2 n_los / n_perp^4, the white level of the lines' weights
 *               (the 2D weighting power of the line positions away from k_perp = 0);
 *   P_N       = (box / n_pix) noise_sigma^2 P_2D,w (white noise of rms
 *               noise_sigma per pixel in delta_F; 0 for noiseless spectra);
 *   P_true    = P_box - P_1D P_2D,w - P_N                          (Eq. 7),
 * averaged in shells b <= |k| / k_f < b + 1, k_f = 2 pi / box, b = 0 ..
 * n_shells - 1 (lya_flux_power_3d_shells), each reporting the mean |k|
 * (k_mean, h/Mpc), the mean P_true and P_box (h^-3 Mpc^3) and the number of
 * modes (host arrays of n_shells; k_mean, p_box and n_modes nullable).
 * flux: device [n_los][n_pix], n_pix = 2^a 3^b; n_perp = 2^a 3^b <= 96.
 * Transforms in FP32, sums in FP64.  Synchronises the stream.
 */
lya_status lya_flux_power_3d_shells(int64_t n_pix, int n_perp, int64_t* n_shells);
lya_status lya_flux_power_3d(const float* flux, const int32_t* cells, int64_t n_los, int64_t n_pix, int n_perp,
                             double box, double noise_sigma, double* k_mean, double* p_true, double* p_box,
                             double* n_modes, void* stream);

/* ======================================================================
 * Serving: a persistent request loop over resident fields.
 *
 * The paper has no serving layer; this is the library's front end for many
 * independent extraction requests, each an instance of Eq. 4-6 plus its own
 * mean-flux normalisation (Sec. 2.3).  A server owns a worker thread, a CUDA
 * stream, one device arena of hbm_budget_bytes and a CUDA graph of one step:
 *   - the optical-depth kernel, persistent (one 1024-thread CTA per SM),
 *     over the step's work list: each CTA takes tasks of up to 8 skewers of
 *     one request, split over 1, 2, 4 or 8 warp groups (the group shape of
 *     each skewer length is chosen by lya_server_autotune);
 *   - the mean-flux root-find of every request whose skewers are complete,
 *     all requests in the same passes (init, then two rounds of two Halley
 *     passes and one flux pass that writes F and its statistics).
 * Each step the worker admits queued requests in arrival order while a slot
 * and arena memory are free, plans the step (a request's skewers may be
 * spread over several steps so that short requests do not wait behind long
 * ones), copies the plan to the device, launches the graph and reads back
 * the finished requests.  Requests that arrive while a step runs join the
 * next one.
 *
 * A request holds 8 bytes per pixel of arena memory (tau and F) and one slot
 * until its root-find ends; then tau is freed and F stays until
 * lya_server_release.  The field must outlive the request: lya_destroy_field
 * returns LYA_EBUSY while a request on it is unfinished.
 * ====================================================================== */
typedef struct lya_server_s* lya_server;

typedef struct {
    size_t hbm_budget_bytes; /* arena size: tau and F of admitted requests       */
    int max_slots;           /* requests in flight at once (1..4096)             */
    double step_target_us;   /* estimated optical-depth work per step, us (> 0)  */
    double tol;              /* root-find tolerance on <F> (> 0; e.g. 1e-12)     */
    int max_iter;            /* root-find pass limit (>= 1; e.g. 50)             */
} lya_server_config;

typedef struct {
    int done;                /* 1 when the request has finished                  */
    lya_status status;       /* LYA_OK, or why it failed (valid when done)       */
    double A;                /* the request's mean-flux constant                  */
    int iterations;          /* root-find passes that updated A                  */
    lya_flux_stats_t stats;  /* statistics of the request's F                    */
    const float* flux;       /* device [n_ids][n_pix] F, owned by the server     */
                             /* until lya_server_release; NULL if failed         */
    int64_t n_ids, n_pix;
    uint64_t t_submit_ns, t_admit_ns, t_done_ns;  /* steady-clock stamps         */
} lya_server_result;

typedef struct {
    uint64_t steps;          /* graph launches so far                            */
    uint64_t submitted, completed, failed;
    size_t arena_used, arena_peak, arena_capacity;
    int slots_in_use, queued;
    int group_shift[14];     /* tuned log2(skewers per CTA) for n_pix = 2^k;    */
                             /* -1 where not tuned (a default is used)          */
} lya_server_info_t;

/* Creates a server on the current device.  LYA_ENOMEM if the arena cannot be
 * allocated. */
lya_status lya_server_create(const lya_server_config* cfg, lya_server* out);

/*
 * Times the optical-depth kernel of the server on up to max_rows skewers of
 * `field` with `params` for every group shape that fits the field's skewer
 * length, and keeps the fastest for that length.  The server must be idle
 * (LYA_EBUSY otherwise).  *shift_out (nullable) gets log2(skewers per CTA).
 */
lya_status lya_server_autotune(lya_server srv, lya_field field, const lya_extract_params* params,
                               int64_t max_rows, int* shift_out);

/*
 * Queues one request: skewers ids[0..n_ids) (host array, copied) of `field`
 * extracted with `params` (F32 precisions only), then A solved so that the
 * mean of exp(-A tau) over all its pixels is target_mean_flux.  Returns
 * LYA_EBUDGET if the request alone exceeds the arena, LYA_EINVAL for a bad
 * argument or an id out of range (F32 compensated, sampled profile, MUFU
 * exponentials only), LYA_ECUDA if the server has failed.
 */
lya_status lya_server_submit(lya_server srv, lya_field field, const lya_extract_params* params,
                             const int64_t* ids, int64_t n_ids, double target_mean_flux,
                             uint64_t* ticket);

/* Current state of a request (never blocks). LYA_EINVAL for an unknown ticket. */
lya_status lya_server_poll(lya_server srv, uint64_t ticket, lya_server_result* out);

/* Waits until the request is done or timeout_s passes (LYA_ETIMEDOUT). */
lya_status lya_server_wait(lya_server srv, uint64_t ticket, double timeout_s, lya_server_result* out);

/* Copies a finished request's F (n_ids * n_pix floats) to dst (device) on stream. */
lya_status lya_server_copy_flux(lya_server srv, uint64_t ticket, float* dst, void* stream);

/* Frees a finished request's F and forgets the ticket (LYA_EBUSY if unfinished). */
lya_status lya_server_release(lya_server srv, uint64_t ticket);

lya_status lya_server_info(lya_server srv, lya_server_info_t* out);

/* Stops the worker (unfinished requests fail with LYA_ECUDA), frees everything. */
lya_status lya_server_destroy(lya_server srv);

/* Human-readable text of a status code (static storage). */
const char* lya_strerror(lya_status status);

/*
 * Number of kernels this library has launched in the process so far (a
 * monotone counter; diagnostics for benchmarks).
 */
uint64_t lya_kernel_launches(void);

/*
 * Used-memory high watermark (bytes) of the memory pool the library draws its
 * per-call scratch from on the current device (diagnostics: the allocating
 * calls' root-find state, partials and statistics buffers come from it; the
 * no-alloc root-find takes nothing from it).  The pool is the library's own,
 * created at first use with its release threshold at the maximum, so its
 * memory stays mapped between calls; the caller's pools are not touched.
 * reset != 0 resets the watermark to the memory currently in use, after
 * reading it into *bytes when bytes is not NULL.  LYA_EINVAL: bytes NULL and
 * reset 0; LYA_ECUDA: the pool could not be created.
 */
lya_status lya_scratch_high_watermark(int reset, uint64_t* bytes);

/* Version string of the library build. */
const char* lya_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LYA_H */
