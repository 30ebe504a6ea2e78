/*
 * lya_oracle.c -- plain FP64 CPU oracle for Lyman-alpha optical-depth
 * extraction along skewers (Greig, Bolton & Wyithe 2011, Sec. 2.3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it; the
 * product library never links or calls it, and it shares no code, header,
 * constant or table with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   Eq. 5   T = T0 (1+delta)^(gamma-1) below the pivot 1+delta = 10, and
 *           T(1+delta > 10) = T(1+delta = 10)          (power-law mode), or
 *           T taken as given per pixel                   (stored mode)
 *   Sec 2.3 b = sqrt(2 k_B T / m_H)
 *   Eq. 4   n_HI = 7.24e-6 nbar_H (T/1e4)^-0.7 (Omega_b h^2/0.024)
 *                  Gamma_-12^-1 (1+delta)^2 ((1+z)/4)^3
 *   Eq. 6   tau(i) = (c sigma_a dR / sqrt(pi)) sum_j n_HI(j)/b(j)
 *                  exp(-((v_H(i) - u(j))/b(j))^2),  u(j) = v_H(j) + v_pec(j)
 *           summed over ALL j (no window), with the velocity difference
 *           taken as the nearest periodic image in [-V/2, V/2).
 *   Sec 2.3 F = exp(-A tau), A solved from <exp(-A tau)> = F_target over
 *           every pixel of every skewer (Newton from the Jensen bound).
 *   Sec 5.2 flux PDF: 21 bins of width 0.05 centred on 0, 0.05, ..., 1,
 *           bin k holding (2k-1)/40 <= F < (2k+1)/40.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - nbar_H is the mean TOTAL hydrogen density (1-Y) Omega_b rho_crit
 *     (1+z)^3 / m_H with Y = 0.24 (the 7.24e-6 factor is the neutral
 *     fraction; the paper's wording "neutral" is read as a slip).
 *   - Eq. 6's sum is periodic: nearest image, ties at exactly +V/2 go to -V/2.
 *   - v_H(i) = i * du; only differences enter.
 *   - A pixel with 1+delta = 0 has n_HI = 0 and contributes nothing.
 *   - dR is the proper pixel width L/(h (1+z) N) Mpc and du = H(z) dR.
 *
 * Precision: every quantity is FP64; FP32 inputs are promoted exactly.
 * The tau sum is a plain "+=" in index order.  The mean-flux sums run over
 * up to ~1e9 pixels, so they use Neumaier (compensated) summation, which
 * only makes the FP64 mean more exact.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- physical constants (cgs) ------------------------------------------ */
#define ORC_C_CMS      2.99792458e10        /* speed of light, cm/s          */
#define ORC_SIGMA_A    4.48e-18             /* Ly-a cross-section, cm^2 (Sec 2.3) */
#define ORC_KB         1.380649e-16         /* Boltzmann, erg/K              */
#define ORC_MH         1.6735575e-24        /* hydrogen atom mass, g         */
#define ORC_MPC_CM     3.0856775814913673e24/* 1 Mpc in cm                   */
#define ORC_G_CGS      6.67430e-8           /* Newton's G, cm^3 g^-1 s^-2    */
#define ORC_KMS_CMS    1.0e5                /* km/s -> cm/s                  */
#define ORC_PI         3.14159265358979323846

typedef struct {
    double box;          /* comoving length of a skewer, h^-1 Mpc            */
    double z;            /* redshift                                          */
    double h, omega_m, omega_l, omega_b;
    double y_he;         /* helium mass fraction used for nbar_H              */
    int    t_mode;       /* 0: T given per pixel; 1: power law from delta     */
    double T0, gamma;    /* Eq. 5                                             */
    double delta_pivot;  /* 1+delta above which T is held constant (10)       */
    double gamma12;      /* photo-ionisation rate in 1e-12 s^-1 (Eq. 4)       */
    int    profile;      /* 0: Eq. 6 as written, the line profile sampled at the
                          * pixel velocity; 1: the profile averaged over the
                          * pixel's velocity cell [v_H - du/2, v_H + du/2)      */
} orc_params;

/* H(z) in km/s/Mpc for a flat LCDM background (Sec. 2, cosmology). */
double orc_hubble(const orc_params* p)
{
    double a3 = (1.0 + p->z) * (1.0 + p->z) * (1.0 + p->z);
    return 100.0 * p->h * sqrt(p->omega_m * a3 + p->omega_l);
}

/* dR: proper width of one pixel, in cm (Eq. 6). */
double orc_pixel_proper_cm(const orc_params* p, int64_t n_pix)
{
    double mpc = p->box / (p->h * (1.0 + p->z) * (double)n_pix);
    return mpc * ORC_MPC_CM;
}

/* du: Hubble-velocity width of one pixel, km/s: H(z) times the proper width. */
double orc_pixel_velocity(const orc_params* p, int64_t n_pix)
{
    double mpc = p->box / (p->h * (1.0 + p->z) * (double)n_pix);
    return orc_hubble(p) * mpc;
}

/* Mean total hydrogen number density, proper, cm^-3 (Eq. 4's nbar_H). */
double orc_mean_nh(const orc_params* p)
{
    double h0_s = 100.0 * p->h * ORC_KMS_CMS / ORC_MPC_CM;           /* s^-1 */
    double rho_crit0 = 3.0 * h0_s * h0_s / (8.0 * ORC_PI * ORC_G_CGS); /* g cm^-3 */
    double a3 = (1.0 + p->z) * (1.0 + p->z) * (1.0 + p->z);
    return (1.0 - p->y_he) * p->omega_b * rho_crit0 * a3 / ORC_MH;
}

/* Eq. 5 with the pivot of Sec. 2.3; rho = 1 + delta. */
double orc_temperature(const orc_params* p, double rho, double t_given)
{
    if (p->t_mode == 0) return t_given;
    double r = rho < p->delta_pivot ? rho : p->delta_pivot;
    return p->T0 * pow(r, p->gamma - 1.0);
}

/* Doppler parameter b = sqrt(2 k_B T / m_H), returned in km/s (Sec. 2.3). */
double orc_doppler_b(double T)
{
    return sqrt(2.0 * ORC_KB * T / ORC_MH) / ORC_KMS_CMS;
}

/* Eq. 4: proper neutral hydrogen density, cm^-3. */
double orc_nhi(const orc_params* p, double rho, double T)
{
    if (rho == 0.0) return 0.0;
    double zf = (1.0 + p->z) / 4.0;
    return 7.24e-6 * orc_mean_nh(p) * pow(T / 1.0e4, -0.7)
         * (p->omega_b * p->h * p->h / 0.024) / p->gamma12
         * rho * rho * zf * zf * zf;
}

/* Nearest periodic image of x in [-V/2, V/2). */
static double nearest_image(double x, double V)
{
    return x - V * floor((x + 0.5 * V) / V);
}

/*
 * Eq. 6 for one skewer: tau[i] for i in [0, N), the plain untruncated sum.
 * rho = 1 + delta, vpec in km/s, temp in K (ignored in power-law mode).
 */
static void tau_one_skewer(const orc_params* p, int64_t N, const float* rho,
                           const float* vpec, const float* temp, double* tau,
                           double* nhi, double* b)
{
    double du = orc_pixel_velocity(p, N);
    double V = du * (double)N;
    double dR = orc_pixel_proper_cm(p, N);
    double pref = ORC_C_CMS * ORC_SIGMA_A * dR / sqrt(ORC_PI);

    for (int64_t j = 0; j < N; ++j) {
        double r = (double)rho[j];
        double T = orc_temperature(p, r, temp ? (double)temp[j] : 0.0);
        nhi[j] = orc_nhi(p, r, T);
        b[j] = nhi[j] > 0.0 ? orc_doppler_b(T) : 1.0;
    }
    for (int64_t i = 0; i < N; ++i) {
        double vh_i = (double)i * du;
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (nhi[j] == 0.0) continue;
            double u_j = (double)j * du + (double)vpec[j];
            double d = nearest_image(vh_i - u_j, V);
            double x = d / b[j];
            double shape;
            if (p->profile == 0) {
                shape = exp(-x * x);
            } else {
                /* (1/du) int_{d-du/2}^{d+du/2} exp(-(y/b)^2) dy
                 *   = (sqrt(pi) b / 2du) [erf((d+du/2)/b) - erf((d-du/2)/b)],
                 * as a difference of erfc of |d| so the far wings do not cancel */
                double ax = fabs(x), hw = 0.5 * du / b[j];
                shape = sqrt(ORC_PI) * b[j] / (2.0 * du) * (erfc(ax - hw) - erfc(ax + hw));
            }
            /* n_HI/b with b in cm/s, as Eq. 6 is written in cgs */
            acc += nhi[j] / (b[j] * ORC_KMS_CMS) * shape;
        }
        tau[i] = pref * acc;
    }
}

/*
 * tau for S skewers of N pixels, row-major [S][N].  temp may be NULL in
 * power-law mode.  Returns 0 on success, -1 on bad arguments or memory.
 */
int orc_tau(const orc_params* p, int64_t S, int64_t N, const float* rho,
            const float* vpec, const float* temp, double* tau)
{
    if (!p || S < 0 || N < 2 || !rho || !vpec || !tau) return -1;
    if (p->t_mode == 0 && !temp) return -1;
    int bad = 0;
#pragma omp parallel reduction(|:bad)
    {
        double* nhi = (double*)malloc((size_t)N * sizeof(double));
        double* b = (double*)malloc((size_t)N * sizeof(double));
        if (!nhi || !b) bad = 1;
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < S; ++s) {
            if (!nhi || !b) continue;
            tau_one_skewer(p, N, rho + s * N, vpec + s * N,
                           temp ? temp + s * N : NULL, tau + s * N, nhi, b);
        }
        free(nhi);
        free(b);
    }
    return bad ? -1 : 0;
}

/* Neumaier compensated accumulator. */
typedef struct { double s, c; } orc_sum;
static void sum_add(orc_sum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double sum_get(const orc_sum* a) { return a->s + a->c; }

/* g(A) = <exp(-A tau)> - F_t and g'(A) = -<tau exp(-A tau)>. */
static void mean_flux_g(const double* tau, int64_t n, double A, double Ft,
                        double* g, double* gp)
{
    orc_sum s0 = {0, 0}, s1 = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double e = exp(-A * tau[i]);
        sum_add(&s0, e);
        sum_add(&s1, tau[i] * e);
    }
    *g = sum_get(&s0) / (double)n - Ft;
    *gp = -sum_get(&s1) / (double)n;
}

/*
 * Mean-flux rescaling (Sec. 2.3): find A with <exp(-A tau)> = Ft over all n
 * optical depths.  Newton from A0 = -ln(Ft)/<tau>; by Jensen g(A0) >= 0 and
 * g is convex and decreasing, so the iterates rise monotonically to the root.
 * A bisection step replaces any Newton step that is non-finite or leaves the
 * bracket.  Stops when |g| <= tol.
 * Returns 0 on success, -1 on bad arguments, -4 on non-convergence.
 */
int orc_rescale(const double* tau, int64_t n, double Ft, double tol,
                int max_iter, double* A_out, int* iters_out)
{
    if (!tau || n <= 0 || !(Ft > 0.0 && Ft < 1.0) || !A_out) return -1;
    orc_sum st = {0, 0};
    int64_t n_zero = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(tau[i] >= 0.0) || !isfinite(tau[i])) return -1;
        sum_add(&st, tau[i]);
        if (tau[i] == 0.0) ++n_zero;
    }
    double mean_tau = sum_get(&st) / (double)n;
    if (!(mean_tau > 0.0)) return -1;
    /* <exp(-A tau)> can never fall below the fraction of zero-tau pixels */
    if ((double)n_zero / (double)n >= Ft) return -4;

    double A = -log(Ft) / mean_tau;
    double lo = A, hi = INFINITY;
    for (int it = 0; it < max_iter; ++it) {
        double g, gp;
        mean_flux_g(tau, n, A, Ft, &g, &gp);
        if (iters_out) *iters_out = it + 1;
        if (fabs(g) <= tol) { *A_out = A; return 0; }
        if (g > 0) lo = A; else hi = A;
        double An = (gp < 0.0) ? A - g / gp : NAN;
        if (!isfinite(An) || An <= lo || An >= hi) {
            An = isfinite(hi) ? 0.5 * (lo + hi) : 2.0 * lo;
        }
        A = An;
    }
    *A_out = A;
    return -4;
}

/* F = exp(-A tau) (Sec. 2.3). */
void orc_flux(const double* tau, int64_t n, double A, double* F)
{
    for (int64_t i = 0; i < n; ++i) F[i] = exp(-A * tau[i]);
}

/*
 * Flux-PDF bin of one flux value (Sec. 5.2): bin k holds
 * (2k-1)/40 <= F < (2k+1)/40, clamped to [0, 20].  For an FP32 value F the
 * product 40F is exact in FP64 (24 + 3 significant bits), so the decision
 * floor((40F + 1)/2) is exact.
 */
int orc_pdf_bin(double F)
{
    double k = floor((40.0 * F + 1.0) / 2.0);
    if (!(k >= 0.0)) return 0;   /* also catches NaN */
    if (k > 20.0) return 20;
    return (int)k;
}

/*
 * Flux statistics over n FP32 flux values: mean, population variance,
 * tau_eff = -ln <F> (Sec. 2.3) and the 21-bin PDF counts (Sec. 5.2).
 */
int orc_flux_stats_f32(const float* F, int64_t n, double* mean, double* var,
                       double* tau_eff, int64_t* pdf)
{
    if (!F || n <= 0) return -1;
    orc_sum s = {0, 0};
    for (int k = 0; k < 21; ++k) pdf[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        sum_add(&s, (double)F[i]);
        pdf[orc_pdf_bin((double)F[i])] += 1;
    }
    double m = sum_get(&s) / (double)n;
    orc_sum v = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double d = (double)F[i] - m;
        sum_add(&v, d * d);
    }
    *mean = m;
    *var = sum_get(&v) / (double)n;
    *tau_eff = -log(m);
    return 0;
}

/* The same statistics over FP64 flux values (the oracle's own F). */
int orc_flux_stats_f64(const double* F, int64_t n, double* mean, double* var,
                       double* tau_eff, int64_t* pdf)
{
    if (!F || n <= 0) return -1;
    orc_sum s = {0, 0};
    for (int k = 0; k < 21; ++k) pdf[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        sum_add(&s, F[i]);
        pdf[orc_pdf_bin(F[i])] += 1;
    }
    double m = sum_get(&s) / (double)n;
    orc_sum v = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double d = F[i] - m;
        sum_add(&v, d * d);
    }
    *mean = m;
    *var = sum_get(&v) / (double)n;
    *tau_eff = -log(m);
    return 0;
}

/* Number of OpenMP threads the oracle will use (for reporting). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
