// lya_api.cu -- the C ABI of liblya.so (declared in include/lya.h).
//
// Host side of the library: argument validation, field ownership, the FP64
// physical constants of Eq. 4-6, and the launches.  Every step of the
// computation runs in the CUDA kernels of tau_extract.cu and mean_flux.cu.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "lya.h"
#include "lya_internal.h"

namespace {

// ---- physical constants (cgs) and the paper's values -------------------------
constexpr double kC = 2.99792458e10;          // speed of light, cm/s
constexpr double kSigmaA = 4.48e-18;          // Ly-alpha cross-section, cm^2 (Sec. 2.3)
constexpr double kBoltz = 1.380649e-16;       // erg/K
constexpr double kMH = 1.6735575e-24;         // hydrogen atom mass, g
constexpr double kMpc = 3.0856775814913673e24;// cm
constexpr double kGrav = 6.67430e-8;          // cm^3 g^-1 s^-2
constexpr double kPi = 3.14159265358979323846;
constexpr double kLog2e = 1.4426950408889634;

struct Physics {
    double du;      // pixel velocity width, km/s
    double K;       // tau_i = K sum_j w_j 2^-(c_j d_ij)^2 with w_j = rho^2 (T/1e4)^-1.2
    double b1e4;    // Doppler parameter at 1e4 K, km/s
};

// Eq. 4 and Eq. 6 with the cosmology of the field, in FP64.
Physics physics(const lya_field_desc& d, double gamma12)
{
    Physics p;
    const double zp = 1.0 + d.z;
    const double hz = 100.0 * d.h * std::sqrt(d.omega_m * zp * zp * zp + d.omega_l);  // km/s/Mpc
    const double dR_mpc = d.box / (d.h * zp * (double)d.n_pix);                      // proper Mpc
    p.du = hz * dR_mpc;
    const double dR_cm = dR_mpc * kMpc;
    const double h0 = 100.0 * d.h * 1.0e5 / kMpc;                                    // s^-1
    const double rho_crit = 3.0 * h0 * h0 / (8.0 * kPi * kGrav);
    const double nbar_h = (1.0 - d.y_he) * d.omega_b * rho_crit * zp * zp * zp / kMH;
    const double q = zp / 4.0;
    // n_HI(T, rho) = n_coef (T/1e4)^-0.7 rho^2     (Eq. 4)
    const double n_coef = 7.24e-6 * nbar_h * (d.omega_b * d.h * d.h / 0.024) / gamma12 * q * q * q;
    p.b1e4 = std::sqrt(2.0 * kBoltz * 1.0e4 / kMH) / 1.0e5;                           // km/s
    // Eq. 6: (c sigma dR / sqrt(pi)) n_HI / b_cgs, with b = b1e4 (T/1e4)^0.5
    p.K = kC * kSigmaA * dR_cm / std::sqrt(kPi) * n_coef / (p.b1e4 * 1.0e5);
    return p;
}

bool desc_ok(const lya_field_desc* d)
{
    if (!d) return false;
    if (!(d->box > 0.0) || !std::isfinite(d->box)) return false;
    if (!(d->z > -1.0) || !std::isfinite(d->z)) return false;
    if (!(d->h > 0.0) || !(d->omega_m >= 0.0) || !(d->omega_l >= 0.0) || !(d->omega_b > 0.0)) return false;
    if (!(d->omega_m * (1.0 + d->z) * (1.0 + d->z) * (1.0 + d->z) + d->omega_l > 0.0)) return false;
    if (!(d->y_he >= 0.0 && d->y_he < 1.0)) return false;
    if (d->n_skewers < 1 || d->n_pix < 16 || d->n_pix > 8192 || (d->n_pix & 1)) return false;
    if (d->has_temp != 0 && d->has_temp != 1) return false;
    return true;
}

lya_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return LYA_OK;
    if (e == cudaErrorMemoryAllocation) return LYA_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver || e == cudaErrorNoKernelImageForDevice)
        return LYA_EDEVICE;
    return LYA_ECUDA;
}

}  // namespace

namespace lya {
static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace lya


namespace {

// The finished check's totals read back on s (after everything before it on
// s), and the field's extents recorded for the window bound.
lya_status record_check(lya_field f, cudaStream_t s)
{
    lya::FieldCheck h{};
    cudaError_t e = cudaMemcpyAsync(&h, f->d_check, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    if (h.bad_rho || h.bad_vpec || h.bad_temp) return LYA_EINVAL;
    std::memcpy(&f->temp_max, &h.temp_max_bits, sizeof(float));
    std::memcpy(&f->rho_max, &h.rho_max_bits, sizeof(float));
    std::memcpy(&f->rho_minpos, &h.rho_minpos_bits, sizeof(float));
    return LYA_OK;
}

// The whole field checked at once.  The host first waits for the work
// already on s (the copies in), so the check kernel is never queued behind
// a copy: a kernel parked behind a long copy can hold up other streams'
// kernels queued after it on the same hardware queue.
lya_status check_and_record(lya_field f, cudaStream_t s)
{
    const int64_t n = f->desc.n_skewers * f->desc.n_pix;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = lya::launch_field_check(f->rho, f->vpec, f->temp, n, f->d_check, s);
    if (e != cudaSuccess) return from_cuda(e);
    return record_check(f, s);
}

lya_status copy_in(lya_field f, const float* rho, const float* vpec, const float* temp, int src,
                   cudaStream_t s)
{
    const size_t bytes = sizeof(float) * (size_t)(f->desc.n_skewers * f->desc.n_pix);
    const cudaMemcpyKind kind = src == LYA_SRC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaMemcpyAsync(f->rho, rho, bytes, kind, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f->vpec, vpec, bytes, kind, s);
    if (e == cudaSuccess && f->temp) e = cudaMemcpyAsync(f->temp, temp, bytes, kind, s);
    return from_cuda(e);
}

// Copies a host field in and validates it.  The copies go in kLoadPieces
// pieces of whole skewers on s, all enqueued at once; the host waits for
// each piece's event and then launches that piece's check on the field's
// check stream, so every check runs while later pieces are still crossing
// the link (the link idles only for the last piece's check), and no check
// kernel ever waits in a queue for a copy (see check_and_record).  Device
// sources (fast copies) take one copy per array and one check.
constexpr int kLoadPieces = 8;

lya_status load_checked(lya_field f, const float* rho, const float* vpec, const float* temp, int src,
                        cudaStream_t s)
{
    const int64_t R = f->desc.n_skewers, N = f->desc.n_pix;
    if (src != LYA_SRC_HOST || R < kLoadPieces) {
        const lya_status st = copy_in(f, rho, vpec, temp, src, s);
        return st != LYA_OK ? st : check_and_record(f, s);
    }
    cudaError_t e = cudaSuccess;
    if (!f->check_stream) {
        e = cudaStreamCreateWithFlags(&f->check_stream, cudaStreamNonBlocking);
        for (int k = 0; e == cudaSuccess && k < kLoadPieces; ++k)
            e = cudaEventCreateWithFlags(&f->piece_ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return from_cuda(e);
    }
    cudaStream_t c = f->check_stream;
    e = lya::launch_field_check_init(f->d_check, c);
    int64_t off[kLoadPieces], cnt[kLoadPieces];
    for (int k = 0; e == cudaSuccess && k < kLoadPieces; ++k) {
        const int64_t r0 = R * k / kLoadPieces, r1 = R * (k + 1) / kLoadPieces;
        off[k] = r0 * N;
        cnt[k] = (r1 - r0) * N;
        const size_t bytes = sizeof(float) * (size_t)cnt[k];
        e = cudaMemcpyAsync(f->rho + off[k], rho + off[k], bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f->vpec + off[k], vpec + off[k], bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && f->temp)
            e = cudaMemcpyAsync(f->temp + off[k], temp + off[k], bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(f->piece_ev[k], s);
    }
    for (int k = 0; e == cudaSuccess && k < kLoadPieces; ++k) {
        e = cudaEventSynchronize(f->piece_ev[k]);          // piece k is on the device
        if (e == cudaSuccess)
            e = lya::launch_field_check_range(f->rho + off[k], f->vpec + off[k],
                                              f->temp ? f->temp + off[k] : nullptr, cnt[k], f->d_check, c);
    }
    if (e != cudaSuccess) {
        (void)cudaStreamSynchronize(s);
        (void)cudaStreamSynchronize(c);
        return from_cuda(e);
    }
    return record_check(f, c);       // every copy on s has landed (each piece's event was waited for)
}

void release(lya_field f)
{
    if (!f) return;
    if (f->check_stream) {
        cudaStreamSynchronize(f->check_stream);
        for (cudaEvent_t ev : f->piece_ev)
            if (ev) cudaEventDestroy(ev);
        cudaStreamDestroy(f->check_stream);
    }
    if (f->owned) {
        cudaFree(f->rho);
        cudaFree(f->vpec);
        cudaFree(f->temp);
    }
    cudaFree(f->d_err);
    cudaFree(f->d_check);
    delete f;
}

}  // namespace

namespace lya {

// Validates the extraction parameters against the field and fills every
// field- and parameter-dependent member of *out (ids, n_rows and tau_out are
// left for the caller): the FP64 constants of Eq. 4-6 in both precisions and
// the window bound w_max from the largest temperature any source can have.
lya_status make_tau_launch(lya_field f, const lya_extract_params* p, TauLaunch* out)
{
    if (!f || !p || !out) return LYA_EINVAL;
    if (p->t_mode != 0 && p->t_mode != 1) return LYA_EINVAL;
    if (p->t_mode == 0 && !f->temp) return LYA_EINVAL;
    if (p->t_mode == 1) {
        if (!(p->T0 > 0.0) || !std::isfinite(p->T0) || !std::isfinite(p->gamma)) return LYA_EINVAL;
        if (!(p->delta_pivot > 0.0)) return LYA_EINVAL;
    }
    if (!(p->gamma12 > 0.0) || !std::isfinite(p->gamma12)) return LYA_EINVAL;
    if (!(p->nsigma >= 1.0 && p->nsigma <= 40.0)) return LYA_EINVAL;
    if (p->precision < LYA_PREC_F32_COMPENSATED || p->precision > LYA_PREC_F64) return LYA_EINVAL;
    if (p->profile != LYA_PROFILE_SAMPLED && p->profile != LYA_PROFILE_AVERAGED) return LYA_EINVAL;
    if (p->profile == LYA_PROFILE_AVERAGED && p->precision == LYA_PREC_F64) return LYA_EINVAL;
    if (p->exp_method < LYA_EXP_MUFU || p->exp_method > LYA_EXP_POLY_SPLIT) return LYA_EINVAL;
    if (p->exp_method != LYA_EXP_MUFU && (p->precision == LYA_PREC_F64 || p->profile != LYA_PROFILE_SAMPLED))
        return LYA_EINVAL;
    const int N = (int)f->desc.n_pix;
    const Physics ph = physics(f->desc, p->gamma12);
    // |v_pec| < c is checked per value; keep |v_pec|/du below 2^22 pixels so the
    // kernels round v/du to whole pixels exactly with the 1.5 * 2^23 shifter
    // (pixels narrower than 0.0715 km/s are refused)
    if (!(ph.du > 2.99792458e5 / 4194304.0)) return LYA_EINVAL;

    // Largest temperature any source can have -> bound on the window half-width
    // (pixels) of every line: nsigma b(T_max)/du + 1/2 (the residual), +1 margin.
    double t_max;
    if (p->t_mode == 0) {
        t_max = f->temp_max;
    } else {
        const double piv = p->delta_pivot;
        const double r_hi = std::fmin((double)f->rho_max, piv);
        const double r_lo = std::fmin((double)f->rho_minpos, piv);
        const double g1 = p->gamma - 1.0;
        t_max = p->T0 * std::fmax(r_hi > 0 ? std::pow(r_hi, g1) : 0.0, r_lo > 0 ? std::pow(r_lo, g1) : 0.0);
    }
    const double b_max = ph.b1e4 * std::sqrt(std::fmax(t_max, 0.0) * 1e-4);
    double w = std::floor(p->nsigma * b_max / ph.du + 0.5) + 1.0;
    if (p->profile == LYA_PROFILE_AVERAGED) w += 1.0;   // the cell average reaches half a pixel further
    if (!(w >= 1.0)) w = 1.0;
    const int w_cap = (N - 1) / 2;
    const int w_max = w > (double)w_cap ? w_cap : (int)w;

    lya::TauLaunch& L = *out;
    L = lya::TauLaunch{};
    L.rho = f->rho;
    L.vpec = f->vpec;
    L.temp = p->t_mode == 0 ? f->temp : nullptr;
    L.n_skewers = f->desc.n_skewers;
    L.n_pix = N;
    L.err = f->d_err;
    L.w_max = w_max;
    L.t_mode = p->t_mode;
    L.profile = p->profile;
    L.exp_method = p->exp_method;
    L.du_hi = (float)ph.du;
    L.du_lo = (float)(ph.du - (double)L.du_hi);
    L.inv_du = (float)(1.0 / ph.du);
    L.c_coef = (float)(std::sqrt(kLog2e) / ph.b1e4);
    L.h_coef = (float)(p->nsigma * std::sqrt(kLog2e));
    L.K = (float)ph.K;
    L.T0 = (float)p->T0;
    L.gm1 = (float)(p->gamma - 1.0);
    L.pivot = std::isfinite(p->delta_pivot) ? (float)p->delta_pivot : INFINITY;
    L.lT0 = (float)std::log2(p->T0 * 1e-4);
    L.lpivot = std::isfinite(p->delta_pivot) ? (float)std::log2(p->delta_pivot) : INFINITY;
    L.lK = (float)std::log2(ph.K);
    L.du_d = ph.du;
    L.inv_du_d = 1.0 / ph.du;
    L.c_coef_d = std::sqrt(kLog2e) / ph.b1e4;
    L.h_coef_d = p->nsigma * std::sqrt(kLog2e);
    L.K_d = ph.K;
    L.T0_d = p->T0;
    L.gm1_d = p->gamma - 1.0;
    L.pivot_d = p->delta_pivot;
    return LYA_OK;
}

}  // namespace lya

extern "C" {

const char* lya_strerror(lya_status s)
{
    switch (s) {
    case LYA_OK: return "success";
    case LYA_EINVAL: return "invalid argument or out-of-domain field value";
    case LYA_ENOMEM: return "out of device memory";
    case LYA_ECUDA: return "CUDA runtime error";
    case LYA_ENOCONV: return "mean-flux root-find did not converge (or no root exists)";
    case LYA_ETIMEDOUT: return "bounded device wait timed out";
    case LYA_EBUDGET: return "request exceeds the memory budget";
    case LYA_EDEVICE: return "no usable sm_103 CUDA device";
    case LYA_EBUSY: return "object in use (a server holds requests on the field, or the server is busy)";
    }
    return "unknown status";
}

const char* lya_version(void) { return "lya 0.1 (sm_103a)"; }

uint64_t lya_kernel_launches(void) { return lya::launches_so_far(); }

lya_status lya_scratch_high_watermark(int reset, uint64_t* bytes)
{
    if (!bytes && !reset) return LYA_EINVAL;
    cudaMemPool_t pool = lya::scratch_pool();
    if (!pool) return LYA_ECUDA;
    if (bytes) {
        unsigned long long v = 0;
        const cudaError_t e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v);
        if (e != cudaSuccess) return from_cuda(e);
        *bytes = (uint64_t)v;
    }
    if (reset) {
        unsigned long long zero = 0;
        return from_cuda(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    return LYA_OK;
}

lya_status lya_create_field(const lya_field_desc* desc, const float* rho, const float* vpec,
                            const float* temp, int src, void* stream, lya_field* out)
{
    if (!out) return LYA_EINVAL;
    *out = nullptr;
    if (!desc_ok(desc) || !rho || !vpec) return LYA_EINVAL;
    if ((desc->has_temp != 0) != (temp != nullptr)) return LYA_EINVAL;
    if (src != LYA_SRC_HOST && src != LYA_SRC_DEVICE_COPY && src != LYA_SRC_DEVICE_BORROW) return LYA_EINVAL;
    if (desc->n_skewers > INT64_MAX / desc->n_pix) return LYA_EINVAL;
    // a borrowed array is read with 16-byte vector loads and bulk copies
    if (src == LYA_SRC_DEVICE_BORROW &&
        ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(vpec) | reinterpret_cast<uintptr_t>(temp)) &
         15) != 0)
        return LYA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lya_field f = new (std::nothrow) lya_field_s();
    if (!f) return LYA_ENOMEM;
    f->desc = *desc;
    cudaGetDevice(&f->device);
    const size_t bytes = sizeof(float) * (size_t)(desc->n_skewers * desc->n_pix);
    cudaError_t e = cudaMalloc((void**)&f->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(f->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&f->d_check, sizeof(lya::FieldCheck));
    if (e != cudaSuccess) { release(f); return from_cuda(e); }
    if (src == LYA_SRC_DEVICE_BORROW) {
        f->owned = false;
        f->rho = const_cast<float*>(rho);
        f->vpec = const_cast<float*>(vpec);
        f->temp = const_cast<float*>(temp);
    } else {
        f->owned = true;
        e = cudaMalloc((void**)&f->rho, bytes);
        if (e == cudaSuccess) e = cudaMalloc((void**)&f->vpec, bytes);
        if (e == cudaSuccess && temp) e = cudaMalloc((void**)&f->temp, bytes);
        if (e != cudaSuccess) { release(f); return from_cuda(e); }
    }
    const lya_status st = src == LYA_SRC_DEVICE_BORROW ? check_and_record(f, s)
                                                       : load_checked(f, rho, vpec, temp, src, s);
    if (st != LYA_OK) { release(f); return st; }
    *out = f;
    return LYA_OK;
}

lya_status lya_field_load(lya_field f, const float* rho, const float* vpec, const float* temp, int src,
                          void* stream)
{
    if (!f || !rho || !vpec || !f->owned) return LYA_EINVAL;
    if ((f->temp != nullptr) != (temp != nullptr)) return LYA_EINVAL;
    if (src != LYA_SRC_HOST && src != LYA_SRC_DEVICE_COPY) return LYA_EINVAL;
    return load_checked(f, rho, vpec, temp, src, static_cast<cudaStream_t>(stream));
}

lya_status lya_destroy_field(lya_field f)
{
    if (!f) return LYA_EINVAL;
    if (f->users.load() != 0) return LYA_EBUSY;      // a server still holds requests on it
    cudaError_t e = cudaDeviceSynchronize();
    release(f);
    return from_cuda(e);
}

lya_status lya_field_shape(lya_field f, int64_t* n_skewers, int64_t* n_pix)
{
    if (!f) return LYA_EINVAL;
    if (n_skewers) *n_skewers = f->desc.n_skewers;
    if (n_pix) *n_pix = f->desc.n_pix;
    return LYA_OK;
}

lya_status lya_field_status(lya_field f, void* stream)
{
    if (!f) return LYA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    return h ? LYA_EINVAL : LYA_OK;
}

lya_status lya_extract_skewers(lya_field f, const lya_extract_params* p, const int64_t* ids, int64_t n_ids,
                               float* tau_out, void* stream)
{
    if (!f || !p) return LYA_EINVAL;
    if (n_ids < 0 || (n_ids > 0 && !tau_out)) return LYA_EINVAL;
    if (!ids && n_ids != 0 && n_ids != f->desc.n_skewers) return LYA_EINVAL;
    if (n_ids > 0x7fffffffLL) return LYA_EINVAL;
    lya::TauLaunch L;
    const lya_status st = lya::make_tau_launch(f, p, &L);
    if (st != LYA_OK) return st;
    if (lya::tau_smem_bytes(L.n_pix, L.w_max, p->precision) > lya::max_dynamic_smem()) return LYA_EINVAL;
    L.ids = ids;
    L.n_rows = n_ids;
    L.tau_out = tau_out;
    return from_cuda(lya::launch_tau(L, p->precision, static_cast<cudaStream_t>(stream)));
}

lya_status lya_rescale_mean_flux(const float* tau, int64_t n, double target, double tol, int max_iter,
                                 double* A_out, float* flux_out, void* stream)
{
    if (!tau || n <= 0 || !A_out) return LYA_EINVAL;
    if (!(target > 0.0 && target < 1.0)) return LYA_EINVAL;
    if (!(tol > 0.0) || max_iter < 1) return LYA_EINVAL;
    return lya::mean_flux_solve(tau, n, target, tol, max_iter, A_out, flux_out,
                                static_cast<cudaStream_t>(stream));
}

lya_status lya_rescale_mean_flux_stats(const float* tau, int64_t n, double target, double tol, int max_iter,
                                       double* A_out, float* flux_out, lya_flux_stats_t* stats_out, void* stream)
{
    if (!tau || n <= 0 || !A_out || !stats_out) return LYA_EINVAL;
    if (!(target > 0.0 && target < 1.0)) return LYA_EINVAL;
    if (!(tol > 0.0) || max_iter < 1) return LYA_EINVAL;
    return lya::mean_flux_solve(tau, n, target, tol, max_iter, A_out, flux_out,
                                static_cast<cudaStream_t>(stream), stats_out);
}

lya_status lya_rescale_mean_flux_noalloc(const float* tau, int64_t n, double target, double tol,
                                         int max_iter, double* A_out, float* flux_out, void* stream)
{
    if (!tau || n <= 0 || !A_out) return LYA_EINVAL;
    if (!(target > 0.0 && target < 1.0)) return LYA_EINVAL;
    if (!(tol > 0.0) || max_iter < 1) return LYA_EINVAL;
    return lya::mean_flux_solve_noalloc(tau, n, target, tol, max_iter, A_out, flux_out,
                                        static_cast<cudaStream_t>(stream));
}

lya_status lya_tau_moments(const float* tau, int64_t n, double out[3], void* stream)
{
    if (!tau || n <= 0 || !out) return LYA_EINVAL;
    return lya::tau_moments_run(tau, n, out, static_cast<cudaStream_t>(stream));
}

lya_status lya_mean_flux_sums(const float* tau, int64_t n, double A, double out[3], void* stream)
{
    if (!tau || n <= 0 || !out || !(A >= 0.0) || !std::isfinite(A)) return LYA_EINVAL;
    return lya::mean_flux_sums_run(tau, n, A, out, static_cast<cudaStream_t>(stream));
}

lya_status lya_flux_at(const float* tau, int64_t n, double A, float* flux_out, void* stream)
{
    if (!tau || n <= 0 || !flux_out || !(A >= 0.0) || !std::isfinite(A)) return LYA_EINVAL;
    return lya::flux_at_run(tau, n, A, flux_out, static_cast<cudaStream_t>(stream));
}

lya_status lya_mean_flux_start(const double totals[4], double target, double tol, int max_iter,
                               lya_mean_flux_iter* it)
{
    if (!totals || !it || !(target > 0.0 && target < 1.0) || !(tol > 0.0) || max_iter < 1) return LYA_EINVAL;
    if (!(totals[3] > 0.0) || !std::isfinite(totals[0]) || !(totals[1] >= 0.0) || !(totals[2] >= 0.0))
        return LYA_EINVAL;
    return lya::mean_flux_start(totals, target, tol, max_iter, it);
}

lya_status lya_mean_flux_step(lya_mean_flux_iter* it, const double sums[3])
{
    if (!it || !sums || !(it->n > 0.0)) return LYA_EINVAL;
    if (!std::isfinite(sums[0]) || !std::isfinite(sums[1]) || !std::isfinite(sums[2])) return LYA_EINVAL;
    return lya::mean_flux_step(it, sums);
}

lya_status lya_rescale_mean_flux_sharded(const float* tau, int64_t n, double target, double tol, int max_iter,
                                         lya_allreduce_fn allreduce, void* user, double* A_out, int* iters_out,
                                         float* flux_out, void* stream)
{
    if (n < 0 || (n > 0 && !tau) || !allreduce || !A_out) return LYA_EINVAL;
    if (!(target > 0.0 && target < 1.0) || !(tol > 0.0) || max_iter < 1) return LYA_EINVAL;
    return lya::mean_flux_sharded(tau, n, target, tol, max_iter, allreduce, user, A_out, iters_out, flux_out,
                                  static_cast<cudaStream_t>(stream));
}

lya_status lya_field_pixel_width(lya_field f, double* du_kms)
{
    if (!f || !du_kms) return LYA_EINVAL;
    *du_kms = physics(f->desc, 1.0).du;
    return LYA_OK;
}

}  // extern "C"

namespace {

struct MockPlan {
    int W, M;
    double du_over_sigma, ratio;
};

lya_status mock_plan(int64_t n_pix, double du, const lya_mock_params* p, MockPlan* out)
{
    if (!p || n_pix < 2 || n_pix > (1 << 24) || !(du > 0.0) || !std::isfinite(du)) return LYA_EINVAL;
    if (!(p->fwhm_kms >= 0.0) || !(p->bin_kms >= 0.0) || !(p->snr >= 0.0) || !(p->max_kms >= 0.0)) return LYA_EINVAL;
    if (!std::isfinite(p->fwhm_kms) || !std::isfinite(p->bin_kms) || !std::isfinite(p->snr) ||
        !std::isfinite(p->max_kms))
        return LYA_EINVAL;
    MockPlan m{};
    if (p->fwhm_kms > 0.0) {
        if (!(p->nsigma > 0.0 && p->nsigma <= 40.0)) return LYA_EINVAL;
        const double sigma = p->fwhm_kms / (2.0 * std::sqrt(2.0 * std::log(2.0)));
        const double w = std::floor(p->nsigma * sigma / du);
        if (2.0 * w + 1.0 > (double)n_pix) return LYA_EINVAL;    // the profile would wrap onto itself
        m.W = (int)w;
        m.du_over_sigma = du / sigma;
    }
    const double B = p->bin_kms > 0.0 ? p->bin_kms : du;
    const double V = (double)n_pix * du;
    const double L = p->max_kms > 0.0 ? std::fmin(V, p->max_kms) : V;
    const double M = std::floor(L / B * (1.0 + 1e-12));
    if (!(M >= 1.0) || M > (double)(1 << 24)) return LYA_EINVAL;
    m.M = (int)M;
    m.ratio = B / du;
    *out = m;
    return LYA_OK;
}

bool two_three_smooth(int64_t n)
{
    if (n < 2) return false;
    while (n % 3 == 0) n /= 3;
    while (n % 2 == 0) n /= 2;
    return n == 1;
}

}  // namespace

extern "C" {

lya_status lya_mock_shape(int64_t n_pix, double du_kms, const lya_mock_params* p, int64_t* n_out)
{
    if (!n_out) return LYA_EINVAL;
    MockPlan m;
    const lya_status st = mock_plan(n_pix, du_kms, p, &m);
    if (st == LYA_OK) *n_out = m.M;
    return st;
}

lya_status lya_mock_spectra(const float* flux, int64_t n_skewers, int64_t n_pix, double du_kms,
                            const lya_mock_params* p, float* out, void* stream)
{
    if (!flux || !out || n_skewers < 1 || n_skewers > 0x7fffffffLL) return LYA_EINVAL;
    MockPlan m;
    const lya_status st = mock_plan(n_pix, du_kms, p, &m);
    if (st != LYA_OK) return st;
    if (lya::mock_smem_bytes((int)n_pix, m.M, m.ratio, m.W) > lya::max_dynamic_smem()) return LYA_EINVAL;
    return lya::mock_spectra_run(flux, n_skewers, (int)n_pix, m.M, m.W, m.du_over_sigma, m.ratio,
                                 p->snr > 0.0 ? 1.0 / p->snr : 0.0, p->seed, p->row0, out,
                                 static_cast<cudaStream_t>(stream));
}

lya_status lya_flux_power_1d(const float* flux, int64_t n_skewers, int64_t n_pix, double du_kms,
                             double* k_out, double* power_out, double* mean_flux_out, void* stream)
{
    if (!flux || !power_out || n_skewers < 1 || !(du_kms > 0.0) || !std::isfinite(du_kms)) return LYA_EINVAL;
    if (!two_three_smooth(n_pix) || n_pix > 65536) return LYA_EINVAL;
    if (lya::flux_ps_smem_bytes((int)n_pix) > lya::max_dynamic_smem()) return LYA_EINVAL;
    const int H = (int)(n_pix / 2 + 1);
    double mean = 0.0;
    const lya_status st = lya::flux_power_run(flux, n_skewers, (int)n_pix, power_out, &mean,
                                              static_cast<cudaStream_t>(stream));
    if (st != LYA_OK) return st;
    if (!(mean > 0.0)) return LYA_EINVAL;                 // no transmitted flux: delta_F undefined
    const double norm = du_kms / (double)n_pix / (double)n_skewers;
    for (int n = 0; n < H; ++n) {
        power_out[n] *= norm;
        if (k_out) k_out[n] = 2.0 * 3.14159265358979323846 * n / ((double)n_pix * du_kms);
    }
    if (mean_flux_out) *mean_flux_out = mean;
    return LYA_OK;
}

lya_status lya_generate_sightlines(const lya_sightline_desc* d, int64_t n_pix, int64_t first_id, int64_t n_ids,
                                   float* rho_out, float* vpec_out, void* stream)
{
    if (!d || n_ids < 0 || n_ids > 0x7fffffffLL || first_id < 0 || (n_ids > 0 && (!rho_out || !vpec_out)))
        return LYA_EINVAL;
    if (n_pix < 4 || (n_pix & 1) || !two_three_smooth(n_pix)) return LYA_EINVAL;
    if (lya::sightline_smem_bytes((int)n_pix) > lya::max_dynamic_smem()) return LYA_EINVAL;
    if (!(d->box > 0.0) || !(d->z > -1.0) || !(d->h > 0.0) || !(d->omega_m >= 0.0) || !(d->omega_l >= 0.0))
        return LYA_EINVAL;
    if (!(d->k_j > 0.0) || !(d->sigma_delta >= 0.0) || !(d->k_f >= 0.0)) return LYA_EINVAL;
    if (!std::isfinite(d->box) || !std::isfinite(d->z) || !std::isfinite(d->k_j) || !std::isfinite(d->sigma_delta) ||
        !std::isfinite(d->k_f))
        return LYA_EINVAL;
    const double zp = 1.0 + d->z;
    const double e2 = d->omega_m * zp * zp * zp + d->omega_l;
    if (!(e2 > 0.0)) return LYA_EINVAL;
    const double aH = 100.0 * std::sqrt(e2) / zp;        // km/s per comoving h^-1 Mpc (h cancels)
    return lya::sightlines_run((int)n_pix, d->box, d->k_j, d->sigma_delta, d->k_f, aH, d->seed, first_id, n_ids,
                               rho_out, vpec_out, static_cast<cudaStream_t>(stream));
}

lya_status lya_flux_power_3d_shells(int64_t n_pix, int n_perp, int64_t* n_shells)
{
    if (!n_shells || n_pix < 2 || n_perp < 2) return LYA_EINVAL;
    *n_shells = lya::flux3d_shells(n_perp, (int)n_pix);
    return LYA_OK;
}

lya_status lya_flux_power_3d(const float* flux, const int32_t* cells, int64_t n_los, int64_t n_pix, int n_perp,
                             double box, double noise_sigma, double* k_mean, double* p_true, double* p_box,
                             double* n_modes, void* stream)
{
    if (!flux || !cells || !p_true || n_los < 1 || n_los > 0x7fffffffLL) return LYA_EINVAL;
    if (!two_three_smooth(n_pix) || n_pix > 65536 || !two_three_smooth(n_perp) || n_perp > 96) return LYA_EINVAL;
    if (!(box > 0.0) || !std::isfinite(box) || !(noise_sigma >= 0.0) || !std::isfinite(noise_sigma)) return LYA_EINVAL;
    for (int64_t i = 0; i < n_los; ++i)
        if (cells[i] < 0 || cells[i] >= n_perp * n_perp) return LYA_EINVAL;
    if (lya::flux3d_los_smem_bytes((int)n_pix) > lya::max_dynamic_smem() ||
        lya::flux3d_plane_smem_bytes(n_perp, (int)n_pix) > lya::max_dynamic_smem())
        return LYA_EINVAL;
    const int ns = lya::flux3d_shells(n_perp, (int)n_pix);
    double* sh = new (std::nothrow) double[4 * (size_t)ns];
    if (!sh) return LYA_ENOMEM;
    const lya_status st = lya::flux_power_3d_run(flux, cells, n_los, (int)n_pix, n_perp, box, noise_sigma, sh, ns,
                                                 static_cast<cudaStream_t>(stream));
    if (st == LYA_OK) {
        const double kf = 2.0 * 3.14159265358979323846 / box;
        for (int b = 0; b < ns; ++b) {
            const double c = sh[4 * b + 3];
            p_true[b] = c > 0.0 ? sh[4 * b] / c : 0.0;
            if (p_box) p_box[b] = c > 0.0 ? sh[4 * b + 1] / c : 0.0;
            if (k_mean) k_mean[b] = c > 0.0 ? kf * sh[4 * b + 2] / c : 0.0;
            if (n_modes) n_modes[b] = c;
        }
    }
    delete[] sh;
    return st;
}

lya_status lya_flux_stats(const float* flux, int64_t n, lya_flux_stats_t* out, void* stream)
{
    if (!flux || n <= 0 || !out) return LYA_EINVAL;
    return lya::flux_stats_run(flux, n, out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
