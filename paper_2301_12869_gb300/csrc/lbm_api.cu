// Host side of liblbm: the C ABI declared in include/lbm.h.
//
// Owns the lattice handle (device buffers, stream, launch plan), validates
// parameters, issues the kernels of lbm_kernels.cu and maps device status to
// error codes. Also carries a host FP64 solver for the Carnahan-Starling
// critical point and coexistence state (Sec. IV, Eqs. EOS and MaxwellRule),
// used to build initial conditions and the interface level of
// LBM_REDUCE_INTERFACE_Y. All arithmetic of the time step runs in the kernels.
#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_ptx.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

namespace {

thread_local char g_err[512] = "";

void set_err(char* buf, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// lattice weights w_i (text after Eq. EquilibriumDistribution), order of Eq. VelocitySet
constexpr double kWeights[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

// ------------------------------------------------------------------ thermodynamics (host, FP64)
// Eq. EOS with eta = b rho / 4: p = rho R T Z(eta) - a rho^2,
// Z = (1 + eta + eta^2 - eta^3)/(1 - eta)^3.
double cs_p(double rho, double T, double a, double b, double R) {
  const double e = b * rho / 4.0;
  return rho * R * T * (1.0 + e + e * e - e * e * e) / ((1.0 - e) * (1.0 - e) * (1.0 - e)) - a * rho * rho;
}
// dp/drho = R T K1(eta) - 2 a rho, K1 = d(eta Z)/d eta = (1 + 4e + 4e^2 - 4e^3 + e^4)/(1 - e)^4
double cs_dp(double rho, double T, double a, double b, double R) {
  const double e = b * rho / 4.0, om = 1.0 - e;
  return R * T * (1.0 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e) / (om * om * om * om) - 2.0 * a * rho;
}
// K2 = d^2(eta Z)/d eta^2 = 4 (2 + 5 e - e^2)/(1 - e)^5; d2p/drho2 = (b/4) R T K2 - 2 a
double cs_K1(double e) { const double om = 1 - e; return (1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e) / (om * om * om * om); }
double cs_K2(double e) { const double om = 1 - e; return 4 * (2 + 5 * e - e * e) / (om * om * om * om * om); }
// chemical potential of the CS free energy: mu = R T [ln rho + (8e - 9e^2 + 3e^3)/(1-e)^3] - 2 a rho
double cs_mu(double rho, double T, double a, double b, double R) {
  const double e = b * rho / 4.0, om = 1.0 - e;
  return R * T * (std::log(rho) + (8 * e - 9 * e * e + 3 * e * e * e) / (om * om * om)) - 2.0 * a * rho;
}

template <class F>
double bisect(F f, double lo, double hi) {
  double flo = f(lo);
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(lo < mid && mid < hi)) break;
    const double fm = f(mid);
    if (fm == 0.0) return mid;
    if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
  }
  return 0.5 * (lo + hi);
}

bool critical(double a, double b, double R, double* rc, double* Tc, double* pc) {
  if (!(a > 0 && b > 0 && R > 0)) return false;
  // dp/drho = 0 and d2p/drho2 = 0  <=>  R T K1 = 8 a e / b and R T K2 = 8 a / b  =>  K1(e) = e K2(e)
  const double e = bisect([](double x) { return cs_K1(x) - x * cs_K2(x); }, 0.01, 0.5);
  *rc = 4.0 * e / b;
  *Tc = 8.0 * a / (b * R * cs_K2(e));
  *pc = cs_p(*rc, *Tc, a, b, R);
  return true;
}

// Coexistence by equal pressure and equal chemical potential (equivalent to the
// equal-area construction of Eqs. MaxwellRule): for trial pressure p on the
// spinodal interval, rho_v / rho_l are the branch roots of p(rho) = p, and
// mu(rho_l) - mu(rho_v) decreases monotonically in p (d/dp = 1/rho_l - 1/rho_v).
bool coexistence(double a, double b, double R, double T, double* rv, double* rl, double* ps) {
  double rc, Tc, pc;
  if (!critical(a, b, R, &rc, &Tc, &pc) || !(T > 0 && T < Tc)) return false;
  const double rmax = 4.0 / b * (1.0 - 1e-12);
  const double s_v = bisect([&](double r) { return cs_dp(r, T, a, b, R); }, 1e-12 * rc, rc);
  const double s_l = bisect([&](double r) { return cs_dp(r, T, a, b, R); }, rc, 0.999 * 4.0 / b);
  const double p_hi = cs_p(s_v, T, a, b, R), p_lo = std::max(cs_p(s_l, T, a, b, R), 0.0);
  auto roots = [&](double p, double* v, double* l) {
    *v = bisect([&](double r) { return cs_p(r, T, a, b, R) - p; }, 1e-300, s_v);
    *l = bisect([&](double r) { return cs_p(r, T, a, b, R) - p; }, s_l, rmax);
  };
  const double p = bisect(
      [&](double pp) {
        double v, l;
        roots(pp, &v, &l);
        return cs_mu(l, T, a, b, R) - cs_mu(v, T, a, b, R);
      },
      p_lo + 1e-14 * p_hi, p_hi * (1.0 - 1e-13));
  roots(p, rv, rl);
  *ps = p;
  return true;
}

}  // namespace

// ------------------------------------------------------------------ handle
struct lbm_handle {
  lbm_params p{};
  int dev = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  bool owns_ws = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  size_t s = 8;          // bytes per real
  size_t N = 0;          // nx * ny
  void* f[2] = {nullptr, nullptr};
  int cur = 0;           // f[cur] holds the state
  double* parts[2] = {nullptr, nullptr};
  int pcur = 0;          // parts[pcur] holds the partials of f[cur]
  int npart = 0;         // partials in parts[pcur]
  int P = 0;             // CTAs of the current step launch (= partials it writes)
  int Pcap = 0;          // partial slots per buffer (largest grid over the tile variants)
  int* status = nullptr;
  double* red = nullptr; // small device outputs
  double* rho_now = nullptr;
  double* rho_prev = nullptr;
  double* ux = nullptr;
  double* uy = nullptr;
  double* rowmean = nullptr;
  void* Tf = nullptr;    // thermal variant: temperature field real[ny][nx]
  void* Tnext = nullptr; // the field after the next energy step (swapped with Tf)
  bool have_prev = false;
  int64_t steps = 0;
  lbm::StepTiling tiling{};
  lbm::StepPhys phys{};
  double rho_mid = NAN;
  char err[512] = "";
};

namespace {

struct Layout {
  size_t f0, f1, parts0, parts1, status, red, rho_now, rho_prev, ux, uy, rowmean, Tf, Tnext, total;
};

int plan_tiling(const lbm_params& p, int nsm, lbm::StepTiling* t, char* err, int variant = 0) {
  const int H = p.precision == LBM_FP32 ? 4 : 2;
  int bw_max = 0;
  if (!lbm::step_variant_info(p.precision, variant, &bw_max, &t->threads, &t->smem_bytes)) {
    set_err(err, "unknown tile variant %d", variant);
    return LBM_EINVAL;
  }
  if ((p.thermal || p.wall == LBM_WALL_ZOU_HE) && !lbm::step_variant_extended(p.precision, variant)) {
    set_err(err, "tile variant %d has no thermal or Zou-He kernels", variant);
    return LBM_EINVAL;
  }
  t->variant = variant;
  t->nx = p.nx;
  t->ny = p.ny;
  t->band_w = std::min(p.nx, bw_max);
  t->nbands = (p.nx + t->band_w - 1) / t->band_w;
  if (t->band_w % H) {
    set_err(err, "internal: band width %d not a multiple of %d", t->band_w, H);
    return LBM_EINVAL;
  }
  int per_sm = 1;
  if (int rc = lbm::step_ctas_per_sm(p.precision, variant, t->threads, t->smem_bytes, &per_sm, err)) return rc;
  // one wave: every CTA resident at once, so neighbouring strips stream their shared
  // halo rows at the same time
  const long target = long(nsm) * per_sm;
  long nstrips = std::max(1L, std::min<long>(p.ny, target / t->nbands));
  t->strip_h = int((p.ny + nstrips - 1) / nstrips);
  t->nstrips = (p.ny + t->strip_h - 1) / t->strip_h;
  t->y_begin = 0;
  t->y_end = p.ny;
  t->ylo = 0;
  t->yhi = p.ny - 1;
  t->n_total = double(p.nx) * double(p.ny);
  return LBM_OK;
}

// Partial slots a handle needs: the largest grid over the tile variants.
int max_partials(const lbm_params& p, int nsm, char* err) {
  int P = 0;
  for (int v = 0; v < lbm::step_num_variants(p.precision); ++v) {
    lbm::StepTiling t;
    if ((p.thermal || p.wall == LBM_WALL_ZOU_HE) && !lbm::step_variant_extended(p.precision, v)) continue;
    if (plan_tiling(p, nsm, &t, err, v)) return -1;
    P = std::max(P, t.nbands * t.nstrips);
  }
  return P;
}

Layout layout_for(const lbm_params& p, int P) {
  const size_t s = p.precision == LBM_FP32 ? 4 : 8;
  const size_t N = size_t(p.nx) * p.ny;
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 256); return at; };
  L.f0 = take(9 * N * s);
  L.f1 = take(9 * N * s);
  L.parts0 = take(size_t(P) * 8);
  L.parts1 = take(size_t(P) * 8);
  L.status = take(sizeof(int));
  L.red = take(8 * sizeof(double));
  L.rho_now = take(N * 8);
  L.rho_prev = take(N * 8);
  L.ux = take(N * 8);
  L.uy = take(N * 8);
  L.rowmean = take(size_t(p.ny) * 8);
  const size_t nT = p.thermal ? N * s : 0;
  L.Tf = take(nT);
  L.Tnext = take(nT);
  L.total = o;
  return L;
}

int validate(const lbm_params* p, char* err) {
  if (!p) { set_err(err, "params is NULL"); return LBM_EINVAL; }
  if (p->size != sizeof(lbm_params)) {
    set_err(err, "params.size is %u, expected %zu (ABI version %d)", p->size, sizeof(lbm_params), LBM_ABI_VERSION);
    return LBM_EINVAL;
  }
  if (p->precision != LBM_FP32 && p->precision != LBM_FP64) { set_err(err, "precision must be LBM_FP32 or LBM_FP64"); return LBM_EINVAL; }
  const int H = p->precision == LBM_FP32 ? 4 : 2;
  if (p->nx <= 0 || p->ny <= 0) { set_err(err, "nx and ny must be positive (got %d x %d)", p->nx, p->ny); return LBM_EINVAL; }
  if (p->nx % H) { set_err(err, "nx = %d must be a multiple of %d for this precision (16-byte rows)", p->nx, H); return LBM_EINVAL; }
  if (double(p->nx) * p->ny > 2.0e9) { set_err(err, "lattice too large (%d x %d)", p->nx, p->ny); return LBM_EINVAL; }
  if (!(p->a >= 0 && p->b > 0 && p->R > 0 && p->T > 0 && std::isfinite(p->a) && std::isfinite(p->T))) {
    set_err(err, "EOS constants must satisfy a >= 0, b > 0, R > 0, T > 0"); return LBM_EINVAL;
  }
  if (!(p->G < 0)) { set_err(err, "G must be negative (psi is real for p_EOS < rho c_s^2)"); return LBM_EINVAL; }
  const double taus[6] = {p->tau_rho, p->tau_e, p->tau_varsigma, p->tau_j, p->tau_q, p->tau_nu};
  for (double t : taus)
    if (!(t > 0.5) || !std::isfinite(t)) { set_err(err, "every relaxation time must be > 1/2"); return LBM_EINVAL; }
  if (!std::isfinite(p->sigma) || !std::isfinite(p->gx) || !std::isfinite(p->gy)) { set_err(err, "sigma and g must be finite"); return LBM_EINVAL; }
  if (p->gravity_form != LBM_GRAVITY_RHO_G && p->gravity_form != LBM_GRAVITY_RHO_MINUS_MEAN_G) {
    set_err(err, "gravity_form must be LBM_GRAVITY_RHO_G or LBM_GRAVITY_RHO_MINUS_MEAN_G"); return LBM_EINVAL;
  }
  if (p->thermal != 0 && p->thermal != 1) { set_err(err, "thermal must be 0 or 1"); return LBM_EINVAL; }
  if (p->wall != LBM_WALL_BOUNCE_BACK && p->wall != LBM_WALL_ZOU_HE) {
    set_err(err, "wall must be LBM_WALL_BOUNCE_BACK or LBM_WALL_ZOU_HE"); return LBM_EINVAL;
  }
  if (p->wall == LBM_WALL_ZOU_HE && p->ny < 3) { set_err(err, "Zou-He walls need ny >= 3"); return LBM_EINVAL; }
  if (p->reserved1 != 0) { set_err(err, "reserved1 must be 0"); return LBM_EINVAL; }
  if (p->thermal && !(p->c_v > 0 && p->kappa >= 0 && p->T_bot > 0 && p->T_top > 0 && std::isfinite(p->c_v) &&
                      std::isfinite(p->kappa) && std::isfinite(p->T_bot) && std::isfinite(p->T_top))) {
    set_err(err, "thermal variant needs c_v > 0, kappa >= 0, T_bot > 0, T_top > 0");
    return LBM_EINVAL;
  }
  return LBM_OK;
}

lbm::StepPhys phys_of(const lbm_params& p, double rho_ref) {
  lbm::StepPhys k{};
  k.rho_ref = rho_ref;
  k.RT = p.R * p.T;
  k.R = p.R;
  k.a = p.a;
  k.b = p.b;
  k.G = p.G;
  k.s_e = 1.0 / p.tau_e;
  k.s_vs = 1.0 / p.tau_varsigma;
  k.s_j = 1.0 / p.tau_j;
  k.s_q = 1.0 / p.tau_q;
  k.s_nu = 1.0 / p.tau_nu;
  k.sig_e = p.sigma / (p.tau_e - 0.5);
  k.sig_vs = p.sigma / (p.tau_varsigma - 0.5);
  k.gx = p.gx;
  k.gy = p.gy;
  k.form = p.gravity_form;
  k.wall = p.wall;
  return k;
}

double midpoint_level(const lbm_params& p) {
  double rv, rl, ps;
  if (coexistence(p.a, p.b, p.R, p.T, &rv, &rl, &ps)) return 0.5 * (rv + rl);
  return NAN;
}

int cuda_fail(lbm_handle* h, cudaError_t e, const char* what) {
  set_err(h ? h->err : g_err, "%s: %s", what, cudaGetErrorString(e));
  return LBM_ECUDA;
}
#define LBM_CUDA(h, call)                                     \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);  \
  } while (0)

int device_status(lbm_handle* h) {
  int st = 0;
  LBM_CUDA(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (st & lbm::STATUS_TIMEOUT) { set_err(h->err, "a device wait timed out"); return LBM_ETIMEOUT; }
  if (st & lbm::STATUS_NONPHYS) {
    set_err(h->err, "non-physical state: rho <= 0, NaN, or 2 (p_EOS - rho/3)/G < 0 somewhere");
    return LBM_ENONPHYS;
  }
  return LBM_OK;
}

// Fresh FP64 partials of the stored state into parts[pcur].
int refresh_partials(lbm_handle* h) {
  LBM_CUDA(h, lbm::launch_partials(h->p.precision, h->f[h->cur], h->p.nx, h->p.ny, h->parts[h->pcur], h->P, h->stream));
  h->npart = h->P;
  return LBM_OK;
}

// A thermal step stores its rho, u for the energy equation in the handle's moment
// scratch (floats for FP32 handles); isothermal steps store none.
void set_thermal_outputs(lbm_handle* h, lbm::StepIO& io) {
  if (!h->p.thermal) return;
  if (h->p.precision == LBM_FP32) {
    io.rho32 = reinterpret_cast<float*>(h->rho_now);
    io.ux32 = reinterpret_cast<float*>(h->ux);
    io.uy32 = reinterpret_cast<float*>(h->uy);
  } else {
    io.rho_out = h->rho_now;
    io.ux_out = h->ux;
    io.uy_out = h->uy;
  }
}

int run_moments(lbm_handle* h, double* rho, double* ux, double* uy) {
  lbm::StepIO io{};
  io.Tfield = h->Tf;
  io.fin = h->f[h->cur];
  io.part_in = h->parts[h->pcur];
  io.npart_in = h->npart;
  io.status = h->status;
  io.rho_out = rho;
  io.ux_out = ux;
  io.uy_out = uy;
  LBM_CUDA(h, lbm::launch_step(h->p.precision, lbm::MODE_MOMENTS, h->tiling, h->phys, io, h->stream));
  return LBM_OK;
}

}  // namespace

// ---- wrappers for the other translation units (lbm_internal.h)
namespace lbm {
namespace {
constexpr int kMaxDevices = 64;
constexpr int kMaxVariants = 16;
}  // namespace

int prepare_step_kernels(int dev, int precision, char* err) {
  static std::atomic<bool> ready[kMaxDevices][2];
  if (dev < 0 || dev >= kMaxDevices) {
    set_err(err, "device index %d beyond the %d this library supports", dev, kMaxDevices);
    return LBM_EINVAL;
  }
  std::atomic<bool>& r = ready[dev][precision == LBM_FP32 ? 1 : 0];
  if (!r.load(std::memory_order_acquire)) {  // two threads may both set it: the same values
    const cudaError_t e = step_prepare(precision);
    if (e != cudaSuccess) {
      set_err(err, "kernel attributes: %s", cudaGetErrorString(e));
      return LBM_ECUDA;
    }
    r.store(true, std::memory_order_release);
  }
  return LBM_OK;
}

int step_ctas_per_sm(int precision, int variant, int threads, int smem_bytes, int* per_sm, char* err) {
  // cache entries hold the count + 1 (0: not asked yet); the threads and shared memory of a
  // variant are fixed, so (device, precision, variant) is the key
  static std::atomic<int> cache[kMaxDevices][2][kMaxVariants];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_err(err, "no CUDA device");
    return LBM_ECUDA;
  }
  if (int rc = prepare_step_kernels(dev, precision, err)) return rc;  // the query depends on the limit
  std::atomic<int>* slot = variant >= 0 && variant < kMaxVariants ? &cache[dev][precision == LBM_FP32 ? 1 : 0][variant]
                                                                   : nullptr;
  int n = slot ? slot->load(std::memory_order_acquire) - 1 : -1;
  if (n < 0) {
    n = std::max(1, step_max_ctas_per_sm(precision, variant, threads, smem_bytes));
    if (slot) slot->store(n + 1, std::memory_order_release);
  }
  *per_sm = n;
  return LBM_OK;
}

int validate_params(const lbm_params* p, char* err) { return validate(p, err); }
StepPhys phys_from_params(const lbm_params& p, double rho_ref) { return phys_of(p, rho_ref); }
int plan_step_tiling(const lbm_params& p, int nsm, StepTiling* t, char* err) { return plan_tiling(p, nsm, t, err); }
void set_last_error(const char* msg) { set_err(g_err, "%s", msg); }
}  // namespace lbm

// ================================================================== public ABI
extern "C" {

void lbm_params_default(lbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->size = sizeof(lbm_params);
  p->precision = LBM_FP64;
  p->a = 0.5;
  p->b = 4.0;
  p->R = 1.0;
  p->G = -1.0;
  p->sigma = 1.385;
  p->tau_rho = p->tau_e = p->tau_varsigma = p->tau_j = p->tau_q = p->tau_nu = 1.0;
  p->gravity_form = LBM_GRAVITY_RHO_G;
  p->rho_ref = NAN;
  p->c_v = 5.0;
  p->kappa = 0.02;
}

int lbm_workspace_bytes(const lbm_params* p, uint64_t* bytes) {
  int rc = validate(p, g_err);
  if (rc) return rc;
  if (!bytes) { set_err(g_err, "bytes is NULL"); return LBM_EINVAL; }
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_err(g_err, "no CUDA device");
    return LBM_ECUDA;
  }
  // the grid plan depends on the occupancy the kernels reach with their shared-memory
  // limit set, as in lbm_init (plan_tiling sets it first)
  lbm::StepTiling t;
  if ((rc = plan_tiling(*p, nsm, &t, g_err))) return rc;
  const int cap = max_partials(*p, nsm, g_err);
  if (cap < 0) return LBM_EINVAL;
  *bytes = layout_for(*p, cap).total;
  return LBM_OK;
}

int lbm_init(const lbm_params* p, const double* rho0, int rho0_where, void* stream, lbm_handle** out) {
  lbm::TraceRange trace("lbm_init");
  int rc = validate(p, g_err);
  if (rc) return rc;
  if (!out || !rho0) { set_err(g_err, "out and rho0 must not be NULL"); return LBM_EINVAL; }
  if (rho0_where != LBM_HOST && rho0_where != LBM_DEVICE) { set_err(g_err, "rho0_where must be LBM_HOST or LBM_DEVICE"); return LBM_EINVAL; }
  *out = nullptr;
  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) { set_err(g_err, "out of host memory"); return LBM_ENOMEM; }
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(stream);
  h->s = p->precision == LBM_FP32 ? 4 : 8;
  h->N = size_t(p->nx) * p->ny;
  auto fail = [&](int code) {
    std::memcpy(g_err, h->err, sizeof(g_err));
    lbm_destroy(h);
    return code;
  };
  if (cudaGetDevice(&h->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev) != cudaSuccess) {
    set_err(h->err, "no CUDA device");
    return fail(LBM_ECUDA);
  }
  if ((rc = lbm::prepare_step_kernels(h->dev, p->precision, h->err))) return fail(rc);
  if ((rc = plan_tiling(*p, h->nsm, &h->tiling, h->err))) return fail(rc);
  cudaError_t e = cudaSuccess;
  h->P = h->tiling.nbands * h->tiling.nstrips;
  h->Pcap = max_partials(*p, h->nsm, h->err);
  if (h->Pcap < 0) return fail(LBM_EINVAL);
  const Layout L = layout_for(*p, h->Pcap);
  if (p->workspace) {
    if (p->workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(p->workspace) & 255)) {
      set_err(h->err, "workspace needs %zu bytes at 256-byte alignment (got %llu)", L.total,
              (unsigned long long)p->workspace_bytes);
      return fail(LBM_ENOMEM);
    }
    h->ws = p->workspace;
  } else {
    e = cudaMalloc(&h->ws, L.total);
    if (e != cudaSuccess) { h->ws = nullptr; cuda_fail(h, e, "cudaMalloc workspace"); return fail(LBM_ENOMEM); }
    h->owns_ws = true;
  }
  h->ws_bytes = L.total;
  char* base = static_cast<char*>(h->ws);
  h->f[0] = base + L.f0;
  h->f[1] = base + L.f1;
  h->parts[0] = reinterpret_cast<double*>(base + L.parts0);
  h->parts[1] = reinterpret_cast<double*>(base + L.parts1);
  h->status = reinterpret_cast<int*>(base + L.status);
  h->red = reinterpret_cast<double*>(base + L.red);
  h->rho_now = reinterpret_cast<double*>(base + L.rho_now);
  h->rho_prev = reinterpret_cast<double*>(base + L.rho_prev);
  h->ux = reinterpret_cast<double*>(base + L.ux);
  h->uy = reinterpret_cast<double*>(base + L.uy);
  h->rowmean = reinterpret_cast<double*>(base + L.rowmean);
  if (p->thermal) {
    h->Tf = base + L.Tf;
    h->Tnext = base + L.Tnext;
  }

  // initial density on the device (staged through the rho_now scratch when on the host)
  const double* rho_dev = rho0;
  if (rho0_where == LBM_HOST) {
    e = cudaMemcpyAsync(h->rho_now, rho0, h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) { cuda_fail(h, e, "copy rho0"); return fail(LBM_ECUDA); }
    rho_dev = h->rho_now;
  }
  double rho_ref = p->rho_ref;
  if (std::isnan(rho_ref) && p->precision == LBM_FP64) rho_ref = 0.0;
  if (std::isnan(rho_ref)) {
    // mean of rho0: FP64 row means on the device, then an FP64 host sum of ny values
    e = lbm::launch_row_means(rho_dev, p->nx, p->ny, h->rowmean, h->stream);
    if (e != cudaSuccess) { cuda_fail(h, e, "row means"); return fail(LBM_ECUDA); }
    double* rm = new (std::nothrow) double[p->ny];
    if (!rm) { set_err(h->err, "out of host memory"); return fail(LBM_ENOMEM); }
    e = cudaMemcpyAsync(rm, h->rowmean, size_t(p->ny) * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    double s = 0.0;
    for (int y = 0; y < p->ny; ++y) s += rm[y];
    delete[] rm;
    if (e != cudaSuccess) { cuda_fail(h, e, "mean of rho0"); return fail(LBM_ECUDA); }
    rho_ref = s / p->ny;
  }
  if (!std::isfinite(rho_ref)) { set_err(h->err, "rho_ref is not finite"); return fail(LBM_EINVAL); }
  h->p.rho_ref = rho_ref;
  h->phys = phys_of(h->p, rho_ref);
  h->rho_mid = midpoint_level(h->p);

  e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  if (e == cudaSuccess)
    e = lbm::launch_init(p->precision, rho_dev, h->f[0], p->nx, p->ny, rho_ref, h->parts[0], h->P, h->stream);
  if (e == cudaSuccess && p->thermal)
    e = lbm::launch_linear_T(p->precision, p->nx, p->ny, p->T_bot, p->T_top, p->wall == LBM_WALL_ZOU_HE ? 1 : 0, h->Tf,
                             h->stream);
  if (e != cudaSuccess) { cuda_fail(h, e, "init kernel"); return fail(LBM_ECUDA); }
  h->cur = 0;
  h->pcur = 0;
  h->npart = h->P;  // the init kernel wrote the partials of the initial state
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) { cuda_fail(h, e, "lbm_init"); return fail(LBM_ECUDA); }
  *out = h;
  return LBM_OK;
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
  lbm::TraceRange trace("lbm_step");
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (nsteps < 0) { set_err(h->err, "nsteps must be >= 0"); return LBM_EINVAL; }
  lbm::StepIO io{};
  io.status = h->status;
  const lbm_params& p = h->p;
  set_thermal_outputs(h, io);
  for (int64_t t = 0; t < nsteps; ++t) {
    io.Tfield = h->Tf;
    io.fin = h->f[h->cur];
    io.fout = h->f[1 - h->cur];
    io.part_in = h->parts[h->pcur];
    io.npart_in = h->npart;
    io.part_out = h->parts[1 - h->pcur];
    LBM_CUDA(h, lbm::launch_step(p.precision, lbm::MODE_STEP, h->tiling, h->phys, io, h->stream));
    h->cur = 1 - h->cur;
    h->pcur = 1 - h->pcur;
    h->npart = h->P;
    ++h->steps;
    if (p.thermal) {
      // T^n -> T^(n+1) with the rho^n, u^n this step formed (force of T^n)
      LBM_CUDA(h, lbm::launch_energy_step(p.precision, p.nx, p.ny, p.wall == LBM_WALL_ZOU_HE ? 1 : 0, p.R, p.b, p.c_v,
                                          p.kappa, p.T_bot, p.T_top, h->rho_now, h->ux, h->uy, h->Tf, h->Tnext,
                                          h->stream));
      std::swap(h->Tf, h->Tnext);
    }
  }
  return LBM_OK;
}

int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy, int where) {
  lbm::TraceRange trace("lbm_moments");
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (where != LBM_HOST && where != LBM_DEVICE) { set_err(h->err, "where must be LBM_HOST or LBM_DEVICE"); return LBM_EINVAL; }
  int rc;
  if (where == LBM_DEVICE) return run_moments(h, rho, ux, uy);
  if ((rc = run_moments(h, rho ? h->rho_now : nullptr, ux ? h->ux : nullptr, uy ? h->uy : nullptr))) return rc;
  const size_t bytes = h->N * sizeof(double);
  if (rho) LBM_CUDA(h, cudaMemcpyAsync(rho, h->rho_now, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (ux) LBM_CUDA(h, cudaMemcpyAsync(ux, h->ux, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (uy) LBM_CUDA(h, cudaMemcpyAsync(uy, h->uy, bytes, cudaMemcpyDeviceToHost, h->stream));
  return device_status(h);
}

int lbm_reduce(lbm_handle* h, int kind, double* out) {
  lbm::TraceRange trace("lbm_reduce");
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (!out) { set_err(h->err, "out is NULL"); return LBM_EINVAL; }
  int rc;
  const int nx = h->p.nx, ny = h->p.ny;
  switch (kind) {
    case LBM_REDUCE_MASS:
    case LBM_REDUCE_MEAN_RHO: {
      double* scratch = h->parts[1 - h->pcur];  // overwritten by the next step anyway
      LBM_CUDA(h, lbm::launch_partials(h->p.precision, h->f[h->cur], nx, ny, scratch, h->P, h->stream));
      LBM_CUDA(h, lbm::launch_sum_partials(scratch, h->P, h->red, h->stream));
      double s = 0.0;
      LBM_CUDA(h, cudaMemcpyAsync(&s, h->red, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      rc = device_status(h);
      const double mass = s + double(h->N) * h->p.rho_ref;
      out[0] = kind == LBM_REDUCE_MASS ? mass : mass / double(h->N);
      return rc;
    }
    case LBM_REDUCE_RESIDUAL: {
      if ((rc = run_moments(h, h->rho_now, nullptr, nullptr))) return rc;
      double r = INFINITY;
      if (h->have_prev) {
        LBM_CUDA(h, lbm::launch_max_abs_diff(h->rho_now, h->rho_prev, h->N, h->red, h->stream));
        LBM_CUDA(h, cudaMemcpyAsync(&r, h->red, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      }
      rc = device_status(h);
      std::swap(h->rho_now, h->rho_prev);
      h->have_prev = true;
      out[0] = r;
      return rc;
    }
    case LBM_REDUCE_MAX_U: {
      if ((rc = run_moments(h, nullptr, h->ux, h->uy))) return rc;
      LBM_CUDA(h, lbm::launch_max_speed(h->ux, h->uy, h->N, h->red, h->stream));
      LBM_CUDA(h, cudaMemcpyAsync(out, h->red, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      return device_status(h);
    }
    case LBM_REDUCE_INTERFACE_Y:
    case LBM_REDUCE_RHO_LV: {
      if ((rc = run_moments(h, h->rho_now, nullptr, nullptr))) return rc;
      LBM_CUDA(h, lbm::launch_row_means(h->rho_now, nx, ny, h->rowmean, h->stream));
      LBM_CUDA(h, lbm::launch_profile_scan(h->rowmean, ny, h->rho_mid, h->red, h->stream));
      double v[3];
      LBM_CUDA(h, cudaMemcpyAsync(v, h->red, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
      rc = device_status(h);
      if (kind == LBM_REDUCE_INTERFACE_Y) {
        out[0] = v[0];
      } else {
        out[0] = v[1];
        out[1] = v[2];
      }
      return rc;
    }
    default:
      set_err(h->err, "unknown reduction kind %d", kind);
      return LBM_EINVAL;
  }
}

int lbm_get_state(lbm_handle* h, double* f, int where, int64_t* steps_done) {
  lbm::TraceRange trace("lbm_get_state");
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (!f || (where != LBM_HOST && where != LBM_DEVICE)) { set_err(h->err, "bad f or where"); return LBM_EINVAL; }
  if (steps_done) *steps_done = h->steps;
  for (int i = 0; i < 9; ++i) {
    const void* plane = static_cast<const char*>(h->f[h->cur]) + size_t(i) * h->N * h->s;
    const double add = kWeights[i] * h->p.rho_ref;
    double* dst = where == LBM_DEVICE ? f + size_t(i) * h->N : h->ux;  // host path stages through ux
    LBM_CUDA(h, lbm::launch_plane_to_double(h->p.precision, plane, dst, h->N, add, h->stream));
    if (where == LBM_HOST)
      LBM_CUDA(h, cudaMemcpyAsync(f + size_t(i) * h->N, h->ux, h->N * sizeof(double), cudaMemcpyDeviceToHost,
                                  h->stream));
  }
  return where == LBM_HOST ? device_status(h) : LBM_OK;
}

int lbm_set_state(lbm_handle* h, const double* f, int where, int64_t steps_done) {
  lbm::TraceRange trace("lbm_set_state");
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (!f || (where != LBM_HOST && where != LBM_DEVICE)) { set_err(h->err, "bad f or where"); return LBM_EINVAL; }
  for (int i = 0; i < 9; ++i) {
    void* plane = static_cast<char*>(h->f[h->cur]) + size_t(i) * h->N * h->s;
    const double sub = kWeights[i] * h->p.rho_ref;
    const double* src = f + size_t(i) * h->N;
    if (where == LBM_HOST) {  // staged through ux, one plane at a time (stream-ordered)
      LBM_CUDA(h, cudaMemcpyAsync(h->ux, src, h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      src = h->ux;
    }
    LBM_CUDA(h, lbm::launch_plane_from_double(h->p.precision, src, plane, h->N, sub, h->stream));
  }
  LBM_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  int rc = refresh_partials(h);
  if (rc) return rc;
  h->have_prev = false;
  h->steps = steps_done;
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_set_temperature(lbm_handle* h, const double* T, int where) {
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (!h->Tf) { set_err(h->err, "the handle is isothermal (thermal = 0)"); return LBM_EINVAL; }
  if (!T || (where != LBM_HOST && where != LBM_DEVICE)) { set_err(h->err, "bad T or where"); return LBM_EINVAL; }
  const double* src = T;
  if (where == LBM_HOST) {  // staged through ux
    LBM_CUDA(h, cudaMemcpyAsync(h->ux, T, h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    src = h->ux;
  }
  LBM_CUDA(h, lbm::launch_plane_from_double(h->p.precision, src, h->Tf, h->N, 0.0, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_get_temperature(lbm_handle* h, double* T, int where) {
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (!h->Tf) { set_err(h->err, "the handle is isothermal (thermal = 0)"); return LBM_EINVAL; }
  if (!T || (where != LBM_HOST && where != LBM_DEVICE)) { set_err(h->err, "bad T or where"); return LBM_EINVAL; }
  double* dst = where == LBM_DEVICE ? T : h->ux;  // host path stages through ux
  LBM_CUDA(h, lbm::launch_plane_to_double(h->p.precision, h->Tf, dst, h->N, 0.0, h->stream));
  if (where == LBM_DEVICE) return LBM_OK;
  LBM_CUDA(h, cudaMemcpyAsync(T, h->ux, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return device_status(h);
}

int lbm_set_params(lbm_handle* h, const lbm_params* p) {
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  int rc = validate(p, h->err);
  if (rc) return rc;
  if (p->nx != h->p.nx || p->ny != h->p.ny || p->precision != h->p.precision || p->a != h->p.a || p->b != h->p.b ||
      p->R != h->p.R || p->thermal != h->p.thermal || p->wall != h->p.wall) {
    set_err(h->err, "nx, ny, precision, a, b, R, thermal and wall cannot change on a live handle");
    return LBM_EINVAL;
  }
  const double rho_ref = h->p.rho_ref;
  void* ws = h->p.workspace;
  const uint64_t wsb = h->p.workspace_bytes;
  h->p = *p;
  h->p.rho_ref = rho_ref;
  h->p.workspace = ws;
  h->p.workspace_bytes = wsb;
  h->phys = phys_of(h->p, rho_ref);
  h->rho_mid = midpoint_level(h->p);
  return LBM_OK;
}

int lbm_status(lbm_handle* h) {
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  return device_status(h);
}

int lbm_destroy(lbm_handle* h) {
  if (!h) return LBM_OK;
  int rc = LBM_OK;
  if (h->owns_ws && h->ws) {
    cudaStreamSynchronize(h->stream);
    if (cudaFree(h->ws) != cudaSuccess) rc = LBM_ECUDA;
  }
  delete h;
  return rc;
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err : g_err; }

int lbm_critical_point(double a, double b, double R, double* rho_c, double* T_c, double* p_c) {
  double rc, Tc, pc;
  if (!critical(a, b, R, &rc, &Tc, &pc)) { set_err(g_err, "need a > 0, b > 0, R > 0"); return LBM_EINVAL; }
  if (rho_c) *rho_c = rc;
  if (T_c) *T_c = Tc;
  if (p_c) *p_c = pc;
  return LBM_OK;
}

int lbm_coexistence(double a, double b, double R, double T, double* rho_v, double* rho_l, double* p_sat) {
  double rv, rl, ps;
  if (!coexistence(a, b, R, T, &rv, &rl, &ps)) { set_err(g_err, "need a, b, R > 0 and 0 < T < T_c"); return LBM_EINVAL; }
  if (rho_v) *rho_v = rv;
  if (rho_l) *rho_l = rl;
  if (p_sat) *p_sat = ps;
  return LBM_OK;
}

int lbm_autotune(lbm_handle* h, int steps, int* variant, double* ms) {
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (steps < 1) { set_err(h->err, "steps must be >= 1"); return LBM_EINVAL; }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LBM_CUDA(h, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(h, ce, "cudaEventCreate"); }
  int best = -1, rc = LBM_OK;
  float best_ms = 0.f;
  lbm::StepTiling best_t{};
  // every candidate reads the current state and writes the other buffer; the state and
  // its partial sums are left as they were
  lbm::StepIO io{};
  io.fin = h->f[h->cur];
  io.fout = h->f[1 - h->cur];
  io.part_in = h->parts[h->pcur];
  io.npart_in = h->npart;
  io.part_out = h->parts[1 - h->pcur];
  io.status = h->status;
  io.Tfield = h->Tf;
  set_thermal_outputs(h, io);
  for (int v = 0; v < lbm::step_num_variants(h->p.precision) && rc == LBM_OK; ++v) {
    lbm::StepTiling t;
    if (plan_tiling(h->p, h->nsm, &t, h->err, v)) continue;
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = lbm::launch_step(h->p.precision, lbm::MODE_STEP, t, h->phys, io, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = lbm::launch_step(h->p.precision, lbm::MODE_STEP, t, h->phys, io, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t_ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
    if (e != cudaSuccess) { rc = cuda_fail(h, e, "autotune"); break; }
    if (best < 0 || t_ms < best_ms) { best = v; best_ms = t_ms; best_t = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (best < 0) { set_err(h->err, "no tile variant fits this lattice"); return LBM_EINVAL; }
  h->tiling = best_t;
  h->P = best_t.nbands * best_t.nstrips;
  if (variant) *variant = best;
  if (ms) *ms = double(best_ms) / steps;
  return LBM_OK;
}

int lbm_tile_variants(int precision) {
  if (precision != LBM_FP32 && precision != LBM_FP64) {
    set_err(g_err, "precision must be LBM_FP32 or LBM_FP64");
    return LBM_EINVAL;
  }
  return lbm::step_num_variants(precision);
}

int lbm_set_tiling(lbm_handle* h, int variant) {
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  lbm::StepTiling t;
  int rc = plan_tiling(h->p, h->nsm, &t, h->err, variant);
  if (rc) return rc;
  h->tiling = t;
  h->P = t.nbands * t.nstrips;
  return LBM_OK;
}

}  // extern "C"

namespace {
// the wait-bound self-check: the bounded wait the library's kernels use, on a barrier that
// expects one arrival and never gets it
__global__ void wait_bound_kernel(long long cycles, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    lbm::mbar_init(&bar, 1);
    lbm::fence_mbar_init();
    if (!lbm::mbar_wait_bounded(&bar, 0u, cycles)) atomicOr(status, lbm::STATUS_TIMEOUT);
  }
}
}  // namespace

extern "C" {

int lbm_wait_bound_selftest(long long cycles) {
  if (cycles < 1 || cycles > 2000000000LL) { set_err(g_err, "cycles must be in [1, 2e9]"); return LBM_EINVAL; }
  int* status = nullptr;
  cudaError_t e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
  if (e == cudaSuccess) {
    wait_bound_kernel<<<1, 32>>>(cycles, status);
    e = cudaGetLastError();
  }
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (status) cudaFree(status);
  if (e != cudaSuccess) { set_err(g_err, "wait-bound self-check: %s", cudaGetErrorString(e)); return LBM_ECUDA; }
  if (st & lbm::STATUS_TIMEOUT) { set_err(g_err, "the bounded wait gave up as intended"); return LBM_ETIMEOUT; }
  set_err(g_err, "the bounded wait did not give up");
  return LBM_OK;
}

int lbm_launch_info(const lbm_handle* h, int* grid, int* block, int* smem_bytes, int* band_width, int* strip_rows,
                    int* stages) {
  if (!h) { set_err(g_err, "handle is NULL"); return LBM_EINVAL; }
  if (grid) *grid = h->tiling.nbands * h->tiling.nstrips;
  if (block) *block = h->tiling.threads;
  if (smem_bytes) *smem_bytes = h->tiling.smem_bytes;
  if (band_width) *band_width = h->tiling.band_w;
  if (strip_rows) *strip_rows = h->tiling.strip_h;
  if (stages) *stages = lbm::stages(h->p.precision, h->tiling.variant);
  return LBM_OK;
}

}  // extern "C"
