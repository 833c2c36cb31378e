// lbm_step_noalloc: one fused time step on caller-owned device populations that
// allocates no device memory (declared in include/lbm.h).
//
// Some callers cannot call cudaMalloc: a host loop that must not stall other
// streams on the implicit device synchronisation an allocation can bring, a
// process whose device memory is reserved up front by another allocator, or a
// plug-in that may not create allocations of its own. lbm_init's handle owns a
// workspace; this entry point instead runs the same kernels with the only
// scratch they need - FP64 partial sums of the mass (for <rho> of
// Eq. Gravity_2) and a status word - in a file-scope __device__ array.
#include "lbm.h"
#include "lbm_internal.h"

#include <cuda_runtime.h>

#include <cstdint>

#include <cmath>
#include <cstdio>
#include <mutex>

namespace {

// Partial-sum slots per buffer; the step's grid must not exceed it.
constexpr int kMaxCtas = 4096;
constexpr int kMaxDevices = 64;

// [0, kMaxCtas): partials of f_in; [kMaxCtas, 2 kMaxCtas): partials the step writes for
// its output; then the status word. 2 * 4096 + 32 doubles = 65 792 bytes per device,
// held by every device that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxCtas + 32];

// Per-device set-up state. A failed set-up is not remembered: the next call on that
// device tries again (under the mutex, so concurrent first calls do it once).
struct DeviceScratch {
  double* ptr = nullptr;  // device address of g_noalloc_scratch on this device; NULL until set up
};
DeviceScratch g_dev[kMaxDevices];
std::mutex g_setup_mutex;

// The scratch array's device address and the step kernels' shared-memory limit, once per
// device with that device current; returns the address or NULL with err set.
double* scratch_on_device(int dev, cudaError_t* err) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceScratch& ds = g_dev[dev];
  *err = cudaSuccess;
  if (ds.ptr) return ds.ptr;
  double* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_scratch);
  if (e == cudaSuccess) e = lbm::step_prepare(LBM_FP32);
  if (e == cudaSuccess) e = lbm::step_prepare(LBM_FP64);
  if (e != cudaSuccess || !ptr) {
    (void)cudaGetLastError();  // not sticky: a later call retries
    *err = e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    return nullptr;
  }
  ds.ptr = ptr;
  return ptr;
}

// true when p is device memory of device dev or managed memory (not host, pinned or
// unregistered memory, nor another device's)
bool is_device_pointer(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

int fail(int code, const char* msg) {
  lbm::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int lbm_step_noalloc(const lbm_params* p, const void* f_in, void* f_out, void* stream) {
  char err[512];
  int rc = lbm::validate_params(p, err);
  if (rc) return fail(rc, err);
  if (p->thermal) return fail(LBM_EINVAL, "lbm_step_noalloc is isothermal (thermal must be 0)");
  if (!f_in || !f_out || f_in == f_out) return fail(LBM_EINVAL, "f_in and f_out must be distinct device arrays");
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(LBM_ECUDA, "no CUDA device");
  if (dev >= kMaxDevices) return fail(LBM_EINVAL, "device index beyond the 64 this entry point supports");

  if (!is_device_pointer(f_in, dev) || !is_device_pointer(f_out, dev))
    return fail(LBM_EINVAL, "f_in and f_out must be device memory of the current device");
  // the step's bulk copies and vector loads start on 16-byte boundaries of the planes
  if ((reinterpret_cast<uintptr_t>(f_in) | reinterpret_cast<uintptr_t>(f_out)) & 15u)
    return fail(LBM_EINVAL, "f_in and f_out must be 16-byte aligned");

  // once per device, with that device current: the scratch array's device address and the
  // kernels' shared-memory limit (both precisions)
  cudaError_t se = cudaSuccess;
  double* scratch = scratch_on_device(dev, &se);
  if (!scratch) {
    snprintf(err, sizeof(err), "scratch set-up failed: %s", cudaGetErrorString(se));
    return fail(LBM_ECUDA, err);
  }

  lbm::StepTiling t;
  if ((rc = lbm::plan_step_tiling(*p, nsm, &t, err))) return fail(rc, err);
  if (t.nbands > kMaxCtas) {
    snprintf(err, sizeof(err), "lattice too wide for the static scratch: %d x-bands > %d (nx <= %d)", t.nbands,
             kMaxCtas, kMaxCtas * t.band_w);
    return fail(LBM_EINVAL, err);
  }
  // The plan fills one wave: nbands x nstrips <= max(nbands, SMs x resident CTAs per SM),
  // 304 on GB300 (152 SMs x 2), so this only acts on a GPU with more than 4096 resident
  // step CTAs: fewer, taller strips (ceil(ny / ceil(ny / m)) <= m strips for m = 4096 / nbands)
  if (t.nbands * t.nstrips > kMaxCtas) {
    const int nstrips = kMaxCtas / t.nbands;
    t.strip_h = (p->ny + nstrips - 1) / nstrips;
    t.nstrips = (p->ny + t.strip_h - 1) / t.strip_h;
  }
  const int P = t.nbands * t.nstrips;
  const double rho_ref = std::isnan(p->rho_ref) ? 0.0 : p->rho_ref;
  if (!std::isfinite(rho_ref)) return fail(LBM_EINVAL, "rho_ref must be finite or NaN");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* part_in = scratch;
  double* part_out = scratch + kMaxCtas;
  int* status = reinterpret_cast<int*>(scratch + 2 * kMaxCtas);
  // <rho> enters only Eq. Gravity_2: the mass partials of f_in (one extra read of it) are
  // formed only for that form
  const bool need_mean = p->gravity_form == LBM_GRAVITY_RHO_MINUS_MEAN_G;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);  // the array keeps the last call's status
  if (e == cudaSuccess && need_mean) e = lbm::launch_partials(p->precision, f_in, p->nx, p->ny, part_in, P, s);
  if (e == cudaSuccess) {
    lbm::StepIO io{};
    io.fin = f_in;
    io.fout = f_out;
    io.part_in = part_in;
    io.npart_in = need_mean ? P : 0;
    io.part_out = part_out;
    io.status = status;
    e = lbm::launch_step(p->precision, lbm::MODE_STEP, t, lbm::phys_from_params(*p, rho_ref), io, s);
  }
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(err, sizeof(err), "lbm_step_noalloc: %s", cudaGetErrorString(e));
    return fail(LBM_ECUDA, err);
  }
  if (st & lbm::STATUS_TIMEOUT) return fail(LBM_ETIMEOUT, "a device wait timed out");
  if (st & lbm::STATUS_NONPHYS)
    return fail(LBM_ENONPHYS, "non-physical state: rho <= 0, NaN, or 2 (p_EOS - rho/3)/G < 0 somewhere");
  return LBM_OK;
}
