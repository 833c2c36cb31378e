// Slabs of one large domain, one per GPU (declared in include/lbm.h, lbm_slab_*).
//
// A domain of nx x ny nodes (x periodic, walls below row 0 and above row ny - 1) is cut
// into horizontal slabs. A slab holds its own rows [y0, y0 + ny_own) plus LBM_SLAB_HALO = 2
// ghost rows below and above, in a caller-owned buffer real[9][ny_own + 4][nx]. One step
// of a slab is the fused kernel of lbm_kernels.cu restricted to the own rows: pull
// streaming (Eq. LBE) reads the ghost row next to the slab, and the Shan-Chen stencil
// (Eq. ShanChenForce) needs psi of that ghost row, which in turn pulls from the outer one;
// walls apply only where the slab meets the domain's bottom or top. Between steps the
// caller refreshes the ghost rows from the neighbouring slabs and adds the slabs' FP64
// mass partials element-wise across ranks (the <rho> of Eq. Gravity_2 is a mean over the
// whole domain; the next step's kernel finishes the sum in a fixed order); these calls
// allocate nothing and move no data between GPUs themselves.
#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_physics.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>

namespace {

constexpr int kHalo = LBM_SLAB_HALO;

int fail(int code, const char* msg) {
  lbm::set_last_error(msg);
  return code;
}

// The step's tiling for a slab: strips over the own rows only, buffer rows, wall rows
// where the slab touches the domain's ends, the whole domain's node count for <rho>.
int slab_tiling(const lbm_params* p, const lbm_slab* s, lbm::StepTiling* t, char* err) {
  int rc = lbm::validate_params(p, err);
  if (rc) return rc;
  if (!s) {
    snprintf(err, 512, "slab is NULL");
    return LBM_EINVAL;
  }
  if (p->thermal) {
    snprintf(err, 512, "slabs are isothermal (thermal must be 0)");
    return LBM_EINVAL;
  }
  if (s->reserved != 0 || s->ny_own < 1 || s->y0 < 0 || s->y0 + s->ny_own > p->ny) {
    snprintf(err, 512, "slab rows [%d, %d) outside the domain's %d rows", s->y0, s->y0 + s->ny_own, p->ny);
    return LBM_EINVAL;
  }
  const bool wall_lo = s->y0 == 0, wall_hi = s->y0 + s->ny_own == p->ny;
  // a halo of kHalo rows must come from the one neighbour on each open side
  if (s->ny_own < kHalo && !(wall_lo && wall_hi)) {
    snprintf(err, 512, "a slab with a neighbour needs at least %d rows (got %d)", kHalo, s->ny_own);
    return LBM_EINVAL;
  }
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    snprintf(err, 512, "no CUDA device");
    return LBM_ECUDA;
  }
  // the plan of the last call on this thread is reused while the device and the lattice's
  // shape are the same (a step is called once per time step; the plan needs an occupancy query)
  struct PlanKey {
    int dev, precision, nx, ny, y0, ny_own, wall;
  };
  thread_local PlanKey last_key{-1, 0, 0, 0, 0, 0, 0};
  thread_local lbm::StepTiling last_plan{};
  const PlanKey key{dev, p->precision, p->nx, p->ny, s->y0, s->ny_own, p->wall};
  if (std::memcmp(&key, &last_key, sizeof(key)) == 0) {
    *t = last_plan;
    return LBM_OK;
  }
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    snprintf(err, 512, "no CUDA device");
    return LBM_ECUDA;
  }
  if ((rc = lbm::prepare_step_kernels(dev, p->precision, err))) return rc;
  lbm_params q = *p;
  q.ny = s->ny_own;  // strips over the own rows
  if ((rc = lbm::plan_step_tiling(q, nsm, t, err))) return rc;
  const int rows = s->ny_own + 2 * kHalo;
  t->ny = rows;
  t->y_begin = kHalo;
  t->y_end = kHalo + s->ny_own;
  t->ylo = wall_lo ? kHalo : 0;
  t->yhi = wall_hi ? kHalo + s->ny_own - 1 : rows - 1;
  t->n_total = double(p->nx) * double(p->ny);
  last_plan = *t;
  last_key = key;
  return LBM_OK;
}

double slab_rho_ref(const lbm_params* p) { return std::isnan(p->rho_ref) ? 0.0 : p->rho_ref; }

// own rows of a slab buffer: g_i = w_i (rho0 - rho_ref), the rest equilibrium of Eq.
// EquilibriumDistribution; rho0 is [ny_own][nx]
template <typename T>
__global__ void slab_init_kernel(const double* __restrict__ rho0, T* __restrict__ f, int nx, int rows, int ny_own,
                                 double rho_ref) {
  const size_t n = size_t(nx) * ny_own, plane = size_t(nx) * rows, off = size_t(kHalo) * nx;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < n; q += size_t(gridDim.x) * blockDim.x) {
    const double d = rho0[q] - rho_ref;
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i * plane + off + q] = T(lbm::w_of(i) * d);
  }
}

// FP64 partial sums of the stored deviations of the own rows (block b: a contiguous chunk)
template <typename T>
__global__ void slab_partials_kernel(const T* __restrict__ f, int nx, int rows, int ny_own, double* __restrict__ part) {
  __shared__ double red[32];
  const size_t n = size_t(nx) * ny_own, plane = size_t(nx) * rows, off = size_t(kHalo) * nx;
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t q0 = blockIdx.x * chunk, q1 = min(n, q0 + chunk);
  lbm::Acc<T> acc;
  for (size_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    T g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = f[i * plane + off + q];
    acc.add9(g);
  }
  const double v = lbm::warp_sum(acc.value());
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const double t = lbm::warp_sum(threadIdx.x < int(blockDim.x >> 5) ? red[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

int grid_for(size_t n) { return int(std::max<size_t>(1, std::min<size_t>(4096, (n + 255) / 256))); }

// the step's bulk copies start on 16-byte boundaries of the planes
bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

}  // namespace

extern "C" {

int lbm_slab_partials(const lbm_params* p, const lbm_slab* s, int* count) {
  char err[512];
  lbm::StepTiling t;
  const int rc = slab_tiling(p, s, &t, err);
  if (rc) return fail(rc, err);
  if (!count) return fail(LBM_EINVAL, "count is NULL");
  *count = std::max(t.nbands * t.nstrips, 1);
  return LBM_OK;
}

int lbm_slab_init(const lbm_params* p, const lbm_slab* s, const double* rho0, void* f, void* stream) {
  char err[512];
  lbm::StepTiling t;
  const int rc = slab_tiling(p, s, &t, err);
  if (rc) return fail(rc, err);
  if (!rho0 || !f) return fail(LBM_EINVAL, "rho0 and f must be device arrays");
  if (misaligned(f)) return fail(LBM_EINVAL, "f must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = size_t(p->nx) * s->ny_own;
  if (p->precision == LBM_FP32)
    slab_init_kernel<float><<<grid_for(n), 256, 0, st>>>(rho0, static_cast<float*>(f), p->nx, t.ny, s->ny_own,
                                                          slab_rho_ref(p));
  else
    slab_init_kernel<double><<<grid_for(n), 256, 0, st>>>(rho0, static_cast<double*>(f), p->nx, t.ny, s->ny_own,
                                                           slab_rho_ref(p));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_slab_mass(const lbm_params* p, const lbm_slab* s, const void* f, double* part, int npart, void* stream) {
  char err[512];
  lbm::StepTiling t;
  const int rc = slab_tiling(p, s, &t, err);
  if (rc) return fail(rc, err);
  if (!f || !part) return fail(LBM_EINVAL, "f and part must be device arrays");
  if (misaligned(f)) return fail(LBM_EINVAL, "f must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int P = std::max(t.nbands * t.nstrips, 1);
  if (npart < P) {
    snprintf(err, sizeof(err), "part holds %d values, the slab needs %d (lbm_slab_partials)", npart, P);
    return fail(LBM_EINVAL, err);
  }
  if (p->precision == LBM_FP32)
    slab_partials_kernel<float><<<P, 256, 0, st>>>(static_cast<const float*>(f), p->nx, t.ny, s->ny_own, part);
  else
    slab_partials_kernel<double><<<P, 256, 0, st>>>(static_cast<const double*>(f), p->nx, t.ny, s->ny_own, part);
  cudaError_t e = cudaGetLastError();
  // the entries past this slab's count are zero: an element-wise sum over ranks adds them
  if (e == cudaSuccess && npart > P) e = cudaMemsetAsync(part + P, 0, sizeof(double) * size_t(npart - P), st);
  if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_slab_step(const lbm_params* p, const lbm_slab* s, const void* f_in, void* f_out, const double* part_in,
                  int npart_in, double* part_out, int npart_out, int* status, void* stream) {
  char err[512];
  lbm::StepTiling t;
  const int rc = slab_tiling(p, s, &t, err);
  if (rc) return fail(rc, err);
  const bool form2 = p->gravity_form == LBM_GRAVITY_RHO_MINUS_MEAN_G;
  if (!f_in || !f_out || f_in == f_out || !part_out || !status || (form2 && (!part_in || npart_in < 1)))
    return fail(LBM_EINVAL,
                "f_in, f_out (distinct), part_out, status (and part_in for Eq. Gravity_2) must be set");
  if (part_in == part_out) return fail(LBM_EINVAL, "part_in and part_out must be distinct");
  if (misaligned(f_in) || misaligned(f_out)) return fail(LBM_EINVAL, "f_in and f_out must be 16-byte aligned");
  if (npart_out < t.nbands * t.nstrips) {
    snprintf(err, sizeof(err), "part_out holds %d values, the step writes %d (lbm_slab_partials)", npart_out,
             t.nbands * t.nstrips);
    return fail(LBM_EINVAL, err);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lbm::StepIO io{};
  io.fin = f_in;
  io.fout = f_out;
  io.part_in = part_in;
  io.npart_in = form2 ? npart_in : 0;
  io.part_out = part_out;
  io.status = status;
  cudaError_t e =
      lbm::launch_step(p->precision, lbm::MODE_STEP, t, lbm::phys_from_params(*p, slab_rho_ref(p)), io, st);
  // the entries past this slab's count are zero (the buffer may hold the last sum over ranks)
  const int P = t.nbands * t.nstrips;
  if (e == cudaSuccess && npart_out > P)
    e = cudaMemsetAsync(part_out + P, 0, sizeof(double) * size_t(npart_out - P), st);
  if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"
