// Energy equation of the thermal variant (arXiv 2301.12869, Sec. III, Eq. Energy_Equation):
//
//   dT/dt = -u . grad T + (kappa/(rho c_v)) lap T - (T/(rho c_v)) (dp_EOS/dT)_rho div u
//
// with (dp_EOS/dT)_rho = rho R Z(eta) of the Carnahan-Starling EOS (Eq. EOS), isotropic
// D2Q9-weighted central differences (d_a phi = 3 sum_i w_i c_ia phi(x + c_i),
// lap phi = 6 sum_i w_i (phi(x + c_i) - phi(x))), Heun's second-order Runge-Kutta with
// dt = 1, and Dirichlet walls half a link beyond the first and last rows (ghost rows
// T(-1) = 2 T_bot - T(0), u(-1) = -u(0), likewise at the top). rho and u come from the
// moments pass that follows each LBM step.
#include "lbm_internal.h"
#include "lbm_physics.cuh"

#include <cuda_runtime.h>

namespace lbm {
namespace {

struct EnergyArgs {
  int nx, ny;
  double R, b, c_v, kappa, T_bot, T_top;
};

template <typename T>
__device__ __forceinline__ T energy_rate(const EnergyArgs& a, const T* src, const double* rho, const double* ux,
                                         const double* uy, int x, int y) {
  const int nx = a.nx, ny = a.ny;
  const size_t node = size_t(y) * nx + x;
  const T tc = src[node];
  T gx = T(0), gy = T(0), lap = T(0), div = T(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int cx = i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
    const int cy = cy_of(i);
    const int xn = x + cx < 0 ? nx - 1 : (x + cx >= nx ? 0 : x + cx);
    const int yn = y + cy;
    T Tn, un_x, un_y;
    if (yn < 0) {  // ghost row below the bottom wall
      const size_t m = size_t(xn);
      Tn = T(2.0 * a.T_bot) - src[m];
      un_x = -T(ux[m]);
      un_y = -T(uy[m]);
    } else if (yn >= ny) {  // ghost row above the top wall
      const size_t m = size_t(ny - 1) * nx + xn;
      Tn = T(2.0 * a.T_top) - src[m];
      un_x = -T(ux[m]);
      un_y = -T(uy[m]);
    } else {
      const size_t m = size_t(yn) * nx + xn;
      Tn = src[m];
      un_x = T(ux[m]);
      un_y = T(uy[m]);
    }
    const T w = T(w_of(i));
    gx += w * T(cx) * Tn;
    gy += w * T(cy) * Tn;
    lap += w * (Tn - tc);
    div += w * (T(cx) * un_x + T(cy) * un_y);
  }
  gx *= T(3);
  gy *= T(3);
  lap *= T(6);
  div *= T(3);
  const T r = T(rho[node]);
  const T eta = T(a.b / 4.0) * r;
  const T om = T(1) - eta;
  const T Z = (T(1) + eta * (T(1) + eta * (T(1) - eta))) / (om * om * om);
  const T dpdT = r * T(a.R) * Z;
  const T inv = T(1) / (r * T(a.c_v));
  return -(T(ux[node]) * gx + T(uy[node]) * gy) + T(a.kappa) * inv * lap - tc * dpdT * inv * div;
}

// stage 1: k1 = L(T), T* = T + k1; stage 2: T <- T + (k1 + L(T*)) / 2
template <typename T>
__global__ void energy_stage_kernel(const EnergyArgs a, int stage, const double* rho, const double* ux,
                                    const double* uy, T* Tcur, T* Tstar, T* k1buf) {
  const size_t n = size_t(a.nx) * a.ny;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < n; q += size_t(gridDim.x) * blockDim.x) {
    const int x = int(q % a.nx), y = int(q / a.nx);
    if (stage == 1) {
      const T k1 = energy_rate(a, Tcur, rho, ux, uy, x, y);
      k1buf[q] = k1;
      Tstar[q] = Tcur[q] + k1;
    } else {
      const T k2 = energy_rate(a, Tstar, rho, ux, uy, x, y);
      Tcur[q] = Tcur[q] + T(0.5) * (k1buf[q] + k2);
    }
  }
}

// the steady conduction profile (Eq. Temp_Profile): linear from T_bot at y = -1/2 to T_top
// at y = ny - 1/2
template <typename T>
__global__ void linear_T_kernel(int nx, int ny, double T_bot, double T_top, T* Tf) {
  const size_t n = size_t(nx) * ny;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < n; q += size_t(gridDim.x) * blockDim.x) {
    const double y = double(q / nx);
    Tf[q] = T(T_bot + (T_top - T_bot) * (y + 0.5) / ny);
  }
}

int grid_of(size_t n) {
  size_t g = (n + 255) / 256;
  return int(g > 8192 ? 8192 : (g < 1 ? 1 : g));
}

}  // namespace

cudaError_t launch_energy_step(int precision, int nx, int ny, double R, double b, double c_v, double kappa,
                               double T_bot, double T_top, const double* rho, const double* ux, const double* uy,
                               void* Tcur, void* Tstar, void* k1, cudaStream_t stream) {
  const EnergyArgs a{nx, ny, R, b, c_v, kappa, T_bot, T_top};
  const int g = grid_of(size_t(nx) * ny);
  for (int stage = 1; stage <= 2; ++stage) {
    if (precision == 1)
      energy_stage_kernel<float><<<g, 256, 0, stream>>>(a, stage, rho, ux, uy, static_cast<float*>(Tcur),
                                                        static_cast<float*>(Tstar), static_cast<float*>(k1));
    else
      energy_stage_kernel<double><<<g, 256, 0, stream>>>(a, stage, rho, ux, uy, static_cast<double*>(Tcur),
                                                         static_cast<double*>(Tstar), static_cast<double*>(k1));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_linear_T(int precision, int nx, int ny, double T_bot, double T_top, void* Tf, cudaStream_t stream) {
  const int g = grid_of(size_t(nx) * ny);
  if (precision == 1)
    linear_T_kernel<float><<<g, 256, 0, stream>>>(nx, ny, T_bot, T_top, static_cast<float*>(Tf));
  else
    linear_T_kernel<double><<<g, 256, 0, stream>>>(nx, ny, T_bot, T_top, static_cast<double*>(Tf));
  return cudaGetLastError();
}

}  // namespace lbm
