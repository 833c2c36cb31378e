// Energy equation of the thermal variant (arXiv 2301.12869, Sec. III, Eq. Energy_Equation):
//
//   dT/dt = -u . grad T + (kappa/(rho c_v)) lap T - (T/(rho c_v)) (dp_EOS/dT)_rho div u
//
// with (dp_EOS/dT)_rho = rho R Z(eta) of the Carnahan-Starling EOS (Eq. EOS), isotropic
// D2Q9-weighted central differences (d_a phi = 3 sum_i w_i c_ia phi(x + c_i),
// lap phi = 6 sum_i w_i (phi(x + c_i) - phi(x))), Heun's second-order Runge-Kutta with
// dt = 1, and Dirichlet walls half a link beyond the first and last rows (ghost rows
// T(-1) = 2 T_bot - T(0), u(-1) = -u(0), likewise at the top) - or, with Zou-He wet-node
// walls, T held at T_bot and T_top on the wall rows 0 and ny - 1 themselves. rho and u come
// from the moments pass that follows each LBM step.
//
// One launch does the whole Heun step. A CTA owns a TX x TY tile of nodes and stages T, u
// with a halo of two nodes in shared memory, and for the tile plus its one-node ring the
// two coefficients of the right-hand side that depend on rho alone (kappa/(rho c_v) and
// R Z(eta)/c_v: the rho of (dp/dT)_rho = rho R Z cancels against 1/(rho c_v)), each
// evaluated once per node. Stage 1 (k1, T* = T + k1) runs on the tile plus its ring,
// stage 2 (k2) on the tile, so no grid-wide barrier separates the stages. The new field
// goes to a second buffer. rho and u come in the field's own precision (FP32 handles get
// them as floats from the moments pass: FP64 conversions are slow on GB300).
#include "lbm_internal.h"
#include "lbm_physics.cuh"
#include "lbm_ptx.cuh"

#include <cuda_runtime.h>

namespace lbm {
namespace {

constexpr int TX = 32, TY = 16;
constexpr int W2 = TX + 4, H2 = TY + 4;  // T, u, v: two-node halo
constexpr int W1 = TX + 2, H1 = TY + 2;  // coefficients, T*, k1: one-node halo

template <typename T>
struct EnergyArgs {
  int nx, ny;
  int wall_nodes;  // 1: rows 0 and ny - 1 are wall nodes at fixed temperature (Zou-He walls)
  T R, b4, c_v, kappa, twoTbot, twoTtop;
};

// D2Q9 direction i: (cx, cy) in the order of Eq. VelocitySet
__device__ __forceinline__ int cx_of(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Right-hand side of the energy equation at the node whose T sits at Ts[c] (row stride sw)
// and whose u, v sit at U[cu], V[cu] (row stride uw); ck = kappa/(rho c_v), cz = R Z/c_v.
template <typename T>
__device__ __forceinline__ T rate(const T* Ts, int c, int sw, const T* U, const T* V, int cu, int uw, T ck, T cz) {
  const T tc = Ts[c];
  T gx = T(0), gy = T(0), lap = T(0), div = T(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int cx = cx_of(i), cy = cy_of(i);
    const T w = T(w_of(i));
    const T tn = Ts[c + cy * sw + cx];
    gx += w * T(cx) * tn;
    gy += w * T(cy) * tn;
    lap += w * (tn - tc);
    div += w * (T(cx) * U[cu + cy * uw + cx] + T(cy) * V[cu + cy * uw + cx]);
  }
  return -(U[cu] * (T(3) * gx) + V[cu] * (T(3) * gy)) + ck * (T(6) * lap) - tc * cz * (T(3) * div);
}

template <typename T>
__global__ void __launch_bounds__(TX * TY) heun_kernel(const EnergyArgs<T> a, const T* __restrict__ rho,
                                                      const T* __restrict__ ux, const T* __restrict__ uy,
                                                      const T* __restrict__ Tin, T* __restrict__ Tout) {
  __shared__ T sT[H2 * W2], sU[H2 * W2], sV[H2 * W2];
  __shared__ T sK[H1 * W1], sZ[H1 * W1], sS[H1 * W1], sk1[H1 * W1];  // kappa/(rho c_v), R Z/c_v, T*, k1
  griddep_wait();  // launched as a dependent of the moments pass: rho, u are complete
  griddep_launch_dependents();
  const int nx = a.nx, ny = a.ny;
  const int tid = threadIdx.y * TX + threadIdx.x;
  // x in [x0 - 2, x0 + TX + 1]: one conditional shift unless the lattice is narrower than that
  const bool wide = nx >= W2;
  auto wrap = [nx, wide](int x) {
    if (wide) return x < 0 ? x + nx : (x >= nx ? x - nx : x);
    x %= nx;
    return x < 0 ? x + nx : x;
  };
  const T inv_cv = recip(a.c_v);
  const int x0 = blockIdx.x * TX;
  for (int y0 = blockIdx.y * TY; y0 < ny; y0 += gridDim.y * TY) {
    // T, u, v on rows y0-2 .. y0+TY+1: ghost rows -1 and ny by the wall rules, rows beyond
    // them are never read
    for (int k = tid; k < H2 * W2; k += TX * TY) {
      const int r = k / W2, y = y0 - 2 + r, x = wrap(x0 - 2 + (k - r * W2));
      T t = T(0), u = T(0), v = T(0);
      if (y >= 0 && y < ny) {
        const size_t n = size_t(y) * nx + x;
        t = Tin[n];
        u = ux[n];
        v = uy[n];
      } else if (y == -1 || y == ny) {
        const size_t n = size_t(y < 0 ? 0 : ny - 1) * nx + x;
        t = (y < 0 ? a.twoTbot : a.twoTtop) - Tin[n];
        u = -ux[n];
        v = -uy[n];
      }
      sT[k] = t;
      sU[k] = u;
      sV[k] = v;
    }
    // the rho-dependent coefficients on the tile and its ring (real rows)
    for (int k = tid; k < H1 * W1; k += TX * TY) {
      const int r = k / W1, y = y0 - 1 + r, x = wrap(x0 - 1 + (k - r * W1));
      T ck = T(0), cz = T(0);
      if (y >= 0 && y < ny) {
        const T rh = rho[size_t(y) * nx + x];
        const T eta = a.b4 * rh;
        const T om = T(1) - eta;
        ck = a.kappa * recip(rh * a.c_v);
        cz = a.R * (T(1) + eta * (T(1) + eta * (T(1) - eta))) * recip(om * om * om) * inv_cv;
      }
      sK[k] = ck;
      sZ[k] = cz;
    }
    __syncthreads();

    // stage 1 on the tile and its ring (real rows only): T* = T + k1
    for (int k = tid; k < H1 * W1; k += TX * TY) {
      const int r = k / W1, c = k - r * W1, y = y0 - 1 + r;
      const int c2 = (r + 1) * W2 + (c + 1);
      if (y >= 0 && y < ny) {
        const T k1 = (a.wall_nodes && (y == 0 || y == ny - 1)) ? T(0) : rate(sT, c2, W2, sU, sV, c2, W2, sK[k], sZ[k]);
        sk1[k] = k1;
        sS[k] = sT[c2] + k1;
      }
    }
    __syncthreads();
    // ghost rows of T* from its first and last rows
    for (int k = tid; k < H1 * W1; k += TX * TY) {
      const int r = k / W1, y = y0 - 1 + r;
      if (y == -1 && !a.wall_nodes) sS[k] = a.twoTbot - sS[k + W1];
      if (y == ny && !a.wall_nodes) sS[k] = a.twoTtop - sS[k - W1];
    }
    __syncthreads();

    // stage 2 on the tile: T_new = T + (k1 + k2)/2
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x < nx && y < ny) {
      const int c1 = (threadIdx.y + 1) * W1 + (threadIdx.x + 1);
      const int c2 = (threadIdx.y + 2) * W2 + (threadIdx.x + 2);
      const T t = sT[c2];
      const T k1 = sk1[c1];
      if (a.wall_nodes && (y == 0 || y == ny - 1)) {
        Tout[size_t(y) * nx + x] = T(0.5) * (y == 0 ? a.twoTbot : a.twoTtop);  // wall node: T_bot / T_top
      } else {
        const T k2 = rate(sS, c1, W1, sU, sV, c2, W2, sK[c1], sZ[c1]);
        Tout[size_t(y) * nx + x] = t + T(0.5) * (k1 + k2);
      }
    }
    __syncthreads();  // the next tile of this CTA overwrites the shared arrays
  }
}

// the steady conduction profile (Eq. Temp_Profile): linear from T_bot at y = -1/2 to T_top
// at y = ny - 1/2 (bounce-back walls), or from row 0 to row ny - 1 (wall nodes)
template <typename T>
__global__ void linear_T_kernel(int nx, int ny, double T_bot, double T_top, int wall_nodes, T* Tf) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  for (int y = blockIdx.y; y < ny; y += gridDim.y)
    if (x < nx)
      Tf[size_t(y) * nx + x] = T(wall_nodes ? T_bot + (T_top - T_bot) * double(y) / double(ny - 1)
                                            : T_bot + (T_top - T_bot) * (double(y) + 0.5) / ny);
}

unsigned rows_grid(int rows) { return unsigned(rows < 65535 ? rows : 65535); }

}  // namespace

cudaError_t launch_energy_step(int precision, int nx, int ny, int wall_nodes, double R, double b, double c_v,
                               double kappa, double T_bot, double T_top, const void* rho, const void* ux,
                               const void* uy, const void* Tin, void* Tout, cudaStream_t stream) {
  const dim3 grid((nx + TX - 1) / TX, rows_grid((ny + TY - 1) / TY)), block(TX, TY);
  if (precision == 1) {
    const EnergyArgs<float> a{nx, ny, wall_nodes, float(R), float(b / 4.0), float(c_v), float(kappa),
                              float(2.0 * T_bot), float(2.0 * T_top)};
    return launch_dependent(heun_kernel<float>, grid, block, 0, stream, a, static_cast<const float*>(rho),
                            static_cast<const float*>(ux), static_cast<const float*>(uy),
                            static_cast<const float*>(Tin), static_cast<float*>(Tout));
  } else {
    const EnergyArgs<double> a{nx, ny, wall_nodes, R, b / 4.0, c_v, kappa, 2.0 * T_bot, 2.0 * T_top};
    return launch_dependent(heun_kernel<double>, grid, block, 0, stream, a, static_cast<const double*>(rho),
                            static_cast<const double*>(ux), static_cast<const double*>(uy),
                            static_cast<const double*>(Tin), static_cast<double*>(Tout));
  }
}

cudaError_t launch_linear_T(int precision, int nx, int ny, double T_bot, double T_top, int wall_nodes, void* Tf,
                            cudaStream_t stream) {
  const dim3 grid((nx + 255) / 256, rows_grid(ny)), block(256);
  if (precision == 1)
    linear_T_kernel<float><<<grid, block, 0, stream>>>(nx, ny, T_bot, T_top, wall_nodes, static_cast<float*>(Tf));
  else
    linear_T_kernel<double><<<grid, block, 0, stream>>>(nx, ny, T_bot, T_top, wall_nodes, static_cast<double*>(Tf));
  return cudaGetLastError();
}

}  // namespace lbm
