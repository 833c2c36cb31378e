// Energy equation of the thermal variant (arXiv 2301.12869, Sec. III, Eq. Energy_Equation):
//
//   dT/dt = -u . grad T + (kappa/(rho c_v)) lap T - (T/(rho c_v)) (dp_EOS/dT)_rho div u
//
// with (dp_EOS/dT)_rho = rho R Z(eta) of the Carnahan-Starling EOS (Eq. EOS), isotropic
// D2Q9-weighted central differences (d_a phi = 3 sum_i w_i c_ia phi(x + c_i),
// lap phi = 6 sum_i w_i (phi(x + c_i) - phi(x))), Heun's second-order Runge-Kutta with
// dt = 1, and Dirichlet walls half a link beyond the first and last rows (ghost rows
// T(-1) = 2 T_bot - T(0), u(-1) = -u(0), likewise at the top) - or, with Zou-He wet-node
// walls, T held at T_bot and T_top on the wall rows 0 and ny - 1 themselves. rho and u are
// those of the same time level as T: the fused LBM step stores them as it collides (the
// streamed populations, the force of T^n).
//
// One launch does the whole Heun step (heun_strip_kernel below): each warp walks a strip
// of rows with the stencil's rows held in registers, computing k1 and T* = T + k1 one row
// ahead of k2, so both Heun stages run in one pass without shared memory or CTA
// barriers. rho and u come in the field's own precision (FP32 handles get them as floats
// from the step: FP64 conversions are slow on GB300).
#include "lbm_internal.h"
#include "lbm_physics.cuh"
#include "lbm_ptx.cuh"

#include <cuda_runtime.h>

namespace lbm {
namespace {

template <typename T>
struct EnergyArgs {
  int nx, ny;
  int wall_nodes;  // 1: rows 0 and ny - 1 are wall nodes at fixed temperature (Zou-He walls)
  T R, b4, c_v, kappa, twoTbot, twoTtop;
};

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// ---- the strip kernel: one warp walks kStripRows rows of kOwn columns
//
// Lane l of a warp holds column x0 - 2 + l (x periodic); lanes 2 .. 29 own their column,
// lanes 0, 1, 30, 31 are its halo. x neighbours come from the adjacent lanes by shuffles,
// y neighbours from a window of rows in registers: walking up, input row q (T, u, v and
// the two rho coefficients) is loaded, k1 and T* = T + k1 are formed for row q - 1, and
// k2 and T_new = T + (k1 + k2)/2 for row q - 2. Lanes 1 .. 30 get valid k1 (their
// neighbours are loaded), so the owned lanes 2 .. 29 have T* on both sides. Each input
// value is loaded once per warp (plus the 4 halo lanes and 2 + 2 halo rows of the strip).
constexpr int kOwn = 28;
constexpr int kStripRows = 16;
constexpr int kStripWarps = 8;  // warps per CTA: consecutive strips of the same columns

template <typename T>
struct Nb {  // a value at the lane's column and at its left and right neighbours
  T c, l, r;
};
template <typename T>
__device__ __forceinline__ Nb<T> nb(T v) {
  return {v, __shfl_up_sync(0xffffffffu, v, 1), __shfl_down_sync(0xffffffffu, v, 1)};
}
template <typename T>
__device__ __forceinline__ Nb<T> affine(T a, T s, const Nb<T>& v) {  // a + s v, pointwise
  return {a + s * v.c, a + s * v.l, a + s * v.r};
}

// Right-hand side of Eq. Energy_Equation at the lane's node of row r from T on rows
// r-1 (ts), r (tc), r+1 (tn), u, v on the same rows and the node's coefficients: the
// D2Q9-weighted differences with w = 1/9 (axes) and 1/36 (diagonals).
template <typename T>
__device__ __forceinline__ T rate_nb(const Nb<T>& ts, const Nb<T>& tc, const Nb<T>& tn, const Nb<T>& us,
                                     const Nb<T>& uc, const Nb<T>& un, const Nb<T>& vs, const Nb<T>& vc,
                                     const Nb<T>& vn, T ck, T cz) {
  const T w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
  const T gx = w1 * (tc.r - tc.l) + w2 * ((tn.r - tn.l) + (ts.r - ts.l));
  const T gy = w1 * (tn.c - ts.c) + w2 * ((tn.r + tn.l) - (ts.r + ts.l));
  const T lap = w1 * ((tc.r + tc.l) + (tn.c + ts.c)) + w2 * ((tn.r + tn.l) + (ts.r + ts.l)) - T(5.0 / 9.0) * tc.c;
  const T div = w1 * ((uc.r - uc.l) + (vn.c - vs.c)) + w2 * (((un.r - un.l) + (us.r - us.l)) + ((vn.r + vn.l) - (vs.r + vs.l)));
  return -(uc.c * (T(3) * gx) + vc.c * (T(3) * gy)) + ck * (T(6) * lap) - tc.c * cz * (T(3) * div);
}

template <typename T>
__global__ void __launch_bounds__(32 * kStripWarps) heun_strip_kernel(const EnergyArgs<T> a, const T* __restrict__ rho,
                                                                      const T* __restrict__ ux, const T* __restrict__ uy,
                                                                      const T* __restrict__ Tin, T* __restrict__ Tout) {
  griddep_wait();  // launched as a dependent of the step: rho, u are complete
  griddep_launch_dependents();
  const int nx = a.nx, ny = a.ny, lane = threadIdx.x;
  const int x0 = blockIdx.x * kOwn;
  int x = x0 - 2 + lane;  // periodic; a narrow lattice wraps more than once
  if (nx >= 32) {
    x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  } else {
    x %= nx;
    if (x < 0) x += nx;
  }
  const bool own = lane >= 2 && lane < 2 + kOwn && x0 + lane - 2 < nx;
  const int ya = (blockIdx.y * kStripWarps + threadIdx.y) * kStripRows;
  if (ya >= ny) return;  // uniform over the warp
  const int yb = min(ya + kStripRows, ny);
  const bool walls = a.wall_nodes != 0;
  const T inv_cv = recip(a.c_v), zero = T(0), half = T(0.5);
  // windows (row index relative to the input row q of the current iteration)
  Nb<T> t0{}, t1{}, t2{};            // T rows q-2, q-1, q
  Nb<T> u0{}, u1{}, u2{}, u3{};      // u rows q-3 .. q
  Nb<T> v0{}, v1{}, v2{}, v3{};      // v rows q-3 .. q
  Nb<T> s0{}, s1{}, s2{};            // T* rows q-3, q-2, q-1
  T ckA = zero, czA = zero, ckB = zero, czB = zero, ckC = zero, czC = zero;  // coefficients, rows q-2, q-1, q
  T k1a = zero, k1b = zero;          // k1 of rows q-2 (a) and q-1 (b)
  // Input rows are loaded four iterations before they are used (a ring of raw T, u, v,
  // rho in registers), so the global-load latency overlaps the work of the rows before.
  // A row outside the strip's range, or beyond the walls, loads nothing.
  const int q_first = ya - 2, q_last = yb + 1;
  auto fetch = [&](int q, T& t, T& u, T& v, T& r) {
    const bool real = q >= 0 && q < ny;
    const bool ghost = !walls && (q == -1 || q == ny);
    t = u = v = r = zero;
    if (q <= q_last && (real || ghost)) {
      const size_t n = size_t(real ? q : (q < 0 ? 0 : ny - 1)) * nx + x;
      t = Tin[n];
      u = ux[n];
      v = uy[n];
      if (real) r = rho[n];
    }
  };
  T pt0, pu0, pv0, pr0, pt1, pu1, pv1, pr1, pt2, pu2, pv2, pr2, pt3, pu3, pv3, pr3;  // rows q .. q + 3
  fetch(q_first, pt0, pu0, pv0, pr0);
  fetch(q_first + 1, pt1, pu1, pv1, pr1);
  fetch(q_first + 2, pt2, pu2, pv2, pr2);
  fetch(q_first + 3, pt3, pu3, pv3, pr3);
  for (int q = q_first; q <= q_last; ++q) {
    // ---- input row q: T, u, v with the wall ghosts, and the rho coefficients
    T tq = pt0, uq = pu0, vq = pv0;
    const T rq = pr0;
    pt0 = pt1; pu0 = pu1; pv0 = pv1; pr0 = pr1;
    pt1 = pt2; pu1 = pu2; pv1 = pv2; pr1 = pr2;
    pt2 = pt3; pu2 = pu3; pv2 = pv3; pr2 = pr3;
    fetch(q + 4, pt3, pu3, pv3, pr3);
    T ckq = zero, czq = zero;
    const bool real = q >= 0 && q < ny;
    const bool ghost = !walls && (q == -1 || q == ny);
    if (real || ghost) {
      if (ghost) {  // T(-1) = 2 T_bot - T(0), u(-1) = -u(0); likewise above the top row
        tq = (q < 0 ? a.twoTbot : a.twoTtop) - tq;
        uq = -uq;
        vq = -vq;
      } else {
        const T rh = rq;
        const T eta = a.b4 * rh;
        const T om = T(1) - eta;
        ckq = a.kappa * recip(rh * a.c_v);
        czq = a.R * (T(1) + eta * (T(1) + eta * (T(1) - eta))) * recip(om * om * om) * inv_cv;
      }
    }
    t0 = t1; t1 = t2; t2 = nb(tq);
    u0 = u1; u1 = u2; u2 = u3; u3 = nb(uq);
    v0 = v1; v1 = v2; v2 = v3; v3 = nb(vq);
    ckA = ckB; czA = czB; ckB = ckC; czB = czC; ckC = ckq; czC = czq;
    // ---- k1 and T* of row r1 = q - 1 (rows r1-1, r1, r1+1 are t0, t1, t2)
    const int r1 = q - 1;
    T k1 = zero;
    if (r1 >= 0 && r1 < ny && !(walls && (r1 == 0 || r1 == ny - 1)))
      k1 = rate_nb(t0, t1, t2, u1, u2, u3, v1, v2, v3, ckB, czB);
    s0 = s1; s1 = s2;
    s2 = nb(t1.c + k1);
    if (!walls && r1 == 0) s1 = affine(a.twoTbot, T(-1), s2);     // T*(-1) = 2 T_bot - T*(0)
    if (!walls && r1 == ny) s2 = affine(a.twoTtop, T(-1), s1);    // T*(ny) = 2 T_top - T*(ny-1)
    k1a = k1b;
    k1b = k1;
    // ---- k2 and T_new of row r2 = q - 2 (T* rows r2-1 .. r2+1 are s0, s1, s2)
    const int r2 = q - 2;
    if (r2 >= ya && r2 < yb && own) {
      T tn;
      if (walls && (r2 == 0 || r2 == ny - 1)) {
        tn = half * (r2 == 0 ? a.twoTbot : a.twoTtop);  // wall node: T_bot / T_top
      } else {
        const T k2 = rate_nb(s0, s1, s2, u0, u1, u2, v0, v1, v2, ckA, czA);
        tn = t0.c + half * (k1a + k2);
      }
      Tout[size_t(r2) * nx + x] = tn;
    }
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
  const int strips = (ny + kStripRows - 1) / kStripRows;
  const dim3 grid((nx + kOwn - 1) / kOwn, (strips + kStripWarps - 1) / kStripWarps), block(32, kStripWarps);
  if (precision == 1) {
    const EnergyArgs<float> a{nx, ny, wall_nodes, float(R), float(b / 4.0), float(c_v), float(kappa),
                              float(2.0 * T_bot), float(2.0 * T_top)};
    return launch_dependent(heun_strip_kernel<float>, grid, block, 0, stream, a, static_cast<const float*>(rho),
                            static_cast<const float*>(ux), static_cast<const float*>(uy),
                            static_cast<const float*>(Tin), static_cast<float*>(Tout));
  } else {
    const EnergyArgs<double> a{nx, ny, wall_nodes, R, b / 4.0, c_v, kappa, 2.0 * T_bot, 2.0 * T_top};
    return launch_dependent(heun_strip_kernel<double>, grid, block, 0, stream, a, static_cast<const double*>(rho),
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
