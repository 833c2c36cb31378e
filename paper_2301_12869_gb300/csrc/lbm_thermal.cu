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
  T b4, kP, kZ, twoTbot, twoTtop;  // b/4, (2/3) kappa/c_v, R/c_v, 2 T_bot, 2 T_top
};

// the walk's value type: one FP64 column per lane, or a pair of neighbouring FP32 columns
// per lane (packed FP32x2 arithmetic, 8-byte loads and stores)
template <typename V>
__device__ __forceinline__ V splat(typename VecTraits<V>::scalar x);
template <>
__device__ __forceinline__ double splat<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ f2 splat<f2>(float x) {
  return make_f2(x, x);
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ f2 recip(f2 x) { return make_f2(rcp_approx(lo(x)), rcp_approx(hi(x))); }

// ---- the strip kernel: one warp walks ROWS rows of 32 W - 4 columns (W columns a lane)
//
// Lane l of a warp holds columns x0 - 2 + W l .. x0 - 1 + W l (x periodic); the lanes whose
// columns lie 2 .. 32 W - 3 from the warp's left edge own them (W = 1: lanes 2 .. 29; W =
// 2: lanes 1 .. 30), the two columns at each edge are halo. x neighbours come from the
// adjacent columns - the lane's other column or a shuffle from the next lane - and y
// neighbours from a window of rows in registers: walking up, input row q (T, u, v, rho) is
// taken in, k1 and T* = T + k1 are formed for row q - 1, and k2 and T_new = T + (k1 + k2)/2
// for row q - 2. k1 is valid one column in from the edges, so the owned columns have T* on
// both sides.
//
// For fixed rho and u the right-hand side of Eq. Energy_Equation is linear in T, so at a
// node it is a 9-point stencil L(phi) = sum_i a_i phi(x + c_i) whose weights follow from
// the D2Q9-weighted differences (c_s^2 = 1/3, P = (2/3) kappa/(rho c_v), U = u/3, V = v/3):
//   axis neighbours   a = P - U c_x - V c_y
//   diagonal ones     a = (P - U c_x - V c_y)/4
//   centre            a = -5 P - (R Z(eta)/c_v) div u
// with div u = (1/3)[du(y) + v(y+1) - v(y-1)] + (1/12)[du(y+1) + du(y-1) + sv(y+1) - sv(y-1)],
// du = u(x+1) - u(x-1), sv = v(x+1) + v(x-1) of each row. Both Heun stages apply the same
// weights (k1 = L(T), k2 = L(T*)): they are formed once, at the first stage, and kept one
// row for the second. The row loop is unrolled in full, so the windows rotate by renaming.
template <typename V>
__host__ __device__ constexpr int own_columns() {
  return 32 * VecTraits<V>::width - 4;
}

template <typename V>
struct Nb {  // a value at the lane's column(s) and at the left and right neighbour of each
  V c, l, r;
};
__device__ __forceinline__ Nb<double> nb(double v) {
  return {v, __shfl_up_sync(0xffffffffu, v, 1), __shfl_down_sync(0xffffffffu, v, 1)};
}
__device__ __forceinline__ Nb<f2> nb(f2 v) {
  const float a = lo(v), b = hi(v);
  const float left = __shfl_up_sync(0xffffffffu, b, 1);    // column 2l - 1: the left lane's second
  const float right = __shfl_down_sync(0xffffffffu, a, 1);  // column 2l + 2: the right lane's first
  return {v, make_f2(left, a), make_f2(b, right)};
}
template <typename V>
__device__ __forceinline__ Nb<V> affine(V a, V s, const Nb<V>& v) {  // a + s v, pointwise
  return {a + s * v.c, a + s * v.l, a + s * v.r};
}
// v(x + 1) - v(x - 1) and v(x + 1) + v(x - 1) at the lane's column(s)
__device__ __forceinline__ double xdiff(double v) {
  return __shfl_down_sync(0xffffffffu, v, 1) - __shfl_up_sync(0xffffffffu, v, 1);
}
__device__ __forceinline__ double xsum(double v) {
  return __shfl_down_sync(0xffffffffu, v, 1) + __shfl_up_sync(0xffffffffu, v, 1);
}
__device__ __forceinline__ f2 xdiff(f2 v) {
  const float a = lo(v), b = hi(v);
  const float left = __shfl_up_sync(0xffffffffu, b, 1), right = __shfl_down_sync(0xffffffffu, a, 1);
  return make_f2(b - left, right - a);
}
__device__ __forceinline__ f2 xsum(f2 v) {
  const float a = lo(v), b = hi(v);
  const float left = __shfl_up_sync(0xffffffffu, b, 1), right = __shfl_down_sync(0xffffffffu, a, 1);
  return make_f2(left + b, a + right);
}

template <typename V>
struct Weights {  // the stencil weights of one node row: centre, E, W, N, S, NE, NW, SE, SW
  V c, e, w, n, s, ne, nw, se, sw;
};
template <typename V>
__device__ __forceinline__ Weights<V> weights(V P, V U, V Vv, V ac) {
  const V quarter = cst<V>(0.25);
  const V q = quarter * P, p = quarter * (U + Vv), m = quarter * (U - Vv);
  return {ac, P - U, P + U, P - Vv, P + Vv, q - p, q + m, q - m, q + p};
}
// L(phi) at the lane's node(s) from phi on the rows below (s), at (c) and above (n)
template <typename V>
__device__ __forceinline__ V apply(const Weights<V>& a, const Nb<V>& s, const Nb<V>& c, const Nb<V>& n) {
  V r0 = a.c * c.c, r1 = a.n * n.c;
  r0 = fmadd(a.e, c.r, r0);
  r1 = fmadd(a.s, s.c, r1);
  r0 = fmadd(a.w, c.l, r0);
  r1 = fmadd(a.ne, n.r, r1);
  r0 = fmadd(a.nw, n.l, r0);
  r1 = fmadd(a.se, s.r, r1);
  r0 = fmadd(a.sw, s.l, r0);
  return r0 + r1;
}

template <typename T, typename V, int ROWS, int WARPS, int AHEAD>
__global__ void __launch_bounds__(32 * WARPS, 2) heun_strip_kernel(const EnergyArgs<T> a, const T* __restrict__ rho,
                                                                   const T* __restrict__ ux, const T* __restrict__ uy,
                                                                   const T* __restrict__ Tin, T* __restrict__ Tout) {
  griddep_wait();  // launched as a dependent of the step: rho, u are complete
  griddep_launch_dependents();
  constexpr int W = VecTraits<V>::width;
  const int nx = a.nx, ny = a.ny, lane = threadIdx.x;
  const int x0 = blockIdx.x * own_columns<V>();
  const int rel = W * lane - 2;  // the lane's first column from the warp's owned ones
  int x = x0 + rel;              // periodic; a narrow lattice wraps more than once
  if (nx >= 32 * W) {
    x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  } else {
    x %= nx;
    if (x < 0) x += nx;
  }
  // (W = 2: nx is a multiple of 4 and x even, so a lane's pair never straddles the seam)
  const bool own = rel >= 0 && rel < own_columns<V>() && x0 + rel < nx;
  const int ya = (blockIdx.y * WARPS + threadIdx.y) * ROWS;
  if (ya >= ny) return;  // uniform over the warp
  const int yb = min(ya + ROWS, ny);
  const bool walls = a.wall_nodes != 0;
  const V zero = cst<V>(0.0), half = cst<V>(0.5), one = cst<V>(1.0), mone = cst<V>(-1.0);
  const V third = cst<V>(1.0 / 3.0), twelfth = cst<V>(1.0 / 12.0);
  const V twoTbot = splat<V>(a.twoTbot), twoTtop = splat<V>(a.twoTtop);
  const V kP = splat<V>(a.kP), kZ = splat<V>(a.kZ), b4 = splat<V>(a.b4);
  auto load = [&](const T* p, size_t n) { return *reinterpret_cast<const V*>(p + n); };
  // Input rows are loaded AHEAD rows before they are used (a ring of raw T, u, v, rho in
  // registers), so the global-load latency overlaps the work of the rows before. A row
  // outside the strip's range, or beyond the walls, loads nothing.
  const int q_last = yb + 1;
  struct Raw {
    V t, u, v, r;
  };
  auto fetch = [&](int q, Raw& w) {
    const bool real = q >= 0 && q < ny;
    const bool ghost = !walls && (q == -1 || q == ny);
    w.t = w.u = w.v = w.r = zero;
    if (q <= q_last && (real || ghost)) {
      const size_t n = size_t(real ? q : (q < 0 ? 0 : ny - 1)) * nx + x;
      w.t = load(Tin, n);
      w.u = load(ux, n);
      w.v = load(uy, n);
      if (real) w.r = load(rho, n);
    }
  };
  Raw ring[AHEAD];
#pragma unroll
  for (int d = 0; d < AHEAD; ++d) fetch(ya - 2 + d, ring[d]);
  // windows (row index relative to the input row q of the current iteration)
  Nb<V> t0{}, t1{}, t2{};                     // T rows q-2, q-1, q
  Nb<V> s0{}, s1{}, s2{};                     // T* rows q-3, q-2, q-1
  V du0 = zero, du1 = zero, du2 = zero;       // du rows q-2, q-1, q
  V vc0 = zero, vc1 = zero, vc2 = zero;       // v rows q-2, q-1, q
  V sv0 = zero, sv1 = zero, sv2 = zero;       // sv rows q-2, q-1, q
  V U1 = zero, U2 = zero, P1 = zero, P2 = zero, Z1 = zero, Z2 = zero;  // rows q-1, q
  Weights<V> wB{zero, zero, zero, zero, zero, zero, zero, zero, zero};  // weights of row q-2
  V k1B = zero;                                                         // k1 of row q-2
#pragma unroll
  for (int it = 0; it < ROWS + 4; ++it) {
    const int q = ya - 2 + it;
    // ---- input row q: T, u, v with the wall ghosts, and the rho-dependent factors
    const Raw in = ring[it % AHEAD];
    if (it + AHEAD < ROWS + 4) fetch(q + AHEAD, ring[it % AHEAD]);
    V tq = in.t, uq = in.u, vq = in.v;
    V Pq = zero, Zq = zero;
    const bool real = q >= 0 && q < ny;
    const bool ghost = !walls && (q == -1 || q == ny);
    if (ghost) {  // T(-1) = 2 T_bot - T(0), u(-1) = -u(0); likewise above the top row
      tq = (q < 0 ? twoTbot : twoTtop) - tq;
      uq = zero - uq;
      vq = zero - vq;
    } else if (real) {
      const V rh = in.r;
      const V eta = b4 * rh;
      const V om = one - eta;
      Pq = kP * recip(rh);                                                        // (2/3) kappa/(rho c_v)
      Zq = kZ * fmadd(eta, fmadd(eta, om, one), one) * recip(om * om * om);       // R Z(eta)/c_v
    }
    t0 = t1; t1 = t2; t2 = nb(tq);
    du0 = du1; du1 = du2; du2 = xdiff(uq);
    vc0 = vc1; vc1 = vc2; vc2 = vq;
    sv0 = sv1; sv1 = sv2; sv2 = xsum(vq);
    U1 = U2; U2 = third * uq;
    P1 = P2; P2 = Pq;
    Z1 = Z2; Z2 = Zq;
    // ---- weights, k1 and T* of row r1 = q - 1 (T rows r1-1, r1, r1+1 are t0, t1, t2)
    const int r1 = q - 1;
    Weights<V> wA{zero, zero, zero, zero, zero, zero, zero, zero, zero};
    V k1 = zero;
    if (it >= 1 && r1 >= 0 && r1 < ny && !(walls && (r1 == 0 || r1 == ny - 1))) {
      const V div = fmadd(third, du1 + (vc2 - vc0), twelfth * ((du2 + du0) + (sv2 - sv0)));
      wA = weights(P1, U1, third * vc1, fmadd(cst<V>(-5.0), P1, zero - Z1 * div));
      k1 = apply(wA, t0, t1, t2);
    }
    s0 = s1; s1 = s2;
    s2 = nb(t1.c + k1);
    if (!walls && r1 == 0) s1 = affine(twoTbot, mone, s2);     // T*(-1) = 2 T_bot - T*(0)
    if (!walls && r1 == ny) s2 = affine(twoTtop, mone, s1);    // T*(ny) = 2 T_top - T*(ny-1)
    // ---- k2 and T_new of row r2 = q - 2 (T* rows r2-1 .. r2+1 are s0, s1, s2)
    const int r2 = q - 2;
    if (it >= 2 && r2 >= ya && r2 < yb && own) {
      V tn;
      if (walls && (r2 == 0 || r2 == ny - 1)) {
        tn = half * (r2 == 0 ? twoTbot : twoTtop);  // wall node: T_bot / T_top
      } else {
        tn = fmadd(half, k1B + apply(wB, s0, s1, s2), t0.c);
      }
      *reinterpret_cast<V*>(Tout + size_t(r2) * nx + x) = tn;
    }
    wB = wA;
    k1B = k1;
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
  // 8-row strips: 2304 warps on the 512 x 2048 column, two 8-warp CTAs per SM
  constexpr int kRows = 8, kWarps = 8, kAhead = 2;
  const int strips = (ny + kRows - 1) / kRows;
  if (precision == 1) {
    const dim3 grid((nx + own_columns<f2>() - 1) / own_columns<f2>(), (strips + kWarps - 1) / kWarps),
        block(32, kWarps);
    const EnergyArgs<float> a{nx, ny, wall_nodes, float(b / 4.0), float(2.0 * kappa / (3.0 * c_v)), float(R / c_v),
                              float(2.0 * T_bot), float(2.0 * T_top)};
    return launch_dependent(heun_strip_kernel<float, f2, kRows, kWarps, kAhead>, grid, block, 0, stream, a,
                            static_cast<const float*>(rho), static_cast<const float*>(ux),
                            static_cast<const float*>(uy), static_cast<const float*>(Tin),
                            static_cast<float*>(Tout));
  }
  const dim3 grid((nx + own_columns<double>() - 1) / own_columns<double>(), (strips + kWarps - 1) / kWarps),
      block(32, kWarps);
  const EnergyArgs<double> a{nx, ny, wall_nodes, b / 4.0, 2.0 * kappa / (3.0 * c_v), R / c_v, 2.0 * T_bot, 2.0 * T_top};
  return launch_dependent(heun_strip_kernel<double, double, kRows, kWarps, kAhead>, grid, block, 0, stream, a,
                          static_cast<const double*>(rho), static_cast<const double*>(ux),
                          static_cast<const double*>(uy), static_cast<const double*>(Tin),
                          static_cast<double*>(Tout));
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
