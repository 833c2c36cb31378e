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
  T R, b4, c_v, kappa, twoTbot, twoTtop, inv_cv;
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
// neighbours from a window of rows in registers: walking up, input row q (T, u, v and the
// two rho coefficients) is loaded, k1 and T* = T + k1 are formed for row q - 1, and k2 and
// T_new = T + (k1 + k2)/2 for row q - 2. k1 is valid one column in from the edges, so the
// owned columns have T* on both sides. Each input value is loaded once per warp (plus
// the halo columns and 2 + 2 halo rows of the strip).
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

// Right-hand side of Eq. Energy_Equation at the lane's node(s) of row r from T on rows
// r-1 (ts), r (tc), r+1 (tn), u, v on the same rows and the node's coefficients: the
// D2Q9-weighted differences with w = 1/9 (axes) and 1/36 (diagonals).
template <typename V>
__device__ __forceinline__ V rate_nb(const Nb<V>& ts, const Nb<V>& tc, const Nb<V>& tn, const Nb<V>& us,
                                     const Nb<V>& uc, const Nb<V>& un, const Nb<V>& vs, const Nb<V>& vc,
                                     const Nb<V>& vn, V ck, V cz) {
  const V w1 = cst<V>(1.0 / 9.0), w2 = cst<V>(1.0 / 36.0), three = cst<V>(3.0);
  const V gx = w1 * (tc.r - tc.l) + w2 * ((tn.r - tn.l) + (ts.r - ts.l));
  const V gy = w1 * (tn.c - ts.c) + w2 * ((tn.r + tn.l) - (ts.r + ts.l));
  const V lap = w1 * ((tc.r + tc.l) + (tn.c + ts.c)) + w2 * ((tn.r + tn.l) + (ts.r + ts.l)) - cst<V>(5.0 / 9.0) * tc.c;
  const V div = w1 * ((uc.r - uc.l) + (vn.c - vs.c)) + w2 * (((un.r - un.l) + (us.r - us.l)) + ((vn.r + vn.l) - (vs.r + vs.l)));
  return (ck * (cst<V>(6.0) * lap) - (uc.c * (three * gx) + vc.c * (three * gy))) - tc.c * cz * (three * div);
}

template <typename T, typename V, int ROWS, int WARPS, int AHEAD>
__global__ void __launch_bounds__(32 * WARPS) heun_strip_kernel(const EnergyArgs<T> a, const T* __restrict__ rho,
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
  const V twoTbot = splat<V>(a.twoTbot), twoTtop = splat<V>(a.twoTtop);
  const V kappa = splat<V>(a.kappa), c_v = splat<V>(a.c_v), R = splat<V>(a.R), b4 = splat<V>(a.b4);
  const V inv_cv = splat<V>(a.inv_cv);
  auto load = [&](const T* p, size_t n) { return *reinterpret_cast<const V*>(p + n); };
  // windows (row index relative to the input row q of the current iteration)
  Nb<V> t0{}, t1{}, t2{};            // T rows q-2, q-1, q
  Nb<V> u0{}, u1{}, u2{}, u3{};      // u rows q-3 .. q
  Nb<V> v0{}, v1{}, v2{}, v3{};      // v rows q-3 .. q
  Nb<V> s0{}, s1{}, s2{};            // T* rows q-3, q-2, q-1
  V ckA = zero, czA = zero, ckB = zero, czB = zero, ckC = zero, czC = zero;  // coefficients, rows q-2, q-1, q
  V k1a = zero, k1b = zero;          // k1 of rows q-2 (a) and q-1 (b)
  // Input rows are loaded AHEAD iterations before they are used (a ring of raw T, u, v,
  // rho in registers), so the global-load latency overlaps the work of the rows before.
  // A row outside the strip's range, or beyond the walls, loads nothing.
  const int q_first = ya - 2, q_last = yb + 1;
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
  for (int d = 0; d < AHEAD; ++d) fetch(q_first + d, ring[d]);
  for (int q = q_first; q <= q_last; ++q) {
    // ---- input row q: T, u, v with the wall ghosts, and the rho coefficients
    Raw in = ring[0];
#pragma unroll
    for (int d = 0; d + 1 < AHEAD; ++d) ring[d] = ring[d + 1];
    fetch(q + AHEAD, ring[AHEAD - 1]);
    V tq = in.t, uq = in.u, vq = in.v;
    V ckq = zero, czq = zero;
    const bool real = q >= 0 && q < ny;
    const bool ghost = !walls && (q == -1 || q == ny);
    if (real || ghost) {
      if (ghost) {  // T(-1) = 2 T_bot - T(0), u(-1) = -u(0); likewise above the top row
        tq = (q < 0 ? twoTbot : twoTtop) - tq;
        uq = zero - uq;
        vq = zero - vq;
      } else {
        const V rh = in.r;
        const V eta = b4 * rh;
        const V om = one - eta;
        ckq = kappa * recip(rh * c_v);
        czq = R * (one + eta * (one + eta * (one - eta))) * recip(om * om * om) * inv_cv;
      }
    }
    t0 = t1; t1 = t2; t2 = nb(tq);
    u0 = u1; u1 = u2; u2 = u3; u3 = nb(uq);
    v0 = v1; v1 = v2; v2 = v3; v3 = nb(vq);
    ckA = ckB; czA = czB; ckB = ckC; czB = czC; ckC = ckq; czC = czq;
    // ---- k1 and T* of row r1 = q - 1 (rows r1-1, r1, r1+1 are t0, t1, t2)
    const int r1 = q - 1;
    V k1 = zero;
    if (r1 >= 0 && r1 < ny && !(walls && (r1 == 0 || r1 == ny - 1)))
      k1 = rate_nb(t0, t1, t2, u1, u2, u3, v1, v2, v3, ckB, czB);
    s0 = s1; s1 = s2;
    s2 = nb(t1.c + k1);
    if (!walls && r1 == 0) s1 = affine(twoTbot, mone, s2);     // T*(-1) = 2 T_bot - T*(0)
    if (!walls && r1 == ny) s2 = affine(twoTtop, mone, s1);    // T*(ny) = 2 T_top - T*(ny-1)
    k1a = k1b;
    k1b = k1;
    // ---- k2 and T_new of row r2 = q - 2 (T* rows r2-1 .. r2+1 are s0, s1, s2)
    const int r2 = q - 2;
    if (r2 >= ya && r2 < yb && own) {
      V tn;
      if (walls && (r2 == 0 || r2 == ny - 1)) {
        tn = half * (r2 == 0 ? twoTbot : twoTtop);  // wall node: T_bot / T_top
      } else {
        const V k2 = rate_nb(s0, s1, s2, u0, u1, u2, v0, v1, v2, ckA, czA);
        tn = t0.c + half * (k1a + k2);
      }
      *reinterpret_cast<V*>(Tout + size_t(r2) * nx + x) = tn;
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
  if (precision == 1) {
    constexpr int kRows = 16, kWarps = 8, kAhead = 4;
    const int strips = (ny + kRows - 1) / kRows;
    const dim3 grid((nx + own_columns<f2>() - 1) / own_columns<f2>(), (strips + kWarps - 1) / kWarps),
        block(32, kWarps);
    const EnergyArgs<float> a{nx, ny, wall_nodes, float(R), float(b / 4.0), float(c_v), float(kappa),
                              float(2.0 * T_bot), float(2.0 * T_top), float(1.0 / c_v)};
    return launch_dependent(heun_strip_kernel<float, f2, kRows, kWarps, kAhead>, grid, block, 0, stream, a,
                            static_cast<const float*>(rho), static_cast<const float*>(ux),
                            static_cast<const float*>(uy), static_cast<const float*>(Tin),
                            static_cast<float*>(Tout));
  }
  constexpr int kRows = 16, kWarps = 8, kAhead = 4;
  const int strips = (ny + kRows - 1) / kRows;
  const dim3 grid((nx + own_columns<double>() - 1) / own_columns<double>(), (strips + kWarps - 1) / kWarps),
      block(32, kWarps);
  const EnergyArgs<double> a{nx, ny, wall_nodes, R, b / 4.0, c_v, kappa, 2.0 * T_bot, 2.0 * T_top, 1.0 / c_v};
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
