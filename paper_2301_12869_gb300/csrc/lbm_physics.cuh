// Per-node physics of the D2Q9 pseudopotential step, shared by the fused step kernels
// (lbm_kernels.cu) and the batched-column kernel (lbm_batch.cu). Method: arXiv
// 2301.12869, Sec. III; equations named inline. Written once for the value types of
// lbm_vec.cuh (float, double, and f2 = a pair of FP32 nodes).
#pragma once

#include "lbm_internal.h"
#include "lbm_vec.cuh"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

namespace lbm {

// ---- D2Q9 velocity set, Eq. VelocitySet: c_0 = (0,0); c_1..4 = (1,0),(0,1),(-1,0),(0,-1);
//      c_5..8 = (1,1),(-1,1),(-1,-1),(1,-1).
__host__ __device__ constexpr int cy_of(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
static_assert(opp_of(1) == 3 && opp_of(2) == 4 && opp_of(3) == 1 && opp_of(4) == 2, "opp");
static_assert(opp_of(5) == 7 && opp_of(6) == 8 && opp_of(7) == 5 && opp_of(8) == 6, "opp");
// lattice weights (text after Eq. EquilibriumDistribution)
__host__ __device__ constexpr double w_of(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

// Physical constants of a step in the value type V (a pair holds the same constant twice).
template <typename V>
struct PhysT {
  V rho_ref, RT, R, a, b4, twoOverG, negG, G2;
  V s_e, s_vs, s_j, s_q, s_nu;      // Lambda entries (general relaxation only)
  V h_e, h_vs, h_j, h_q, h_nu;      // 1 - s/2 (diagonal of I - Lambda/2)
  V sig_e, nsig_vs;                 // sigma/(tau_e - 1/2), -sigma/(tau_varsigma - 1/2)
  V gx, gy;
  int form;
};

template <typename V>
V host_value(double c);
template <>
inline float host_value<float>(double c) { return float(c); }
template <>
inline double host_value<double>(double c) { return c; }
template <>
inline f2 host_value<f2>(double c) {  // {c, c}: the low word is the first component
  const float x = float(c);
  uint32_t b;
  memcpy(&b, &x, 4);
  return f2{uint64_t(b) | (uint64_t(b) << 32)};
}

template <typename V>
PhysT<V> to_phys(const StepPhys& p) {
  auto c = [](double x) { return host_value<V>(x); };
  PhysT<V> k;
  k.rho_ref = c(p.rho_ref);
  k.RT = c(p.RT);
  k.R = c(p.R);
  k.a = c(p.a);
  k.b4 = c(p.b / 4.0);
  k.twoOverG = c(2.0 / p.G);
  k.negG = c(-p.G);
  k.G2 = c(p.G * p.G);
  k.s_e = c(p.s_e); k.s_vs = c(p.s_vs); k.s_j = c(p.s_j); k.s_q = c(p.s_q); k.s_nu = c(p.s_nu);
  k.h_e = c(1.0 - 0.5 * p.s_e); k.h_vs = c(1.0 - 0.5 * p.s_vs); k.h_j = c(1.0 - 0.5 * p.s_j);
  k.h_q = c(1.0 - 0.5 * p.s_q); k.h_nu = c(1.0 - 0.5 * p.s_nu);
  k.sig_e = c(p.sig_e); k.nsig_vs = c(-p.sig_vs);
  k.gx = c(p.gx); k.gy = c(p.gy);
  k.form = p.form;
  return k;
}

// ---- compensated accumulation of the per-thread mass partial
template <typename V>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ void add(double x, int = 0) { s += x; }
  __device__ void add9(const double (&v)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) s += v[i];
  }
  __device__ double value() const { return s; }
};
template <typename V>
struct Acc {  // float or f2: two-sum (Knuth) pairs, error-free to FP32 x FP32 precision
  // (add9 adds every value; the default FP32 step kernel adds each node's FP32 sum of its
  // stored values once: a rounding of 2^-24 relative per node, which can add up coherently
  // over identical nodes - at most ~1e-8 of <rho>, a force change of |g| 1e-8 <rho>)
  V hi[3] = {cst<V>(0.0), cst<V>(0.0), cst<V>(0.0)};
  V lo[3] = {cst<V>(0.0), cst<V>(0.0), cst<V>(0.0)};
  __device__ void add(V x, int c = 0) {
    const V s = hi[c] + x;
    const V bp = s - hi[c];
    const V err = (hi[c] - (s - bp)) + (x - bp);
    hi[c] = s;
    lo[c] = lo[c] + err;
  }
  // every value separately, so the total is the sum of the stored values to ~2^-48
  // relative (a sum formed first in FP32 would round identical nodes identically, and
  // those errors add up coherently over uniform regions); three independent chains keep
  // the dependency path short
  __device__ void add9(const V (&v)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) add(v[i], i % 3);
  }
  __device__ double value() const {
    return (hsum(hi[0]) + hsum(lo[0])) + (hsum(hi[1]) + hsum(lo[1])) + (hsum(hi[2]) + hsum(lo[2]));
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// Sum of part[0..n) in a fixed order (lane-strided, then a butterfly), by one warp.
// Every lane returns the same bits; every caller that uses this order gets the same value.
__device__ __forceinline__ double warp_sum_partials(const double* part, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int q = lane; q < n; q += 32) s += part[q];
  return warp_sum(s);
}

// ---- per-node physics, written once for float, double and f2

// Eq. EOS (Carnahan-Starling) and Eq. InteractionPotential with c = 1, c_s^2 = 1/3.
template <typename V>
__device__ __forceinline__ V psi_of(V rho, V RT, const PhysT<V>& k, int& flag) {
  const V one = cst<V>(1.0);
  const V eta = k.b4 * rho;
  const V om = one - eta;
  const V num = fmadd(eta, fmadd(eta, om, one), one);  // 1 + eta + eta^2 - eta^3
  const V p = fast_div(rho * RT * num, om * om * om) - k.a * rho * rho;
  bool bad = false;
  const V psi = sqrt_checked(k.twoOverG * fmadd(rho, cst<V>(-1.0 / 3.0), p), bad);
  if (bad) flag |= STATUS_NONPHYS;  // 2 (p_EOS - rho/3)/G < 0 or NaN: psi undefined
  return psi;
}
// isothermal: R T of the parameters
template <typename V>
__device__ __forceinline__ V psi_of(V rho, const PhysT<V>& k, int& flag) {
  return psi_of(rho, k.RT, k, flag);
}

// Zou-He wet-node wall (Sec. III: no-slip condition of Zou and He on the solid walls) at a
// node of row 0 (bottom) or ny - 1: the populations entering from outside the lattice
// (bottom: i = 2, 5, 6; top: i = 4, 7, 8) are set so that the velocity of Eq. Momentum,
// half force included, vanishes, with the normal population's non-equilibrium part
// bounced back. F_int = 0 on wall rows, so F = F_g; its rho dependence makes the wall
// density the solution of rho (1 + s g_y/2) = K (+ s <rho> g_y/2 for Eq. Gravity_2), with
// s = +1 (bottom) / -1 (top) and K the sum of the known populations counted as the moment
// condition requires. Works on deviations g_i = f_i - w_i rho_ref (the weights of the
// formulas cancel pairwise); dmean = <rho> - rho_ref.
template <typename V>
__device__ __forceinline__ void zou_he(V (&g)[9], bool bottom, V dmean, const PhysT<V>& k) {
  const V half = cst<V>(0.5), quarter = cst<V>(0.25), one = cst<V>(1.0);
  const V s_half_gy = bottom ? half * k.gy : cst<V>(-0.5) * k.gy;  // s g_y / 2
  const V Kg = bottom ? (g[0] + g[1] + g[3]) + cst<V>(2.0) * (g[4] + g[7] + g[8])
                      : (g[0] + g[1] + g[3]) + cst<V>(2.0) * (g[2] + g[5] + g[6]);
  // rho - rho_ref: form 1 (Kg - s gy/2 rho_ref)/(1 + s gy/2); form 2 (Kg + s gy/2 dmean)/(1 + s gy/2)
  const V num = (k.form == 2) ? fmadd(s_half_gy, dmean, Kg) : Kg - s_half_gy * k.rho_ref;
  const V dr = fast_div(num, one + s_half_gy);
  const V base = (k.form == 2) ? (dr - dmean) : (k.rho_ref + dr);
  const V Fx = base * k.gx, Fy = base * k.gy;
  const V d13 = half * (g[1] - g[3]);
  if (bottom) {
    g[2] = g[4];
    g[5] = g[7] - d13 - quarter * (Fx + Fy);
    g[6] = g[8] + d13 + quarter * (Fx - Fy);
  } else {
    g[4] = g[2];
    g[7] = g[5] + d13 + quarter * (Fx + Fy);
    g[8] = g[6] - d13 + quarter * (Fy - Fx);
  }
}

template <typename V>
__device__ __forceinline__ V sum9(const V (&g)[9]) {
  return ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
}

// One node (or a pair): forces, velocity and the MRT collision with Li's forcing in
// moment space, on deviations g. (Sx, Sy) = sum_i w(|c_i|^2) psi(x + c_i) c_i (zero on
// wall rows), so F_int = -G psi S and |F_int|^2 / psi^2 = G^2 |S|^2.
template <typename V, bool UNIT>
__device__ __forceinline__ void collide_node(const V (&g)[9], V psi_c, V Sx, V Sy, V dmean, const PhysT<V>& k,
                                             V (&o)[9], V& rho_o, V& ux_o, V& uy_o, int& flag) {
  const V half = cst<V>(0.5);
  // moments of g with the rows of Eq. MatrixMRT
  const V s13 = g[1] + g[3], s24 = g[2] + g[4];
  const V s57 = g[5] + g[7], s68 = g[6] + g[8];
  const V axis = s13 + s24, diag = s57 + s68;
  const V dr = (g[0] + axis) + diag;  // rho - rho_ref, Eq. Density
  const V rho = k.rho_ref + dr;
  const V d13 = g[1] - g[3], d24 = g[2] - g[4];
  const V d57 = g[5] - g[7], d68 = g[6] - g[8];
  const V jx = d13 + (d57 - d68);
  const V jy = d24 + (d57 + d68);
  // forces: Eq. ShanChenForce, Eqs. Gravity_1 / Gravity_2, F = F_int + F_g
  const V base = (k.form == 2) ? (dr - dmean) : rho;
  const V nGpsi = k.negG * psi_c;
  const V Fx = fmadd(nGpsi, Sx, base * k.gx);
  const V Fy = fmadd(nGpsi, Sy, base * k.gy);
  if (nonpositive(rho)) flag |= STATUS_NONPHYS;
  // Eq. Momentum: rho u = sum_i f_i c_i + F/2
  const V inv_rho = fast_div(cst<V>(1.0), rho);
  const V ux = fmadd(half, Fx, jx) * inv_rho;
  const V uy = fmadd(half, Fy, jy) * inv_rho;
  rho_o = rho;
  ux_o = ux;
  uy_o = uy;
  // equilibrium moments M f^eq of Eq. EquilibriumDistribution, less those of w rho_ref
  const V rux = rho * ux, ruy = rho * uy;
  const V ru2 = fmadd(rux, ux, ruy * uy);
  const V meq_e = fmadd(cst<V>(3.0), ru2, cst<V>(-2.0) * dr);
  const V meq_eps = fmadd(cst<V>(-3.0), ru2, dr);
  const V rvv = ruy * uy;
  const V meq_pxx = fmadd(rux, ux, cst<V>(-1.0) * rvv);
  const V meq_pxy = rux * uy;
  // source vector of Eq. LiFS
  const V uyFy = uy * Fy;
  const V uF = fmadd(ux, Fx, uyFy);
  const V ratio = k.G2 * fmadd(Sx, Sx, Sy * Sy);
  const V St_e = fmadd(cst<V>(6.0), uF, k.sig_e * ratio);
  const V St_eps = fmadd(cst<V>(-6.0), uF, k.nsig_vs * ratio);
  const V St_pxx = fmadd(cst<V>(-4.0), uyFy, uF + uF);  // 2 (ux Fx - uy Fy)
  const V St_pxy = fmadd(ux, Fy, uy * Fx);
  // m* = m - Lambda (m - m_eq) + (I - Lambda/2) S~   (Eqs. LBE, OperatorMRT, LiFS),
  // then f* = M^-1 m* with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
  // (the rows of M are orthogonal). a_* / d_* are the axis / diagonal combinations
  // (j/6 - 2 q/12) and (j/6 + q/12) of the back-transform.
  V e_s, eps_s, pxx_s, pxy_s, a_x, a_y, d_x, d_y;
  if constexpr (UNIT) {
    // every tau = 1 (Lambda = I): m* = m_eq + S~/2; then q* = -j* exactly, so
    // a = j*/3 and d = j*/12
    e_s = fmadd(half, St_e, meq_e);
    eps_s = fmadd(half, St_eps, meq_eps);
    pxx_s = fmadd(half, St_pxx, meq_pxx);
    pxy_s = fmadd(half, St_pxy, meq_pxy);
    const V jx_s = fmadd(half, Fx, rux);
    const V jy_s = fmadd(half, Fy, ruy);
    a_x = jx_s * cst<V>(1.0 / 3.0);
    a_y = jy_s * cst<V>(1.0 / 3.0);
    d_x = jx_s * cst<V>(1.0 / 12.0);
    d_y = jy_s * cst<V>(1.0 / 12.0);
  } else {
    const V two = cst<V>(2.0);
    const V m_e = fmadd(cst<V>(-4.0), g[0], fmadd(two, diag, cst<V>(-1.0) * axis));
    const V m_eps = fmadd(cst<V>(4.0), g[0], fmadd(cst<V>(-2.0), axis, diag));
    const V m_qx = fmadd(cst<V>(-2.0), d13, d57 - d68);
    const V m_qy = fmadd(cst<V>(-2.0), d24, d57 + d68);
    const V m_pxx = s13 - s24;
    const V m_pxy = s57 - s68;
    e_s = fmadd(k.h_e, St_e, fmadd(k.s_e, meq_e - m_e, m_e));
    eps_s = fmadd(k.h_vs, St_eps, fmadd(k.s_vs, meq_eps - m_eps, m_eps));
    const V jx_s = fmadd(k.h_j, Fx, fmadd(k.s_j, rux - jx, jx));
    const V jy_s = fmadd(k.h_j, Fy, fmadd(k.s_j, ruy - jy, jy));
    const V qx_s = fmadd(cst<V>(-1.0) * k.h_q, Fx, fmadd(k.s_q, cst<V>(-1.0) * rux - m_qx, m_qx));
    const V qy_s = fmadd(cst<V>(-1.0) * k.h_q, Fy, fmadd(k.s_q, cst<V>(-1.0) * ruy - m_qy, m_qy));
    pxx_s = fmadd(k.h_nu, St_pxx, fmadd(k.s_nu, meq_pxx - m_pxx, m_pxx));
    pxy_s = fmadd(k.h_nu, St_pxy, fmadd(k.s_nu, meq_pxy - m_pxy, m_pxy));
    const V j6 = cst<V>(1.0 / 6.0), q6 = cst<V>(1.0 / 6.0), q12 = cst<V>(1.0 / 12.0);
    a_x = fmadd(j6, jx_s, cst<V>(-1.0) * q6 * qx_s);
    a_y = fmadd(j6, jy_s, cst<V>(-1.0) * q6 * qy_s);
    d_x = fmadd(j6, jx_s, q12 * qx_s);
    d_y = fmadd(j6, jy_s, q12 * qy_s);
  }
  const V r9 = dr * cst<V>(1.0 / 9.0);
  const V e36 = e_s * cst<V>(1.0 / 36.0), eps36 = eps_s * cst<V>(1.0 / 36.0);
  const V pxx4 = pxx_s * cst<V>(0.25), pxy4 = pxy_s * cst<V>(0.25);
  const V b_ax = fmadd(cst<V>(-2.0), eps36, r9 - e36);  // r/9 - e/36 - 2 eps/36
  const V b_dg = fmadd(cst<V>(2.0), e36, r9 + eps36);   // r/9 + 2 e/36 + eps/36
  o[0] = fmadd(cst<V>(4.0), eps36 - e36, r9);
  const V t_p = b_ax + pxx4, t_m = b_ax - pxx4;
  o[1] = t_p + a_x;
  o[3] = t_p - a_x;
  o[2] = t_m + a_y;
  o[4] = t_m - a_y;
  const V u_p = b_dg + pxy4, u_m = b_dg - pxy4;
  const V dxy = d_x + d_y, dyx = d_y - d_x;
  o[5] = u_p + dxy;
  o[7] = u_p - dxy;
  o[6] = u_m + dyx;
  o[8] = u_m - dyx;
}

}  // namespace lbm
