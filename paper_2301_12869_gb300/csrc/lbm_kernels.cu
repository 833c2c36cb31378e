// CUDA kernels of liblbm for sm_103a: the fused D2Q9 pseudopotential LBM step
// and its helpers. Method: arXiv 2301.12869, Sec. III (equations named inline).
//
// Fused step, one launch per time step. CTA b owns a band of nodes along x
// (width band_w, x periodic) and a strip of rows; it walks its rows bottom-up:
//
//   for each pulled row r (strip rows plus one halo row below and above):
//     1. the bulk-copy engine (cp.async.bulk, completion on an mbarrier) brings
//        the 9 source rows that pull streaming (Eq. LBE) needs for row r into a
//        shared-memory stage: plane i from row r - c_iy, or - where the link
//        crosses a wall - plane opp(i) of row r (halfway bounce-back); each
//        copy carries 16 bytes of x halo on both sides (periodic wrap);
//     2. every thread computes rho (Eq. Density) and psi (Eqs. EOS,
//        InteractionPotential) of row r for the band plus one x halo node on
//        each side into a 4-row psi ring;
//     3. one CTA barrier; the stage of row r-2 is refilled with row r-2+S;
//     4. row r-1 is collided: Shan-Chen force from the 3x3 psi stencil
//        (Eq. ShanChenForce), gravity (Eqs. Gravity_1/2), velocity
//        (Eq. Momentum), MRT with Li's forcing (Eqs. OperatorMRT, LiFS) in
//        moment space, and the 9 post-collision values are stored.
//
// The populations are stored as deviations g_i = f_i - w_i rho_ref, which
// turns every moment of the reference rest state into a constant that the
// collision handles exactly (w is the rest equilibrium of Eq.
// EquilibriumDistribution). Each CTA adds up the values it stores into one FP64
// partial; the next step's CTAs all finish that sum in the same fixed order,
// which gives sum_x rho of the populations they are about to stream - the
// same-step <rho> of Eq. Gravity_2, because streaming only permutes values.
#include "lbm_internal.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

namespace lbm {
namespace {

constexpr int kStages = 4;           // pipeline depth (rows of source planes in shared memory)
constexpr int kMaxThreads = 512;
constexpr long long kWaitCycles = 4000000000LL;   // bound of an mbarrier wait (about 2 s)

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

template <typename T>
struct PhysT {
  T rho_ref, RT, a, b4, twoOverG, G, G2;
  T s_e, s_vs, s_j, s_q, s_nu;      // Lambda entries
  T h_e, h_vs, h_j, h_q, h_nu;      // 1 - s/2 (diagonal of I - Lambda/2)
  T sig_e, sig_vs;                  // sigma/(tau_e - 1/2), sigma/(tau_varsigma - 1/2)
  T gx, gy;
  int form;
};

template <typename T>
PhysT<T> to_phys(const StepPhys& p) {
  PhysT<T> k;
  k.rho_ref = T(p.rho_ref);
  k.RT = T(p.RT);
  k.a = T(p.a);
  k.b4 = T(p.b / 4.0);
  k.twoOverG = T(2.0 / p.G);
  k.G = T(p.G);
  k.G2 = T(p.G * p.G);
  k.s_e = T(p.s_e); k.s_vs = T(p.s_vs); k.s_j = T(p.s_j); k.s_q = T(p.s_q); k.s_nu = T(p.s_nu);
  k.h_e = T(1.0 - 0.5 * p.s_e); k.h_vs = T(1.0 - 0.5 * p.s_vs); k.h_j = T(1.0 - 0.5 * p.s_j);
  k.h_q = T(1.0 - 0.5 * p.s_q); k.h_nu = T(1.0 - 0.5 * p.s_nu);
  k.sig_e = T(p.sig_e); k.sig_vs = T(p.sig_vs);
  k.gx = T(p.gx); k.gy = T(p.gy);
  k.form = p.form;
  return k;
}

// ---- PTX wrappers: mbarrier and the bulk-copy (TMA) engine
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity; gives up after kWaitCycles.
__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// ---- compensated accumulation of the per-thread mass partial
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ void add(double x) { s += x; }
  __device__ double value() const { return s; }
};
template <>
struct Acc<float> {  // two-sum (Knuth) pair: error-free to FP32 x FP32 precision
  float hi = 0.f, lo = 0.f;
  __device__ void add(float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
  }
  __device__ double value() const { return double(hi) + double(lo); }
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

// ---- per-node physics
// Eq. EOS (Carnahan-Starling) and Eq. InteractionPotential with c = 1, c_s^2 = 1/3.
template <typename T>
__device__ __forceinline__ T psi_of(T rho, const PhysT<T>& k, int& flag) {
  const T eta = k.b4 * rho;
  const T om = T(1) - eta;
  const T num = T(1) + eta * (T(1) + eta * (T(1) - eta));
  const T p = rho * k.RT * num / (om * om * om) - k.a * rho * rho;
  T rad = k.twoOverG * (p - rho * T(1.0 / 3.0));
  if (!(rad >= T(0))) {  // psi undefined (or NaN): non-physical state
    flag |= STATUS_NONPHYS;
    rad = T(0);
  }
  return sqrt(rad);
}

// Pull streaming (Eq. LBE) from a stage: slot i holds the source row of plane i at
// x offset -c_ix, or, where the link crosses a wall, plane opp(i) of the node's own
// row and column (halfway bounce-back: no x offset).
template <typename T>
__device__ __forceinline__ void pull(const T* st, int SW, int loc, bool lo_wall, bool hi_wall, T (&g)[9]) {
  g[0] = st[0 * SW + loc];
  g[1] = st[1 * SW + loc - 1];
  g[2] = st[2 * SW + loc];
  g[3] = st[3 * SW + loc + 1];
  g[4] = st[4 * SW + loc];
  g[5] = st[5 * SW + loc - (lo_wall ? 0 : 1)];
  g[6] = st[6 * SW + loc + (lo_wall ? 0 : 1)];
  g[7] = st[7 * SW + loc + (hi_wall ? 0 : 1)];
  g[8] = st[8 * SW + loc - (hi_wall ? 0 : 1)];
}

template <typename T>
__device__ __forceinline__ T sum9(const T (&g)[9]) {
  return ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
}

// One node: forces, velocity and the MRT collision with Li's forcing in moment
// space, on deviations g. (Sx, Sy) = sum_i w(|c_i|^2) psi(x + c_i) c_i (zero on wall
// rows), so F_int = -G psi S and |F_int|^2 / psi^2 = G^2 |S|^2.
template <typename T>
__device__ __forceinline__ void collide_node(const T (&g)[9], T psi_c, T Sx, T Sy, T dmean, const PhysT<T>& k,
                                             T (&o)[9], T& rho_o, T& ux_o, T& uy_o, int& flag) {
  // moments of g with the rows of Eq. MatrixMRT
  const T s13 = g[1] + g[3], s24 = g[2] + g[4];
  const T s57 = g[5] + g[7], s68 = g[6] + g[8];
  const T axis = s13 + s24, diag = s57 + s68;
  const T dr = (g[0] + axis) + diag;  // rho - rho_ref, Eq. Density
  const T rho = k.rho_ref + dr;
  const T d13 = g[1] - g[3], d24 = g[2] - g[4];
  const T d57 = g[5] - g[7], d68 = g[6] - g[8];
  const T jx = d13 + (d57 - d68);
  const T jy = d24 + (d57 + d68);
  // forces: Eq. ShanChenForce, Eqs. Gravity_1 / Gravity_2, F = F_int + F_g
  const T base = (k.form == 2) ? (dr - dmean) : rho;
  const T Fx = -k.G * psi_c * Sx + base * k.gx;
  const T Fy = -k.G * psi_c * Sy + base * k.gy;
  if (!(rho > T(0))) flag |= STATUS_NONPHYS;
  // Eq. Momentum: rho u = sum_i f_i c_i + F/2
  const T inv_rho = T(1) / rho;
  const T ux = (jx + T(0.5) * Fx) * inv_rho;
  const T uy = (jy + T(0.5) * Fy) * inv_rho;
  rho_o = rho;
  ux_o = ux;
  uy_o = uy;
  // non-conserved moments m = M g
  const T m_e = T(-4) * g[0] - axis + T(2) * diag;
  const T m_eps = T(4) * g[0] - T(2) * axis + diag;
  const T m_qx = T(-2) * d13 + (d57 - d68);
  const T m_qy = T(-2) * d24 + (d57 + d68);
  const T m_pxx = s13 - s24;
  const T m_pxy = s57 - s68;
  // equilibrium moments M f^eq of Eq. EquilibriumDistribution, less those of w rho_ref
  const T rux = rho * ux, ruy = rho * uy;
  const T ru2 = rux * ux + ruy * uy;
  const T meq_e = T(-2) * dr + T(3) * ru2;
  const T meq_eps = dr - T(3) * ru2;
  const T meq_pxx = rux * ux - ruy * uy;
  const T meq_pxy = rux * uy;
  // source vector of Eq. LiFS
  const T uF = ux * Fx + uy * Fy;
  const T ratio = k.G2 * (Sx * Sx + Sy * Sy);
  const T St_e = T(6) * uF + k.sig_e * ratio;
  const T St_eps = T(-6) * uF - k.sig_vs * ratio;
  const T St_pxx = T(2) * (ux * Fx - uy * Fy);
  const T St_pxy = ux * Fy + uy * Fx;
  // m* = m - Lambda (m - m_eq) + (I - Lambda/2) S~   (Eqs. LBE, OperatorMRT, LiFS)
  const T e_s = m_e - k.s_e * (m_e - meq_e) + k.h_e * St_e;
  const T eps_s = m_eps - k.s_vs * (m_eps - meq_eps) + k.h_vs * St_eps;
  const T jx_s = jx - k.s_j * (jx - rux) + k.h_j * Fx;
  const T qx_s = m_qx - k.s_q * (m_qx + rux) - k.h_q * Fx;
  const T jy_s = jy - k.s_j * (jy - ruy) + k.h_j * Fy;
  const T qy_s = m_qy - k.s_q * (m_qy + ruy) - k.h_q * Fy;
  const T pxx_s = m_pxx - k.s_nu * (m_pxx - meq_pxx) + k.h_nu * St_pxx;
  const T pxy_s = m_pxy - k.s_nu * (m_pxy - meq_pxy) + k.h_nu * St_pxy;
  // f* = M^-1 m* with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
  // (the rows of M are orthogonal)
  const T r9 = dr * T(1.0 / 9.0);
  const T e36 = e_s * T(1.0 / 36.0), eps36 = eps_s * T(1.0 / 36.0);
  const T jx6 = jx_s * T(1.0 / 6.0), qx12 = qx_s * T(1.0 / 12.0);
  const T jy6 = jy_s * T(1.0 / 6.0), qy12 = qy_s * T(1.0 / 12.0);
  const T pxx4 = pxx_s * T(0.25), pxy4 = pxy_s * T(0.25);
  const T b_ax = r9 - e36 - T(2) * eps36;
  const T b_dg = r9 + T(2) * e36 + eps36;
  const T a_x = jx6 - T(2) * qx12, a_y = jy6 - T(2) * qy12;
  const T d_x = jx6 + qx12, d_y = jy6 + qy12;
  o[0] = r9 - T(4) * e36 + T(4) * eps36;
  o[1] = b_ax + a_x + pxx4;
  o[2] = b_ax + a_y - pxx4;
  o[3] = b_ax - a_x + pxx4;
  o[4] = b_ax - a_y - pxx4;
  o[5] = b_dg + d_x + d_y + pxy4;
  o[6] = b_dg - d_x + d_y - pxy4;
  o[7] = b_dg - d_x - d_y + pxy4;
  o[8] = b_dg + d_x - d_y - pxy4;
}

template <typename T>
__host__ __device__ constexpr int halo_of() { return int(16 / sizeof(T)); }

template <typename T>
__host__ __device__ size_t step_smem(int band_w) {
  const size_t SW = size_t(band_w) + 2 * halo_of<T>();
  size_t off = (size_t(kStages) * 9 * SW + 4 * (size_t(band_w) + 2)) * sizeof(T);
  off = (off + 15) & ~size_t(15);
  return off + kStages * sizeof(uint64_t) + 33 * sizeof(double);
}

// ---- the fused step (MODE_STEP) / moments export (MODE_MOMENTS)
template <typename T, int MODE>
__global__ void __launch_bounds__(kMaxThreads, 1) step_kernel(const StepTiling tl, const PhysT<T> k, const StepIO io) {
  constexpr int H = halo_of<T>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int BW = tl.band_w;
  const int SW = BW + 2 * H;
  const int RW = BW + 2;
  T* stage = reinterpret_cast<T*>(smem_raw);
  T* ring = stage + size_t(kStages) * 9 * SW;
  size_t off = (size_t(kStages) * 9 * SW + 4 * size_t(RW)) * sizeof(T);
  off = (off + 15) & ~size_t(15);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + off);
  double* red = reinterpret_cast<double*>(smem_raw + off + kStages * sizeof(uint64_t));

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nx = tl.nx, ny = tl.ny;
  const int band = blockIdx.x % tl.nbands, strip = blockIdx.x / tl.nbands;
  const int xa = band * BW, xb = min(xa + BW, nx), w = xb - xa;
  const int ya = strip * tl.strip_h, yb = min(ya + tl.strip_h, ny);

  // <rho> - rho_ref of Eq. Gravity_2: the previous step's partials, finished in a fixed order
  T dmean = T(0);
  if (k.form == 2) {
    if (warp == 0) {
      const double s = warp_sum_partials(io.part_in, io.npart_in);
      if (lane == 0) red[32] = s;
    }
    __syncthreads();
    dmean = T(red[32] / (double(nx) * double(ny)));
  }
  if (ya >= yb || w <= 0) {  // empty tile (uniform across the CTA)
    if (MODE == MODE_STEP && tid == 0) io.part_out[blockIdx.x] = 0.0;
    return;
  }

  const int r_lo = max(ya - 1, 0), r_hi = min(yb, ny - 1);
  const int nrows = r_hi - r_lo + 1;
  const T* fin = static_cast<const T*>(io.fin);
  T* fout = static_cast<T*>(io.fout);
  const uint32_t row_bytes = uint32_t(9 * (w + 2 * H) * sizeof(T));
  const int xl = (xa >= H) ? xa - H : nx - H;   // left halo source (periodic)
  const int xr = (xb + H <= nx) ? xb : 0;       // right halo source (periodic)

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // producer: row kk of the walk into stage kk % kStages
  auto issue = [&](int kk) {
    const int r = r_lo + kk, s = kk % kStages;
    mbar_expect_tx(&full[s], row_bytes);
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
      int plane = i, row = r - cy_of(i);
      if (row < 0 || row >= ny) {
        plane = opp_of(i);
        row = r;
      }
      const T* src = fin + (size_t(plane) * ny + row) * size_t(nx);
      T* dst = stage + (size_t(s) * 9 + i) * SW;
      bulk_g2s(dst, src + xl, H * sizeof(T), &full[s]);
      bulk_g2s(dst + H, src + xa, uint32_t(w * sizeof(T)), &full[s]);
      bulk_g2s(dst + H + w, src + xr, H * sizeof(T), &full[s]);
    }
  };
  int issued = 0;
  if (tid == 0) {
    for (; issued < min(kStages, nrows); ++issued) issue(issued);
  }

  int flag = 0;
  Acc<T> acc;

  auto collide_row = [&](int y, int s) {
    const T* st = stage + size_t(s) * 9 * SW;
    const bool lo_wall = (y == 0), hi_wall = (y == ny - 1);
    const bool interior = !lo_wall && !hi_wall;
    const T* pc = ring + (y & 3) * RW;
    const T* pn = ring + ((y + 1) & 3) * RW;
    const T* ps = ring + ((y - 1) & 3) * RW;
    for (int j = 1 + tid; j <= w; j += nthr) {
      T g[9];
      pull(st, SW, j - 1 + H, lo_wall, hi_wall, g);
      T Sx = T(0), Sy = T(0);
      if (interior) {  // Eq. ShanChenForce stencil: w(1) = 1/3, w(2) = 1/12
        const T E = pc[j + 1], Wt = pc[j - 1], N = pn[j], S = ps[j];
        const T NE = pn[j + 1], NW = pn[j - 1], SE = ps[j + 1], SWt = ps[j - 1];
        Sx = T(1.0 / 3.0) * (E - Wt) + T(1.0 / 12.0) * ((NE - NW) + (SE - SWt));
        Sy = T(1.0 / 3.0) * (N - S) + T(1.0 / 12.0) * ((NE + NW) - (SE + SWt));
      }
      T o[9], rho, ux, uy;
      collide_node<T>(g, pc[j], Sx, Sy, dmean, k, o, rho, ux, uy, flag);
      const size_t x = size_t(xa + j - 1);
      if (MODE == MODE_STEP) {
        const size_t plane = size_t(ny) * nx;
        T* dst = fout + size_t(y) * nx + x;
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[i * plane] = o[i];
        acc.add(sum9(o));
      } else {
        const size_t idx = size_t(y) * nx + x;
        if (io.rho_out) io.rho_out[idx] = double(rho);
        if (io.ux_out) io.ux_out[idx] = double(ux);
        if (io.uy_out) io.uy_out[idx] = double(uy);
      }
    }
  };

  bool failed = false;
  int kk = 0;
  for (; kk < nrows; ++kk) {
    const int r = r_lo + kk, s = kk % kStages;
    const bool ok = mbar_wait_bounded(&full[s], uint32_t((kk / kStages) & 1));
    if (ok) {
      const T* st = stage + size_t(s) * 9 * SW;
      const bool lo_wall = (r == 0), hi_wall = (r == ny - 1);
      T* pr = ring + (r & 3) * RW;
      for (int j = tid; j < w + 2; j += nthr) {  // x = xa - 1 + j
        T g[9];
        pull(st, SW, j - 1 + H, lo_wall, hi_wall, g);
        pr[j] = psi_of<T>(k.rho_ref + sum9(g), k, flag);
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid == 0 && kk >= 2 && issued < nrows) issue(issued++);
    if (kk >= 1 && r - 1 >= ya) collide_row(r - 1, (kk - 1) % kStages);
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(io.status, STATUS_TIMEOUT);
      // let the copies still in flight land before the CTA's shared memory is released
      for (int q = kk; q < issued; ++q)
        (void)mbar_wait_bounded(&full[q % kStages], uint32_t((q / kStages) & 1), kWaitCycles / 8);
    }
    return;
  }
  if (r_hi == yb - 1) collide_row(yb - 1, (nrows - 1) % kStages);  // top wall row (yb == ny)

  if (__syncthreads_or(flag) && tid == 0) atomicOr(io.status, STATUS_NONPHYS);
  if (MODE == MODE_STEP) {
    const double v = warp_sum(acc.value());
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
      const int nw = (nthr + 31) >> 5;
      const double t = warp_sum(lane < nw ? red[lane] : 0.0);
      if (lane == 0) io.part_out[blockIdx.x] = t;
    }
  }
}

// ---- initial state g_i = f_i^eq(rho0, 0) - w_i rho_ref = w_i (rho0 - rho_ref)
template <typename T>
__global__ void init_kernel(const double* __restrict__ rho0, T* __restrict__ f, int nx, int ny, double rho_ref) {
  const size_t n = size_t(nx) * ny;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < n; q += size_t(gridDim.x) * blockDim.x) {
    const double d = rho0[q] - rho_ref;
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i * n + q] = T(w_of(i) * d);
  }
}

// ---- FP64 partial sums of sum_i g_i: block b covers nodes [b*chunk, (b+1)*chunk)
template <typename T>
__global__ void partials_kernel(const T* __restrict__ f, int nx, int ny, double* __restrict__ part) {
  __shared__ double red[32];
  const size_t n = size_t(nx) * ny;
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t q0 = blockIdx.x * chunk, q1 = min(n, q0 + chunk);
  double s = 0.0;
  for (size_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    double node = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) node += double(f[i * n + q]);
    s += node;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    const double t = warp_sum(threadIdx.x < nw ? red[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(const double* part, int npart, double* out) {
  const double s = warp_sum_partials(part, npart);
  if (threadIdx.x == 0) out[0] = s;
}

// one population plane: out[q] = plane[q] + add  /  plane[q] = in[q] - sub
template <typename T>
__global__ void plane_to_double_kernel(const T* __restrict__ plane, double* __restrict__ out, size_t n, double add) {
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < n; q += size_t(gridDim.x) * blockDim.x)
    out[q] = double(plane[q]) + add;
}

template <typename T>
__global__ void plane_from_double_kernel(const double* __restrict__ in, T* __restrict__ plane, size_t n, double sub) {
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < n; q += size_t(gridDim.x) * blockDim.x)
    plane[q] = T(in[q] - sub);
}

// non-negative doubles order like their bit patterns; NaN (0x7ff8...) sorts above +inf
__device__ __forceinline__ void atomic_max_nonneg(double* out, double v) {
  if (v != v) v = __longlong_as_double(0x7ff8000000000000LL);
  atomicMax(reinterpret_cast<unsigned long long*>(out), static_cast<unsigned long long>(__double_as_longlong(v)));
}

__global__ void max_abs_diff_kernel(const double* a, const double* b, size_t n, double* out) {
  double m = 0.0;
  bool nan = false;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < n; q += size_t(gridDim.x) * blockDim.x) {
    const double d = fabs(a[q] - (b ? b[q] : 0.0));
    nan |= (d != d);
    m = fmax(m, d);
  }
  if (nan) m = __longlong_as_double(0x7ff8000000000000LL);
  atomic_max_nonneg(out, m);
}

__global__ void max_speed_kernel(const double* ux, const double* uy, size_t n, double* out) {
  double m = 0.0;
  bool nan = false;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < n; q += size_t(gridDim.x) * blockDim.x) {
    const double s = sqrt(ux[q] * ux[q] + uy[q] * uy[q]);
    nan |= (s != s);
    m = fmax(m, s);
  }
  if (nan) m = __longlong_as_double(0x7ff8000000000000LL);
  atomic_max_nonneg(out, m);
}

__global__ void row_means_kernel(const double* rho, int nx, int ny, double* rowmean) {
  __shared__ double red[32];
  const int y = blockIdx.x;
  double s = 0.0;
  for (int x = threadIdx.x; x < nx; x += blockDim.x) s += rho[size_t(y) * nx + x];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    const double t = warp_sum(threadIdx.x < nw ? red[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) rowmean[y] = t / nx;
  }
}

__global__ void profile_scan_kernel(const double* prof, int ny, double level, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double cross = __longlong_as_double(0x7ff8000000000000LL);
  double mx = prof[0], mn = prof[0];
  bool found = false;
  for (int y = 0; y < ny; ++y) {
    mx = fmax(mx, prof[y]);
    mn = fmin(mn, prof[y]);
    if (!found && y + 1 < ny) {
      const double lo = prof[y], hi = prof[y + 1];
      if ((lo - level) * (hi - level) <= 0.0 && lo != hi) {
        cross = y + (level - lo) / (hi - lo);
        found = true;
      }
    }
  }
  out[0] = cross;
  out[1] = mx;
  out[2] = mn;
}

template <typename T>
cudaError_t prepare_t() {
  cudaError_t e = cudaFuncSetAttribute(step_kernel<T, MODE_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(step_kernel<T, MODE_MOMENTS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              227 * 1024);
}

int grid_for(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return int(g);
}

}  // namespace

// ---------------------------------------------------------------- launch wrappers
int stages() { return kStages; }

size_t step_smem_bytes(int precision, int band_w, int /*threads*/) {
  return precision == 1 ? step_smem<float>(band_w) : step_smem<double>(band_w);
}

int step_max_ctas_per_sm(int precision, int mode, int threads, int smem_bytes) {
  int n = 0;
  const void* fn = nullptr;
  if (precision == 1)
    fn = mode == MODE_STEP ? (const void*)step_kernel<float, MODE_STEP> : (const void*)step_kernel<float, MODE_MOMENTS>;
  else
    fn = mode == MODE_STEP ? (const void*)step_kernel<double, MODE_STEP> : (const void*)step_kernel<double, MODE_MOMENTS>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem_bytes) != cudaSuccess) return 0;
  return n;
}

cudaError_t step_prepare(int precision) { return precision == 1 ? prepare_t<float>() : prepare_t<double>(); }

cudaError_t launch_step(int precision, int mode, const StepTiling& t, const StepPhys& ph, const StepIO& io,
                        cudaStream_t stream) {
  const dim3 grid(t.nbands * t.nstrips), block(t.threads);
  if (precision == 1) {
    const PhysT<float> k = to_phys<float>(ph);
    if (mode == MODE_STEP)
      step_kernel<float, MODE_STEP><<<grid, block, t.smem_bytes, stream>>>(t, k, io);
    else
      step_kernel<float, MODE_MOMENTS><<<grid, block, t.smem_bytes, stream>>>(t, k, io);
  } else {
    const PhysT<double> k = to_phys<double>(ph);
    if (mode == MODE_STEP)
      step_kernel<double, MODE_STEP><<<grid, block, t.smem_bytes, stream>>>(t, k, io);
    else
      step_kernel<double, MODE_MOMENTS><<<grid, block, t.smem_bytes, stream>>>(t, k, io);
  }
  return cudaGetLastError();
}

cudaError_t launch_init(int precision, const double* rho0, void* f, int nx, int ny, double rho_ref,
                        cudaStream_t stream) {
  const size_t n = size_t(nx) * ny;
  if (precision == 1)
    init_kernel<float><<<grid_for(n, 256), 256, 0, stream>>>(rho0, static_cast<float*>(f), nx, ny, rho_ref);
  else
    init_kernel<double><<<grid_for(n, 256), 256, 0, stream>>>(rho0, static_cast<double*>(f), nx, ny, rho_ref);
  return cudaGetLastError();
}

cudaError_t launch_partials(int precision, const void* f, int nx, int ny, double* part, int npart,
                            cudaStream_t stream) {
  if (precision == 1)
    partials_kernel<float><<<npart, 256, 0, stream>>>(static_cast<const float*>(f), nx, ny, part);
  else
    partials_kernel<double><<<npart, 256, 0, stream>>>(static_cast<const double*>(f), nx, ny, part);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* part, int npart, double* out, cudaStream_t stream) {
  sum_partials_kernel<<<1, 32, 0, stream>>>(part, npart, out);
  return cudaGetLastError();
}

cudaError_t launch_plane_to_double(int precision, const void* plane, double* out, size_t n, double add,
                                   cudaStream_t stream) {
  if (precision == 1)
    plane_to_double_kernel<float><<<grid_for(n, 256), 256, 0, stream>>>(static_cast<const float*>(plane), out, n, add);
  else
    plane_to_double_kernel<double><<<grid_for(n, 256), 256, 0, stream>>>(static_cast<const double*>(plane), out, n,
                                                                         add);
  return cudaGetLastError();
}

cudaError_t launch_plane_from_double(int precision, const double* in, void* plane, size_t n, double sub,
                                     cudaStream_t stream) {
  if (precision == 1)
    plane_from_double_kernel<float><<<grid_for(n, 256), 256, 0, stream>>>(in, static_cast<float*>(plane), n, sub);
  else
    plane_from_double_kernel<double><<<grid_for(n, 256), 256, 0, stream>>>(in, static_cast<double*>(plane), n, sub);
  return cudaGetLastError();
}

cudaError_t launch_max_abs_diff(const double* a, const double* b, size_t n, double* out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), stream);
  if (e != cudaSuccess) return e;
  max_abs_diff_kernel<<<grid_for(n, 256), 256, 0, stream>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t launch_max_speed(const double* ux, const double* uy, size_t n, double* out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), stream);
  if (e != cudaSuccess) return e;
  max_speed_kernel<<<grid_for(n, 256), 256, 0, stream>>>(ux, uy, n, out);
  return cudaGetLastError();
}

cudaError_t launch_row_means(const double* rho, int nx, int ny, double* rowmean, cudaStream_t stream) {
  row_means_kernel<<<ny, 256, 0, stream>>>(rho, nx, ny, rowmean);
  return cudaGetLastError();
}

cudaError_t launch_profile_scan(const double* rowmean, int ny, double level, double* out, cudaStream_t stream) {
  profile_scan_kernel<<<1, 32, 0, stream>>>(rowmean, ny, level, out);
  return cudaGetLastError();
}

}  // namespace lbm
