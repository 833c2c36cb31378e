// CUDA kernels of liblbm for sm_103a: the fused D2Q9 pseudopotential LBM step
// and its helpers. Method: arXiv 2301.12869, Sec. III (equations named inline).
//
// Fused step, one launch per time step. CTA b owns a band of nodes along x
// (x periodic) and a strip of rows, which it walks row by row (even strips upward,
// odd strips downward, so neighbouring strips read their shared halo rows together).
// For each pulled row r (the strip's rows plus one halo row below and above) the
// bulk-copy engine (cp.async.bulk, completion on an mbarrier) brings the 9 source
// rows that pull streaming (Eq. LBE) needs into a shared-memory stage: plane i from
// row r - c_iy, or - where the link crosses a wall - plane opp(i) of row r (halfway
// bounce-back), each with 16 bytes of periodic x halo on both sides. From the stage,
// rho (Eq. Density) and psi (Eqs. EOS, InteractionPotential) of row r are formed;
// once psi of rows r-2, r-1 and r is known, row r-1 is collided: the Shan-Chen force
// from the 3x3 psi stencil (Eq. ShanChenForce), gravity (Eqs. Gravity_1/2), the
// velocity (Eq. Momentum) and MRT with Li's forcing (Eqs. OperatorMRT, LiFS) in
// moment space, and its 9 post-collision values are stored.
//
// Default FP32 kernel (step_kernel_ws): one producer warp issues the copies into a
// ring of S stages; 8 consumer warps each own 64 nodes (a pair of neighbouring nodes
// per lane, evaluated with packed FP32x2 instructions, value type f2 of lbm_vec.cuh)
// and walk the rows without any CTA barrier: psi of the three rows around the
// collided row stays in registers, x neighbours come by warp shuffles, and a stage is
// refilled once every consumer warp has arrived on its `empty` mbarrier.
// Other tile variants (step_kernel, FP64 and the tuner's alternatives) keep psi in a
// 4-row shared ring and take one CTA barrier per row.
//
// The populations are stored as deviations g_i = f_i - w_i rho_ref, which
// turns every moment of the reference rest state into a constant that the
// collision handles exactly (w is the rest equilibrium of Eq.
// EquilibriumDistribution). Each CTA adds up the values it stores into one FP64
// partial; the next step's CTAs all finish that sum in the same fixed order,
// which gives sum_x rho of the populations they are about to stream - the
// same-step <rho> of Eq. Gravity_2, because streaming only permutes values.
#include "lbm_internal.h"
#include "lbm_physics.cuh"
#include "lbm_ptx.cuh"
#include "lbm_vec.cuh"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>

namespace lbm {
namespace {

constexpr int kStages = 4;           // pipeline depth (rows of source planes in shared memory)
// ---- PTX wrappers of the bulk-copy (TMA) engine; mbarrier helpers are in lbm_ptx.cuh
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

template <typename T>
__host__ __device__ constexpr int halo_of() { return int(16 / sizeof(T)); }

template <typename T, int BW>
__host__ __device__ constexpr size_t step_smem() {
  constexpr int SW = BW + 2 * halo_of<T>();
  constexpr size_t off = ((size_t(kStages) * 9 * SW + 4 * (size_t(BW) + 2)) * sizeof(T) + 15) & ~size_t(15);
  return off + kStages * sizeof(uint64_t) + 33 * sizeof(double);
}

// Pull streaming (Eq. LBE) from a stage: slot i holds the source row of plane i at
// x offset -c_ix, or, where the link crosses a wall, plane opp(i) of the node's own
// row and column (halfway bounce-back: no x offset). `loc` is the node's stage index.
template <int SW, typename T>
__device__ __forceinline__ void pull(const T* st, int loc, bool lo_wall, bool hi_wall, T (&g)[9]) {
  const T* p = st + loc;
  g[0] = p[0 * SW];
  g[1] = p[1 * SW - 1];
  g[2] = p[2 * SW];
  g[3] = p[3 * SW + 1];
  g[4] = p[4 * SW];
  g[5] = lo_wall ? p[5 * SW] : p[5 * SW - 1];
  g[6] = lo_wall ? p[6 * SW] : p[6 * SW + 1];
  g[7] = hi_wall ? p[7 * SW] : p[7 * SW + 1];
  g[8] = hi_wall ? p[8 * SW] : p[8 * SW - 1];
}

// The same for two neighbouring nodes at stage indices loc, loc + 1 (loc even): the
// unshifted planes are one 8-byte load, the shifted ones two 4-byte loads.
template <int SW>
__device__ __forceinline__ void pull(const float* st, int loc, bool lo_wall, bool hi_wall, f2 (&g)[9]) {
  const float* p = st + loc;
  auto pair = [&](int off) { return make_f2(p[off], p[off + 1]); };
  auto aligned = [&](int off) { return *reinterpret_cast<const f2*>(p + off); };
  if (!(lo_wall || hi_wall)) {  // interior row (uniform over a warp): no selects
    g[0] = aligned(0 * SW);
    g[1] = pair(1 * SW - 1);
    g[2] = aligned(2 * SW);
    g[3] = pair(3 * SW + 1);
    g[4] = aligned(4 * SW);
    g[5] = pair(5 * SW - 1);
    g[6] = pair(6 * SW + 1);
    g[7] = pair(7 * SW + 1);
    g[8] = pair(8 * SW - 1);
    return;
  }
  g[0] = aligned(0 * SW);
  g[1] = pair(1 * SW - 1);
  g[2] = aligned(2 * SW);
  g[3] = pair(3 * SW + 1);
  g[4] = aligned(4 * SW);
  g[5] = lo_wall ? aligned(5 * SW) : pair(5 * SW - 1);
  g[6] = lo_wall ? aligned(6 * SW) : pair(6 * SW + 1);
  g[7] = hi_wall ? aligned(7 * SW) : pair(7 * SW + 1);
  g[8] = hi_wall ? aligned(8 * SW) : pair(8 * SW - 1);
}

// value(s) of a field at p: one node, or an aligned pair of nodes
__device__ __forceinline__ float load_value(const float* p, float) { return *p; }
__device__ __forceinline__ double load_value(const double* p, double) { return *p; }
__device__ __forceinline__ f2 load_value(const float* p, f2) { return *reinterpret_cast<const f2*>(p); }
__device__ __forceinline__ int wrap_x(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

// ---- the fused step (MODE_STEP) / moments export (MODE_MOMENTS)
//
// Template parameters: storage type T, value type V (T, or f2 for pairs of FP32 nodes),
// mode, all-unit relaxation, band width BW (nodes along x per CTA), nodes per thread NPT
// (threads = BW / NPT; a thread owns NPT / width(V) values), CTAs per SM the launch
// bounds aim for; TH: thermal variant, psi uses R T(x) of the field io.Tfield (else R T),
// and a step also stores each node's rho, u for the energy equation; ZH: Zou-He wet-node
// walls on rows 0 and ny - 1 (else halfway bounce-back).
// CTA b: x band (b % nbands) of width tl.band_w (<= BW), strip (b / nbands) of
// tl.strip_h rows. Even strips walk their rows upward, odd strips downward, so two
// neighbouring strips reach their common halo rows at the same time (L2 reuse).
template <typename T, typename V, int MODE, bool UNIT, int BW, int NPT, int MINB, bool TH = false, bool ZH = false>
__global__ void __launch_bounds__(BW / NPT, MINB) step_kernel(const StepTiling tl, const PhysT<V> k, const StepIO io) {
  griddep_wait();  // launched as a dependent of the previous step: its state is complete
  griddep_launch_dependents();
  constexpr int NT = BW / NPT;
  constexpr int VW = VecTraits<V>::width;  // nodes per value
  constexpr int NU = NPT / VW;             // values per thread
  static_assert(NU * VW == NPT, "NPT must be a multiple of the value width");
  constexpr int H = halo_of<T>();
  constexpr int SW = BW + 2 * H;  // stage row: H halo, band, H halo
  constexpr int RW = BW + 2;      // psi ring row: one halo node each side
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* stage = reinterpret_cast<T*>(smem_raw);
  T* ring = stage + size_t(kStages) * 9 * SW;
  constexpr size_t off = ((size_t(kStages) * 9 * SW + 4 * size_t(RW)) * sizeof(T) + 15) & ~size_t(15);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + off);
  double* red = reinterpret_cast<double*>(smem_raw + off + kStages * sizeof(uint64_t));

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nx = tl.nx, ny = tl.ny;
  const int band = blockIdx.x % tl.nbands, strip = blockIdx.x / tl.nbands;
  const int xa = band * tl.band_w, xb = min(xa + tl.band_w, nx), w = xb - xa;
  const int ya = tl.y_begin + strip * tl.strip_h, yb = min(ya + tl.strip_h, tl.y_end);

  // <rho> - rho_ref of Eq. Gravity_2: the previous step's partials, finished in a fixed order
  V dmean = cst<V>(0.0);
  if (k.form == 2) {
    if (warp == 0) {
      const double s = warp_sum_partials(io.part_in, io.npart_in);
      if (lane == 0) red[32] = s;
    }
    __syncthreads();
    dmean = cst<V>(red[32] / tl.n_total);
  }
  if (ya >= yb || w <= 0) {  // empty tile (uniform across the CTA)
    if (MODE == MODE_STEP && tid == 0) io.part_out[blockIdx.x] = 0.0;
    return;
  }

  const int r_lo = max(ya - 1, tl.ylo), r_hi = min(yb, tl.yhi);
  const int nrows = r_hi - r_lo + 1;
  const bool up = (strip & 1) == 0;
  auto row_of = [&](int kk) { return up ? r_lo + kk : r_hi - kk; };
  const T* fin = static_cast<const T*>(io.fin);
  T* fout = static_cast<T*>(io.fout);
  const T* Tf = TH ? static_cast<const T*>(io.Tfield) : nullptr;  // thermal variant: local temperature

  // contiguous pieces of the periodic span [xa - H, xb + H): (global x, stage x, count)
  // piece 0 starts at the left halo; interior bands need only it
  int npc, g0, s0, n0, g1 = 0, s1 = 0, n1 = 0, g2 = 0, s2 = 0, n2 = 0;
  if (xa >= H) {
    g0 = xa - H; s0 = 0; n0 = w + H; npc = 1;
  } else {
    g0 = nx - H; s0 = 0; n0 = H;
    g1 = xa;     s1 = H; n1 = w; npc = 2;
  }
  if (xb + H <= nx) {
    if (npc == 1) n0 += H; else n1 += H;
  } else if (npc == 1) {
    g1 = 0; s1 = H + w; n1 = H; npc = 2;
  } else {
    g2 = 0; s2 = H + w; n2 = H; npc = 3;
  }
  const uint32_t row_bytes = uint32_t(9 * (w + 2 * H) * sizeof(T));

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // producer (all lanes of warp 0): walk row kk into stage kk % kStages, one copy per lane
  auto issue = [&](int kk) {
    const int q = row_of(kk), s = kk % kStages;
    if (lane == 0) mbar_expect_tx(&full[s], row_bytes);
    __syncwarp();
    for (int c = lane; c < 9 * npc; c += 32) {
      const int i = c / npc, pc = c - i * npc;
      int plane = i, row = q - cy_of(i);
      if (row < tl.ylo || row > tl.yhi) {
        plane = opp_of(i);
        row = q;
      }
      const int gx = pc == 0 ? g0 : (pc == 1 ? g1 : g2);
      const int sx = pc == 0 ? s0 : (pc == 1 ? s1 : s2);
      const int cnt = pc == 0 ? n0 : (pc == 1 ? n1 : n2);
      const T* src = fin + (size_t(plane) * ny + row) * size_t(nx) + gx;
      T* dst = stage + (size_t(s) * 9 + i) * SW + sx;
      bulk_g2s(dst, src, uint32_t(cnt * sizeof(T)), &full[s]);
    }
  };
  int issued = 0;  // meaningful in warp 0
  if (warp == 0) {
    for (; issued < min(kStages, nrows); ++issued) issue(issued);
  }

  int flag = 0;
  Acc<V> acc;

  auto collide_row = [&](int y, int s, auto full_band) {
    constexpr bool FULL = decltype(full_band)::value;  // w == BW: no per-node bounds checks
    const T* st = stage + size_t(s) * 9 * SW;
    const bool lo_wall = (y == tl.ylo), hi_wall = (y == tl.yhi);
    const bool interior = !lo_wall && !hi_wall;
    const T* pc = ring + (y & 3) * RW;
    const T* pn = ring + ((y + 1) & 3) * RW;
    const T* ps = ring + ((y - 1) & 3) * RW;
    T* dst_row = fout + size_t(y) * nx + xa;
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int j = 1 + VW * (tid + u * NT);  // first node x = xa + j - 1 of this value
      if (!FULL && j > w) continue;
      V g[9];
      pull<SW>(st, j - 1 + H, lo_wall, hi_wall, g);
      if constexpr (ZH) {
        if (!interior) zou_he(g, lo_wall, dmean, k);
      }
      V Sx = cst<V>(0.0), Sy = cst<V>(0.0), psi_c;
      const V c13 = cst<V>(1.0 / 3.0), c112 = cst<V>(1.0 / 12.0);
      if constexpr (VW == 1) {
        psi_c = pc[j];
        if (interior) {  // Eq. ShanChenForce stencil: w(1) = 1/3, w(2) = 1/12
          const V E = pc[j + 1], Wt = pc[j - 1], N = pn[j], S = ps[j];
          const V NE = pn[j + 1], NW = pn[j - 1], SE = ps[j + 1], SWt = ps[j - 1];
          Sx = fmadd(c13, E - Wt, c112 * ((NE - NW) + (SE - SWt)));
          Sy = fmadd(c13, N - S, c112 * ((NE + NW) - (SE + SWt)));
        }
      } else {
        // ring values j-1 .. j+2 of a row as two aligned pairs A = (j-1, j), B = (j+1, j+2):
        // for the node pair (j, j+1) west = A, east = B, centre = (A.hi, B.lo)
        const f2 Ac = *reinterpret_cast<const f2*>(pc + j - 1), Bc = *reinterpret_cast<const f2*>(pc + j + 1);
        psi_c = make_f2(hi(Ac), lo(Bc));
        if (interior) {
          const f2 An = *reinterpret_cast<const f2*>(pn + j - 1), Bn = *reinterpret_cast<const f2*>(pn + j + 1);
          const f2 As = *reinterpret_cast<const f2*>(ps + j - 1), Bs = *reinterpret_cast<const f2*>(ps + j + 1);
          const f2 Nc = make_f2(hi(An), lo(Bn)), Sc = make_f2(hi(As), lo(Bs));
          Sx = fmadd(c13, Bc - Ac, c112 * ((Bn - An) + (Bs - As)));
          Sy = fmadd(c13, Nc - Sc, c112 * ((Bn + An) - (Bs + As)));
        }
      }
      V o[9], rho, ux, uy;
      collide_node<V, UNIT>(g, psi_c, Sx, Sy, dmean, k, o, rho, ux, uy, flag);
      if (MODE == MODE_STEP) {
        const size_t plane = size_t(ny) * nx;
        T* dst = dst_row + (j - 1);
#pragma unroll
        for (int i = 0; i < 9; ++i) *reinterpret_cast<V*>(dst + i * plane) = o[i];
        acc.add9(o);
        if constexpr (TH) {  // this step's rho, u for the energy equation (Eq. Energy_Equation)
          static_assert(VW == 1, "thermal instantiations are one node per value");
          const size_t idx = size_t(y) * nx + xa + (j - 1);
          io.rho_out[idx] = double(rho);
          io.ux_out[idx] = double(ux);
          io.uy_out[idx] = double(uy);
        }
      } else {
        const size_t idx = size_t(y) * nx + xa + (j - 1);
        if constexpr (VW == 1) {
          if (io.rho_out) io.rho_out[idx] = double(rho);
          if (io.ux_out) io.ux_out[idx] = double(ux);
          if (io.uy_out) io.uy_out[idx] = double(uy);
        } else {
          if (io.rho_out) { io.rho_out[idx] = lo(rho); io.rho_out[idx + 1] = hi(rho); }
          if (io.ux_out) { io.ux_out[idx] = lo(ux); io.ux_out[idx + 1] = hi(ux); }
          if (io.uy_out) { io.uy_out[idx] = lo(uy); io.uy_out[idx + 1] = hi(uy); }
        }
      }
    }
  };

  bool failed = false;
  int kk = 0;
  for (; kk < nrows; ++kk) {
    const int q = row_of(kk), s = kk % kStages;
    const bool ok = mbar_wait_bounded(&full[s], uint32_t((kk / kStages) & 1));
    if (ok) {
      // rho and psi of pulled row q for the band and one halo node on each side
      const T* st = stage + size_t(s) * 9 * SW;
      const bool lo_wall = (q == tl.ylo), hi_wall = (q == tl.yhi);
      T* pr = ring + (q & 3) * RW;
      auto psi_row = [&](auto full_band) {
        constexpr bool FULL = decltype(full_band)::value;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int j = 1 + VW * (tid + u * NT);  // x = xa - 1 + j
          if (FULL || j <= w) {
            V g[9];
            pull<SW>(st, j - 1 + H, lo_wall, hi_wall, g);
            if constexpr (ZH) {
              if (lo_wall || hi_wall) zou_he(g, lo_wall, dmean, k);
            }
            const V RT = TH ? k.R * load_value(Tf + size_t(q) * nx + xa + j - 1, V{}) : k.RT;
            const V psi = psi_of<V>(k.rho_ref + sum9(g), RT, k, flag);
            if constexpr (VW == 1) {
              pr[j] = psi;
            } else {
              pr[j] = lo(psi);
              pr[j + 1] = hi(psi);
            }
          }
        }
      };
      if (w == BW)
        psi_row(std::true_type{});
      else
        psi_row(std::false_type{});
      if (warp == (NT / 32) - 1 && lane < 2) {  // the two halo nodes x = xa - 1 and x = xb
        const int j = lane ? w + 1 : 0;
        T g[9];
        pull<SW>(st, j - 1 + H, lo_wall, hi_wall, g);
        T rho_h;
        if constexpr (ZH) {
          V gv[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            if constexpr (VW == 1) gv[i] = g[i]; else gv[i] = make_f2(g[i], g[i]);
          }
          if (lo_wall || hi_wall) zou_he(gv, lo_wall, dmean, k);
          if constexpr (VW == 1) rho_h = sum9(gv); else rho_h = lo(sum9(gv));
        } else {
          rho_h = sum9(g);
        }
        const T Th = TH ? Tf[size_t(q) * nx + wrap_x(xa + j - 1, nx)] : T(0);
        V rho_v, T_v;
        if constexpr (VW == 1) {
          rho_v = rho_h;
          T_v = Th;
        } else {
          rho_v = make_f2(rho_h, rho_h);
          T_v = make_f2(Th, Th);
        }
        const V psi = psi_of<V>(k.rho_ref + rho_v, TH ? k.R * T_v : k.RT, k, flag);
        if constexpr (VW == 1) pr[j] = psi; else pr[j] = lo(psi);
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    // stage of walk row kk - 2 is free: every thread finished colliding it before the barrier
    if (warp == 0 && kk >= 2 && issued < nrows) issue(issued++);
    if (kk >= 1) {
      const int y = row_of(kk - 1);
      if (y >= ya && y < yb) {
        if (w == BW)
          collide_row(y, (kk - 1) % kStages, std::true_type{});
        else
          collide_row(y, (kk - 1) % kStages, std::false_type{});
      }
    }
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
  {  // last walk row: own only at a wall (no halo row beyond it), psi neighbours not needed
    const int y = row_of(nrows - 1);
    if (y >= ya && y < yb) collide_row(y, (nrows - 1) % kStages, std::false_type{});
  }

  if (__syncthreads_or(flag) && tid == 0) atomicOr(io.status, STATUS_NONPHYS);
  if (MODE == MODE_STEP) {
    const double v = warp_sum(acc.value());
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
      const double t = warp_sum(lane < NT / 32 ? red[lane] : 0.0);
      if (lane == 0) io.part_out[blockIdx.x] = t;
    }
  }
}

// ---- the fused step without CTA barriers in the row loop (FP32 node pairs)
//
// NWC consumer warps each own 64 nodes of the band (32 lanes x one pair) and walk the
// strip's rows on their own: psi of the three rows around the collided row stays in
// registers, x-neighbours come from the adjacent lanes by shuffles, and only the lanes at
// a warp's edges evaluate one extra psi value from the stage (which holds the whole band
// plus halos). One producer warp refills a stage once every consumer warp has arrived on
// that stage's `empty` mbarrier. Template: mode, all-unit relaxation, consumer warps,
// stages, CTAs per SM the launch bounds aim for, thermal (psi from R T(x)), Zou-He walls.
template <int NWC, int S>
__host__ __device__ constexpr size_t ws_smem() {
  constexpr int SW = 64 * NWC + 8;
  constexpr size_t off = (size_t(S) * 9 * SW * sizeof(float) + 15) & ~size_t(15);
  return off + 2 * S * sizeof(uint64_t) + (NWC + 2) * sizeof(double);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct PsiRow {  // psi at the left neighbour, the lane's own pair, the right neighbour
  float l;
  f2 c;
  float r;
};

template <int MODE, bool UNIT, int NWC, int S, int MINB, bool TH = false, bool ZH = false>
__global__ void __launch_bounds__((NWC + 1) * 32, MINB)
    step_kernel_ws(const StepTiling tl, const PhysT<f2> k, const StepIO io) {
  griddep_wait();  // launched as a dependent of the previous step: its state is complete
  griddep_launch_dependents();
  using T = float;
  using V = f2;
  constexpr int BW = 64 * NWC;
  constexpr int H = 4;
  constexpr int SW = BW + 2 * H;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage = reinterpret_cast<float*>(smem_raw);
  constexpr size_t off = (size_t(S) * 9 * SW * sizeof(float) + 15) & ~size_t(15);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + off);
  uint64_t* empty = full + S;
  double* red = reinterpret_cast<double*>(empty + S);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nx = tl.nx, ny = tl.ny;
  const int band = blockIdx.x % tl.nbands, strip = blockIdx.x / tl.nbands;
  const int xa = band * tl.band_w, xb = min(xa + tl.band_w, nx), w = xb - xa;
  const int ya = tl.y_begin + strip * tl.strip_h, yb = min(ya + tl.strip_h, tl.y_end);

  if (ya >= yb || w <= 0) {  // empty tile (uniform across the CTA)
    if (MODE == MODE_STEP && tid == 0) io.part_out[blockIdx.x] = 0.0;
    return;
  }

  const int r_lo = max(ya - 1, tl.ylo), r_hi = min(yb, tl.yhi);
  const int nrows = r_hi - r_lo + 1;
  const bool up = (strip & 1) == 0;
  auto row_of = [&](int kk) { return up ? r_lo + kk : r_hi - kk; };
  const T* fin = static_cast<const T*>(io.fin);
  T* fout = static_cast<T*>(io.fout);
  const T* Tf = TH ? static_cast<const T*>(io.Tfield) : nullptr;  // thermal variant: local temperature

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NWC);
    }
    fence_mbar_init();
  }
  __syncthreads();

  int flag = 0;
  V dmean = cst<V>(0.0);  // <rho> - rho_ref of Eq. Gravity_2 (consumer warps only)
  if (warp == NWC) {
    // ---------------- producer warp (it starts copying at once: it does not need <rho>)
    int npc, g0, s0, n0, g1 = 0, s1 = 0, n1 = 0, g2 = 0, s2 = 0, n2 = 0;
    if (xa >= H) {
      g0 = xa - H; s0 = 0; n0 = w + H; npc = 1;
    } else {
      g0 = nx - H; s0 = 0; n0 = H;
      g1 = xa;     s1 = H; n1 = w; npc = 2;
    }
    if (xb + H <= nx) {
      if (npc == 1) n0 += H; else n1 += H;
    } else if (npc == 1) {
      g1 = 0; s1 = H + w; n1 = H; npc = 2;
    } else {
      g2 = 0; s2 = H + w; n2 = H; npc = 3;
    }
    const uint32_t row_bytes = uint32_t(9 * (w + 2 * H) * sizeof(T));
    int kk = 0;
    for (; kk < nrows; ++kk) {
      const int s = kk % S;
      // the stage's previous row (kk - S) must be released by every consumer warp
      if (kk >= S && !__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], uint32_t(((kk / S) - 1) & 1)))) {
        flag |= STATUS_TIMEOUT;
        break;
      }
      const int q = row_of(kk);
      if (lane == 0) mbar_expect_tx(&full[s], row_bytes);
      __syncwarp();
      for (int c = lane; c < 9 * npc; c += 32) {
        const int i = c / npc, pc = c - i * npc;
        int plane = i, row = q - cy_of(i);
        if (row < tl.ylo || row > tl.yhi) {
          plane = opp_of(i);
          row = q;
        }
        const int gx = pc == 0 ? g0 : (pc == 1 ? g1 : g2);
        const int sx = pc == 0 ? s0 : (pc == 1 ? s1 : s2);
        const int cnt = pc == 0 ? n0 : (pc == 1 ? n1 : n2);
        const T* src = fin + (size_t(plane) * ny + row) * size_t(nx) + gx;
        T* dst = stage + (size_t(s) * 9 + i) * SW + sx;
        bulk_g2s(dst, src, uint32_t(cnt * sizeof(T)), &full[s]);
      }
    }
    if (flag && lane == 0) {
      // let the copies in flight land before the CTA's shared memory is released
      for (int q = max(0, kk - S); q < kk; ++q)
        (void)mbar_wait_bounded(&full[q % S], uint32_t((q / S) & 1), kWaitCycles / 8);
    }
  } else {
    // <rho> from the previous step's partials, finished in a fixed order by consumer warp 0
    // while the producer's first copies are in flight; named barrier 1 spans the consumers
    if (k.form == 2) {
      if (warp == 0) {
        const double s = warp_sum_partials(io.part_in, io.npart_in);
        if (lane == 0) red[NWC + 1] = s;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(NWC * 32) : "memory");
      dmean = cst<V>(red[NWC + 1] / tl.n_total);
    }
    // ---------------- consumer warp: nodes j, j+1 of the band (x = xa + j - 1)
    const int j = 1 + 64 * warp + 2 * lane;
    const bool active = j <= w;  // w is a multiple of 4, so j + 1 <= w too
    const bool need_l = active && lane == 0;
    const bool need_r = active && (lane == 31 || j + 2 > w);
    Acc<V> acc;
    PsiRow pm{0.f, cst<V>(0.0), 0.f}, p0 = pm, pp = pm;  // rows kk-2, kk-1, kk of the walk
    const V c13 = cst<V>(1.0 / 3.0), c112 = cst<V>(1.0 / 12.0);

    auto scalar_psi = [&](const T* st, int q, int jh, bool lo_wall, bool hi_wall) {
      T g[9];
      pull<SW>(st, jh - 1 + H, lo_wall, hi_wall, g);
      T rh;
      if constexpr (ZH) {
        V gv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) gv[i] = make_f2(g[i], g[i]);
        if (lo_wall || hi_wall) zou_he(gv, lo_wall, dmean, k);
        rh = lo(sum9(gv));
      } else {
        rh = sum9(g);
      }
      const T Th = TH ? Tf[size_t(q) * nx + wrap_x(xa + jh - 1, nx)] : T(0);
      const V RT = TH ? k.R * make_f2(Th, Th) : k.RT;
      return lo(psi_of<V>(k.rho_ref + make_f2(rh, rh), RT, k, flag));
    };
    // g: the pulled populations of row y, kept in registers since its psi pass
    auto collide = [&](int y, const V (&g)[9], const PsiRow& ps, const PsiRow& pc, const PsiRow& pn) {
      const bool lo_wall = (y == tl.ylo), hi_wall = (y == tl.yhi);
      V Sx = cst<V>(0.0), Sy = cst<V>(0.0);
      if (!lo_wall && !hi_wall) {  // Eq. ShanChenForce stencil: w(1) = 1/3, w(2) = 1/12
        // per row: west (psi(j-1), psi(j)), east (psi(j+1), psi(j+2)), centre (psi(j), psi(j+1))
        const V Wc = make_f2(pc.l, lo(pc.c)), Ec = make_f2(hi(pc.c), pc.r);
        const V Wn = make_f2(pn.l, lo(pn.c)), En = make_f2(hi(pn.c), pn.r);
        const V Ws = make_f2(ps.l, lo(ps.c)), Es = make_f2(hi(ps.c), ps.r);
        Sx = fmadd(c13, Ec - Wc, c112 * ((En - Wn) + (Es - Ws)));
        Sy = fmadd(c13, pn.c - ps.c, c112 * ((En + Wn) - (Es + Ws)));
      }
      V o[9], rho, ux, uy;
      collide_node<V, UNIT>(g, pc.c, Sx, Sy, dmean, k, o, rho, ux, uy, flag);
      const size_t node = size_t(y) * nx + xa + (j - 1);
      if (MODE == MODE_STEP) {
        const size_t plane = size_t(ny) * nx;
#pragma unroll
        for (int i = 0; i < 9; ++i) *reinterpret_cast<V*>(fout + node + i * plane) = o[i];
        acc.add(sum9(o));  // the node pair's stored values, summed in FP32 first
        if constexpr (TH) {
          // this step's rho, u for the energy equation (Eq. Energy_Equation) as floats: one
          // aligned pair per lane, no FP64 conversion (slow on GB300)
          *reinterpret_cast<V*>(io.rho32 + node) = rho;
          *reinterpret_cast<V*>(io.ux32 + node) = ux;
          *reinterpret_cast<V*>(io.uy32 + node) = uy;
        }
      } else {
        if (io.rho_out) { io.rho_out[node] = lo(rho); io.rho_out[node + 1] = hi(rho); }
        if (io.ux_out) { io.ux_out[node] = lo(ux); io.ux_out[node + 1] = hi(ux); }
        if (io.uy_out) { io.uy_out[node] = lo(uy); io.uy_out[node + 1] = hi(uy); }
      }
    };

    bool failed = false;
    V gp[9];  // pulled populations of walk row kk - 1
#pragma unroll
    for (int i = 0; i < 9; ++i) gp[i] = cst<V>(0.0);
    // two rows per iteration: the row state rotates by renaming instead of copies (the
    // Zou-He kernels, with their wall-row code, would spill)
    constexpr int kRowUnroll = ZH ? 1 : 2;
    // thermal variant: T of the next walk row is loaded one row ahead, so its latency hides
    // behind the current row's work
    const T* Tcol = TH ? Tf + xa + j - 1 : nullptr;
    V Tq = cst<V>(0.0);
    if constexpr (TH) {
      if (active) Tq = load_value(Tcol + size_t(row_of(0)) * nx, V{});
    }
#pragma unroll kRowUnroll
    for (int kk = 0; kk < nrows; ++kk) {
      const int q = row_of(kk), s = kk % S;
      V Tn = cst<V>(0.0);
      if constexpr (TH) {
        if (active && kk + 1 < nrows) Tn = load_value(Tcol + size_t(row_of(kk + 1)) * nx, V{});
      }
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], uint32_t((kk / S) & 1)))) {
        flag |= STATUS_TIMEOUT;
        failed = true;
        break;
      }
      const T* st = stage + size_t(s) * 9 * SW;
      const bool lo_wall = (q == tl.ylo), hi_wall = (q == tl.yhi);
      V g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = cst<V>(0.0);
      if (active) pull<SW>(st, j - 1 + H, lo_wall, hi_wall, g);
      if constexpr (ZH) {
        if (active && (lo_wall || hi_wall)) zou_he(g, lo_wall, dmean, k);
      }
      float el = 0.f, er = 0.f;  // psi of the warp-edge neighbours (another warp's or the halo)
      if (need_l || need_r) {
        const float v = scalar_psi(st, q, need_l ? j - 1 : j + 2, lo_wall, hi_wall);
        if (need_l) el = v; else er = v;
        if (need_l && need_r) er = scalar_psi(st, q, j + 2, lo_wall, hi_wall);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);  // this warp has read everything it needs of row kk
      PsiRow nw;
      if (active) {
        const V RT = TH ? k.R * Tq : k.RT;
        nw.c = psi_of<V>(k.rho_ref + sum9(g), RT, k, flag);
      } else {
        nw.c = cst<V>(0.0);
      }
      nw.l = __shfl_up_sync(0xffffffffu, hi(nw.c), 1);
      nw.r = __shfl_down_sync(0xffffffffu, lo(nw.c), 1);
      if (need_l) nw.l = el;
      if (need_r) nw.r = er;
      pm = p0;
      p0 = pp;
      pp = nw;
      if (kk >= 1) {
        const int y = row_of(kk - 1);
        if (active && y >= ya && y < yb) {
          // walk rows kk-2 / kk are south / north of y when walking up, and the reverse down
          if (up)
            collide(y, gp, pm, p0, pp);
          else
            collide(y, gp, pp, p0, pm);
        }
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) gp[i] = g[i];
      if constexpr (TH) Tq = Tn;
    }
    if (!failed) {  // last walk row: own only at a wall, where the stencil is not needed
      const int y = row_of(nrows - 1);
      if (active && y >= ya && y < yb) collide(y, gp, pp, pp, pp);
    }
    if (MODE == MODE_STEP) {
      const double v = warp_sum(acc.value());
      if (lane == 0) red[warp] = v;
    }
  }

  // one barrier for both status bits; a warp with a bit set reports it (one atomic per warp)
  if (__syncthreads_or(flag)) {
    const int wf = __reduce_or_sync(0xffffffffu, flag);
    if (lane == 0 && wf) atomicOr(io.status, wf);
  }
  if (MODE == MODE_STEP && warp == 0) {
    const double t = warp_sum(lane < NWC ? red[lane] : 0.0);
    if (lane == 0) io.part_out[blockIdx.x] = t;
  }
}

// ---- vector access for the whole-lattice passes: a lane takes 4 FP32 nodes (16-byte loads
// and stores of each plane; n = nx ny is a multiple of 4 for FP32, whose rows are 16-byte
// multiples) or 2 FP64 nodes, as node pairs of the accumulator's value type
template <typename T>
struct Quad;
template <>
struct Quad<float> {
  static constexpr int nodes = 4;
  using V = f2;
  __device__ static void load(const float* p, V (&v)[2]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = make_f2(q.x, q.y);
    v[1] = make_f2(q.z, q.w);
  }
  // store d rounded to FP32 and return the stored values as pairs
  __device__ static void store(float* p, const double (&d)[4], V (&v)[2]) {
    const float4 q = make_float4(float(d[0]), float(d[1]), float(d[2]), float(d[3]));
    *reinterpret_cast<float4*>(p) = q;
    v[0] = make_f2(q.x, q.y);
    v[1] = make_f2(q.z, q.w);
  }
};
template <>
struct Quad<double> {
  static constexpr int nodes = 2;
  using V = double;
  __device__ static void load(const double* p, V (&v)[2]) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x;
    v[1] = q.y;
  }
  __device__ static void store(double* p, const double (&d)[2], V (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(d[0], d[1]);
    v[0] = d[0];
    v[1] = d[1];
  }
};

// a block's FP64 total of its threads' accumulators, written to part[blockIdx.x]
template <typename V>
__device__ __forceinline__ void block_partial(const Acc<V>& acc, double* part) {
  __shared__ double red[32];
  const double s = warp_sum(acc.value());
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    const double t = warp_sum(threadIdx.x < nw ? red[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// ---- initial state g_i = f_i^eq(rho0, 0) - w_i rho_ref = w_i (rho0 - rho_ref), and the FP64
// partial sums of the stored values (every value into the two-sum pairs, as partials_kernel
// adds them): block b covers vector groups [b*chunk, (b+1)*chunk) and writes part[b]
template <typename T>
__global__ void init_kernel(const double* __restrict__ rho0, T* __restrict__ f, int nx, int ny, double rho_ref,
                            double* __restrict__ part) {
  using Q = Quad<T>;
  using V = typename Q::V;
  constexpr int NQ = Q::nodes;
  const size_t n = size_t(nx) * ny, groups = n / NQ;
  const size_t chunk = (groups + gridDim.x - 1) / gridDim.x;
  const size_t k0 = blockIdx.x * chunk, k1 = min(groups, k0 + chunk);
  Acc<V> acc;
  for (size_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double d[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) d[j] = rho0[k * NQ + j] - rho_ref;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      double v[NQ];
#pragma unroll
      for (int j = 0; j < NQ; ++j) v[j] = w_of(i) * d[j];
      V g[2];
      Q::store(f + i * n + k * NQ, v, g);
      acc.add(g[0], i % 3);
      acc.add(g[1], i % 3);
    }
  }
  block_partial(acc, part);
}

// ---- FP64 partial sums of sum_i g_i: block b covers vector groups [b*chunk, (b+1)*chunk).
// FP32 storage: every value into the per-thread two-sum pairs (GB300's FP64 pipe is slow),
// four nodes a thread per plane; FP64 storage: plain FP64 sums, two nodes a thread.
template <typename T>
__global__ void partials_kernel(const T* __restrict__ f, int nx, int ny, double* __restrict__ part) {
  using Q = Quad<T>;
  using V = typename Q::V;
  constexpr int NQ = Q::nodes;
  const size_t n = size_t(nx) * ny, groups = n / NQ;
  const size_t chunk = (groups + gridDim.x - 1) / gridDim.x;
  const size_t k0 = blockIdx.x * chunk, k1 = min(groups, k0 + chunk);
  Acc<V> acc;
#pragma unroll 2
  for (size_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    V g[9][2];
#pragma unroll
    for (int i = 0; i < 9; ++i) Q::load(f + i * n + k * NQ, g[i]);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      acc.add(g[i][0], i % 3);
      acc.add(g[i][1], i % 3);
    }
  }
  block_partial(acc, part);
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

// ---- tile variants of the fused kernel: (value type, band width, nodes per thread,
// CTAs/SM). Variant 0 of each precision is the default; lbm_autotune times the others.
using StepFnF = void (*)(StepTiling, PhysT<float>, StepIO);
using StepFnP = void (*)(StepTiling, PhysT<f2>, StepIO);
using StepFnD = void (*)(StepTiling, PhysT<double>, StepIO);

template <typename Fn>
struct ExtFns {  // kernels of one extension of a tile variant (nullptr: not built)
  Fn step = nullptr, step_unit = nullptr, moments = nullptr;
};
// extensions: [0] thermal, [1] Zou-He walls, [2] thermal with Zou-He walls
constexpr int kExt = 3;
__host__ __device__ constexpr int ext_index(bool th, bool zh) { return th && zh ? 2 : (zh ? 1 : 0); }

struct VariantF {  // FP32 storage; `paired` variants evaluate two nodes per value
  int bw, threads, stages;
  bool paired;
  StepFnF step, step_unit, moments;      // scalar variants
  StepFnP pstep, pstep_unit, pmoments;   // paired variants
  size_t smem;
  ExtFns<StepFnP> ext[kExt] = {};        // paired extensions (variant 0 only)
};
struct VariantD {
  int bw, threads, stages;
  StepFnD step, step_unit, moments;
  size_t smem;
  ExtFns<StepFnD> ext[kExt] = {};
};

template <int BW, int NPT, int MINB>
constexpr VariantF make_f() {
  return VariantF{BW, BW / NPT, kStages, false,
                  step_kernel<float, float, MODE_STEP, false, BW, NPT, MINB>,
                  step_kernel<float, float, MODE_STEP, true, BW, NPT, MINB>,
                  step_kernel<float, float, MODE_MOMENTS, false, BW, NPT, MINB>,
                  nullptr, nullptr, nullptr, step_smem<float, BW>()};
}
template <int BW, int NPT, int MINB>
constexpr VariantF make_p() {
  return VariantF{BW, BW / NPT, kStages, true, nullptr, nullptr, nullptr,
                  step_kernel<float, f2, MODE_STEP, false, BW, NPT, MINB>,
                  step_kernel<float, f2, MODE_STEP, true, BW, NPT, MINB>,
                  step_kernel<float, f2, MODE_MOMENTS, false, BW, NPT, MINB>, step_smem<float, BW>()};
}
template <int BW, int NPT, int MINB>
constexpr VariantD make_d() {
  return VariantD{BW, BW / NPT, kStages, step_kernel<double, double, MODE_STEP, false, BW, NPT, MINB>,
                  step_kernel<double, double, MODE_STEP, true, BW, NPT, MINB>,
                  step_kernel<double, double, MODE_MOMENTS, false, BW, NPT, MINB>, step_smem<double, BW>()};
}
// the same tile with the thermal and Zou-He kernels as well
template <int BW, int NPT, int MINB, bool TH, bool ZH>
constexpr ExtFns<StepFnD> ext_d() {
  return {step_kernel<double, double, MODE_STEP, false, BW, NPT, MINB, TH, ZH>,
          step_kernel<double, double, MODE_STEP, true, BW, NPT, MINB, TH, ZH>,
          step_kernel<double, double, MODE_MOMENTS, false, BW, NPT, MINB, TH, ZH>};
}
template <int BW, int NPT, int MINB>
constexpr VariantD make_d_ext() {
  VariantD v = make_d<BW, NPT, MINB>();
  v.ext[0] = ext_d<BW, NPT, MINB, true, false>();
  v.ext[1] = ext_d<BW, NPT, MINB, false, true>();
  v.ext[2] = ext_d<BW, NPT, MINB, true, true>();
  return v;
}

template <int NWC, int S, int MINB>
constexpr VariantF make_ws() {
  return VariantF{64 * NWC, (NWC + 1) * 32, S, true, nullptr, nullptr, nullptr,
                  step_kernel_ws<MODE_STEP, false, NWC, S, MINB>, step_kernel_ws<MODE_STEP, true, NWC, S, MINB>,
                  step_kernel_ws<MODE_MOMENTS, false, NWC, S, MINB>, ws_smem<NWC, S>()};
}
template <int NWC, int S, int MINB, bool TH, bool ZH>
constexpr ExtFns<StepFnP> ext_ws() {
  return {step_kernel_ws<MODE_STEP, false, NWC, S, MINB, TH, ZH>, step_kernel_ws<MODE_STEP, true, NWC, S, MINB, TH, ZH>,
          step_kernel_ws<MODE_MOMENTS, false, NWC, S, MINB, TH, ZH>};
}
template <int NWC, int S, int MINB>
constexpr VariantF make_ws_ext() {
  VariantF v = make_ws<NWC, S, MINB>();
  v.ext[0] = ext_ws<NWC, S, MINB, true, false>();
  v.ext[1] = ext_ws<NWC, S, MINB, false, true>();
  v.ext[2] = ext_ws<NWC, S, MINB, true, true>();
  return v;
}

const VariantF kVariantsF[] = {
    make_ws_ext<8, 3, 2>(),  // barrier-free: 8 consumer warps + producer, 3 stages, 56 KB (+ thermal, Zou-He)
    make_ws<4, 4, 4>(),      // barrier-free: 4 consumer warps + producer, 4 stages, 38 KB
    make_p<256, 2, 5>(),     // pairs, 4 warps, 42 KB shared, one CTA barrier per row
    make_f<256, 2, 5>(),     // scalar, 4 warps, 42 KB shared, one CTA barrier per row
    make_p<512, 4, 2>(),     // two pairs per thread, 4 warps, 83 KB shared
    make_ws<4, 6, 3>(),      // barrier-free, 6 stages, 57 KB
    make_ws<2, 6, 6>(),      // barrier-free, 2 consumer warps, 29 KB
    make_ws<8, 3, 3>(),      // barrier-free, 8 consumer warps, 3 stages, 3 CTAs per SM (72 registers)
};
const VariantD kVariantsD[] = {
    make_d_ext<128, 1, 4>(),  // (+ thermal, Zou-He)
    make_d<64, 1, 8>(),
};
constexpr int kNumF = sizeof(kVariantsF) / sizeof(kVariantsF[0]);
constexpr int kNumD = sizeof(kVariantsD) / sizeof(kVariantsD[0]);

template <class Fn>
cudaError_t set_smem(Fn fn, size_t smem) {
  if (!fn) return cudaSuccess;
  return cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}
cudaError_t prepare_variant(const VariantF& v) {
  cudaError_t e = cudaSuccess;
  for (auto fn : {v.step, v.step_unit, v.moments})
    if (e == cudaSuccess) e = set_smem(fn, v.smem);
  for (auto fn : {v.pstep, v.pstep_unit, v.pmoments})
    if (e == cudaSuccess) e = set_smem(fn, v.smem);
  for (const auto& x : v.ext)
    for (auto fn : {x.step, x.step_unit, x.moments})
      if (e == cudaSuccess) e = set_smem(fn, v.smem);
  return e;
}
cudaError_t prepare_variant(const VariantD& v) {
  cudaError_t e = cudaSuccess;
  for (auto fn : {v.step, v.step_unit, v.moments})
    if (e == cudaSuccess) e = set_smem(fn, v.smem);
  for (const auto& x : v.ext)
    for (auto fn : {x.step, x.step_unit, x.moments})
      if (e == cudaSuccess) e = set_smem(fn, v.smem);
  return e;
}

bool unit_relaxation(const StepPhys& p) {
  return p.s_e == 1.0 && p.s_vs == 1.0 && p.s_j == 1.0 && p.s_q == 1.0 && p.s_nu == 1.0;
}

int grid_for(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return int(g);
}

}  // namespace

// ---------------------------------------------------------------- launch wrappers
int stages(int precision, int variant) {
  return precision == 1 ? kVariantsF[variant].stages : kVariantsD[variant].stages;
}

int step_num_variants(int precision) { return precision == 1 ? kNumF : kNumD; }

bool step_variant_extended(int precision, int variant) {
  if (variant < 0 || variant >= step_num_variants(precision)) return false;
  return precision == 1 ? kVariantsF[variant].ext[0].step != nullptr : kVariantsD[variant].ext[0].step != nullptr;
}

bool step_variant_info(int precision, int variant, int* band_w, int* threads, int* smem) {
  if (variant < 0 || variant >= step_num_variants(precision)) return false;
  if (precision == 1) {
    *band_w = kVariantsF[variant].bw; *threads = kVariantsF[variant].threads; *smem = int(kVariantsF[variant].smem);
  } else {
    *band_w = kVariantsD[variant].bw; *threads = kVariantsD[variant].threads; *smem = int(kVariantsD[variant].smem);
  }
  return true;
}

int step_max_ctas_per_sm(int precision, int variant, int threads, int smem_bytes) {
  const void* fn;
  if (precision == 1) {
    const VariantF& v = kVariantsF[variant];
    fn = v.paired ? (const void*)v.pstep : (const void*)v.step;
  } else {
    fn = (const void*)kVariantsD[variant].step;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem_bytes) != cudaSuccess) return 0;
  return n;
}

cudaError_t step_prepare(int precision) {
  if (precision == 1) {
    for (const auto& v : kVariantsF) {
      cudaError_t e = prepare_variant(v);
      if (e != cudaSuccess) return e;
    }
  } else {
    for (const auto& v : kVariantsD) {
      cudaError_t e = prepare_variant(v);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_step(int precision, int mode, const StepTiling& t, const StepPhys& ph, const StepIO& io,
                        cudaStream_t stream) {
  const dim3 grid(t.nbands * t.nstrips), block(t.threads);
  const bool unit = unit_relaxation(ph);
  const bool th = io.Tfield != nullptr, zh = ph.wall == LBM_WALL_ZOU_HE;
  // a thermal step stores its rho, u: refuse a launch without somewhere to put them
  if (th && mode == MODE_STEP &&
      !(precision == 1 ? (io.rho32 && io.ux32 && io.uy32) : (io.rho_out && io.ux_out && io.uy_out)))
    return cudaErrorInvalidValue;
  if (precision == 1) {
    const VariantF& v = kVariantsF[t.variant];
    if (th || zh) {
      const ExtFns<StepFnP>& x = v.ext[ext_index(th, zh)];
      const StepFnP fn = mode == MODE_MOMENTS ? x.moments : (unit ? x.step_unit : x.step);
      if (!fn) return cudaErrorInvalidValue;  // no extension kernels for this tile variant
      return launch_dependent(fn, grid, block, t.smem_bytes, stream, t, to_phys<f2>(ph), io);
    } else if (v.paired) {
      const StepFnP fn = mode == MODE_MOMENTS ? v.pmoments : (unit ? v.pstep_unit : v.pstep);
      return launch_dependent(fn, grid, block, t.smem_bytes, stream, t, to_phys<f2>(ph), io);
    } else {
      const StepFnF fn = mode == MODE_MOMENTS ? v.moments : (unit ? v.step_unit : v.step);
      return launch_dependent(fn, grid, block, t.smem_bytes, stream, t, to_phys<float>(ph), io);
    }
  } else {
    const VariantD& v = kVariantsD[t.variant];
    StepFnD fn = mode == MODE_MOMENTS ? v.moments : (unit ? v.step_unit : v.step);
    if (th || zh) {
      const ExtFns<StepFnD>& x = v.ext[ext_index(th, zh)];
      fn = mode == MODE_MOMENTS ? x.moments : (unit ? x.step_unit : x.step);
    }
    if (!fn) return cudaErrorInvalidValue;  // no extension kernels for this tile variant
    return launch_dependent(fn, grid, block, t.smem_bytes, stream, t, to_phys<double>(ph), io);
  }
}

cudaError_t launch_init(int precision, const double* rho0, void* f, int nx, int ny, double rho_ref, double* part,
                        int npart, cudaStream_t stream) {
  if (precision == 1)
    init_kernel<float><<<npart, 256, 0, stream>>>(rho0, static_cast<float*>(f), nx, ny, rho_ref, part);
  else
    init_kernel<double><<<npart, 256, 0, stream>>>(rho0, static_cast<double*>(f), nx, ny, rho_ref, part);
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
