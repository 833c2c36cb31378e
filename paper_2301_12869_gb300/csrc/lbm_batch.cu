// Batched independent columns: one persistent launch advances thousands of small
// nx x ny_c lattices (each with its own height, temperature, gravity and gravity form)
// to a residual target. Method per column: the same step as lbm_kernels.cu (arXiv
// 2301.12869, Sec. III), evaluated by lbm_physics.cuh.
//
// Design: a CTA takes one column at a time by atomic work stealing (tallest first) and
// iterates it to convergence. The column's two population buffers stay in global memory
// - with a few hundred columns in flight the working set is L2-resident on GB300 - while
// psi, the residual snapshot and the partial sums live in shared memory. A step is two
// phases over all nodes of the column with one CTA barrier after each: (A) pull, rho and
// psi; (B) pull, Shan-Chen stencil, collision, store, and a CTA-wide FP64 reduction of
// the stored mass that gives the next step's <rho> (Eq. Gravity_2). Every `check_every`
// steps the residual max |rho_t - rho_(t-1)| decides whether the column has converged; it
// is evaluated in FP64 from the stored populations (an FP32 density rounds at 3e-8 and
// would hide the FP32 state's changes below that).
// The launch (counter reset + kernel) is captured once per batch into a CUDA graph; the
// run parameters live in device memory so the graph is reused by every run.
#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_dd.cuh"
#include "lbm_physics.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <iterator>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

namespace {

// threads per column CTA: the candidates of lbm_batch_autotune (256 by default)
constexpr int kThreadChoices[3] = {128, 256, 512};
constexpr int kDefaultThreads = 256;

struct BatchCol {
  int ny, form;
  long long node_off;  // nodes of the columns before this one
  double RT, gx, gy, rho_ref;
};

constexpr int kMpeK = 4;  // extrapolation order: kMpeK + 2 snapshots per cycle

struct RunParams {
  double tol;
  long long max_steps;
  int check_every;
  int stall_checks;  // > 0: a column also stops after this many checks without a 1 % gain
  int mpe_checks;    // > 0: a state snapshot every mpe_checks residual checks, extrapolation per cycle
  void* snap;        // kMpeK + 2 slots of 9 * total_nodes reals (NULL: no extrapolation)
  long long slot;    // elements per slot (9 * total_nodes)
};

struct BatchArgs {
  const BatchCol* cols;
  const int* order;  // processing order (tallest first)
  int ncols, nx;
  void* fA;  // state of every column (concatenated [col][9][ny][nx]); always holds the state between runs
  void* fB;  // second buffer of the same layout
  double a, b, G, sig_e, sig_vs, s_e, s_vs, s_j, s_q, s_nu;
  const RunParams* run;
  int* counter;
  long long* steps;
  double* resid;
  int* status;
  double* rho_out;  // MODE_MOMENTS outputs, concatenated like rho0
  double* ux_out;
  double* uy_out;
  long long* col_ns;  // per column: device nanoseconds its CTAs spent on it, summed over runs
  int zh;             // Zou-He wet-node walls on rows 0 and ny - 1 (else halfway bounce-back)
};

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
__device__ lbm::PhysT<T> column_phys(const BatchArgs& a, const BatchCol& c) {
  lbm::PhysT<T> k;
  k.rho_ref = lbm::from_double<T>(c.rho_ref);
  k.RT = lbm::from_double<T>(c.RT);
  k.R = lbm::from_double<T>(0.0);  // unused: batched columns are isothermal
  k.a = lbm::from_double<T>(a.a);
  k.b4 = lbm::from_double<T>(a.b / 4.0);
  k.twoOverG = lbm::from_double<T>(2.0 / a.G);
  k.negG = lbm::from_double<T>(-a.G);
  k.G2 = lbm::from_double<T>(a.G * a.G);
  k.s_e = lbm::from_double<T>(a.s_e); k.s_vs = lbm::from_double<T>(a.s_vs); k.s_j = lbm::from_double<T>(a.s_j); k.s_q = lbm::from_double<T>(a.s_q); k.s_nu = lbm::from_double<T>(a.s_nu);
  k.h_e = lbm::from_double<T>(1.0 - 0.5 * a.s_e); k.h_vs = lbm::from_double<T>(1.0 - 0.5 * a.s_vs); k.h_j = lbm::from_double<T>(1.0 - 0.5 * a.s_j);
  k.h_q = lbm::from_double<T>(1.0 - 0.5 * a.s_q); k.h_nu = lbm::from_double<T>(1.0 - 0.5 * a.s_nu);
  k.sig_e = lbm::from_double<T>(a.sig_e);
  k.nsig_vs = lbm::from_double<T>(-a.sig_vs);
  k.gx = lbm::from_double<T>(c.gx);
  k.gy = lbm::from_double<T>(c.gy);
  k.form = c.form;
  return k;
}

// pull streaming (Eq. LBE) of node (x, y) of a column: f_i(x, y) = f*_i(x - c_ix, y - c_iy),
// x periodic; at the walls the opposite population of the same node (halfway bounce-back)
template <typename T>
__device__ __forceinline__ void pull_col(const T* f, int nx, int ny, int N, int x, int y, T (&g)[9]) {
  const int xl = x == 0 ? nx - 1 : x - 1, xr = x == nx - 1 ? 0 : x + 1;
  const int node = y * nx + x;
  const bool lo = (y == 0), hi = (y == ny - 1);
  g[0] = f[0 * N + node];
  g[1] = f[1 * N + y * nx + xl];
  g[3] = f[3 * N + y * nx + xr];
  g[2] = lo ? f[4 * N + node] : f[2 * N + (y - 1) * nx + x];
  g[5] = lo ? f[7 * N + node] : f[5 * N + (y - 1) * nx + xl];
  g[6] = lo ? f[8 * N + node] : f[6 * N + (y - 1) * nx + xr];
  g[4] = hi ? f[2 * N + node] : f[4 * N + (y + 1) * nx + x];
  g[7] = hi ? f[5 * N + node] : f[7 * N + (y + 1) * nx + xr];
  g[8] = hi ? f[6 * N + node] : f[8 * N + (y + 1) * nx + xl];
}

// lane 0's value in every lane of the warp
__device__ __forceinline__ float bcast_lane0(float v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ double bcast_lane0(double v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ lbm::dd bcast_lane0(lbm::dd v) {
  return lbm::dd{__shfl_sync(0xffffffffu, v.hi, 0), __shfl_sync(0xffffffffu, v.lo, 0)};
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}

// stalls count only below this residual: about 30 ulp of an FP32 / FP64 density of 0.3
template <typename T>
constexpr double kStallBelow = sizeof(T) == 4 ? 1e-6 : 1e-13;

// sum of the stored (deviation) populations of a node in FP64, in a fixed order
template <typename T>
__device__ __forceinline__ double sum9_fp64(const T (&g)[9]) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) s += lbm::hsum(g[i]);
  return s;
}

// Minimal polynomial extrapolation of a column's fixed-point iteration (no counterpart in the
// paper; it changes the way to the steady state, not the state). The slow modes of a column
// decay as damped oscillations, so a single-ratio (Aitken) step does not apply; from
// kMpeK + 2 snapshots x_0..x_{kMpeK+1} taken every few hundred steps, with differences
// u_j = x_{j+1} - x_j, the coefficients c (c_kMpeK = 1) minimising |sum_j c_j u_j| give the
// estimate s = sum_j c_j x_j / sum_j c_j of the fixed point (j = 0..kMpeK). The Gram matrix
// is reduced over the CTA in FP64 and solved by one thread (Gaussian elimination with
// partial pivoting). The estimate replaces `cur` only if every node keeps a positive
// density; returns whether it did. Uniform over the CTA.
template <typename T, int NT>
__device__ bool mpe_extrapolate(const RunParams& run, int N, T* cur, const T* slot0, int tid, int lane, int warp,
                                const lbm::PhysT<T>& k) {
  constexpr int NU = kMpeK + 1, NG = NU * (NU + 1) / 2, NW = NT / 32;
  __shared__ double part[NG][NW];
  __shared__ double gam[NU];
  __shared__ int ok_s;
  const size_t slot = size_t(run.slot);
  double G[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) G[i] = 0.0;
  for (int e = tid; e < 9 * N; e += NT) {
    double x[NU + 1], u[NU];
#pragma unroll
    for (int j = 0; j <= NU; ++j) x[j] = lbm::hsum(slot0[j * slot + e]);
#pragma unroll
    for (int j = 0; j < NU; ++j) u[j] = x[j + 1] - x[j];
    int m = 0;
#pragma unroll
    for (int i = 0; i < NU; ++i)
#pragma unroll
      for (int j = i; j < NU; ++j) G[m++] += u[i] * u[j];
  }
#pragma unroll
  for (int i = 0; i < NG; ++i) {
    const double v = lbm::warp_sum(G[i]);
    if (lane == 0) part[i][warp] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double g[NG];
    for (int i = 0; i < NG; ++i) {
      g[i] = 0.0;
      for (int w = 0; w < NW; ++w) g[i] += part[i][w];
    }
    auto at = [&](int i, int j) {
      if (i > j) {
        const int t = i;
        i = j;
        j = t;
      }
      return g[i * NU - i * (i - 1) / 2 + (j - i)];
    };
    // sum_{j<K} G_ij c_j = -G_iK for i < K (K = kMpeK), c_K = 1
    double Am[kMpeK][kMpeK + 1];
    for (int i = 0; i < kMpeK; ++i) {
      for (int j = 0; j < kMpeK; ++j) Am[i][j] = at(i, j);
      Am[i][kMpeK] = -at(i, kMpeK);
    }
    bool ok = at(kMpeK, kMpeK) > 0.0;
    const double scale = at(0, 0) + at(kMpeK, kMpeK);
    for (int ci = 0; ci < kMpeK && ok; ++ci) {
      int piv = ci;
      for (int i = ci + 1; i < kMpeK; ++i)
        if (fabs(Am[i][ci]) > fabs(Am[piv][ci])) piv = i;
      if (!(fabs(Am[piv][ci]) > 1e-14 * scale)) {
        ok = false;
        break;
      }
      if (piv != ci)
        for (int j = 0; j <= kMpeK; ++j) {
          const double t = Am[ci][j];
          Am[ci][j] = Am[piv][j];
          Am[piv][j] = t;
        }
      for (int i = ci + 1; i < kMpeK; ++i) {
        const double f = Am[i][ci] / Am[ci][ci];
        for (int j = ci; j <= kMpeK; ++j) Am[i][j] -= f * Am[ci][j];
      }
    }
    double cvec[NU];
    cvec[kMpeK] = 1.0;
    for (int i = kMpeK - 1; i >= 0 && ok; --i) {
      double sum = Am[i][kMpeK];
      for (int j = i + 1; j < kMpeK; ++j) sum -= Am[i][j] * cvec[j];
      cvec[i] = sum / Am[i][i];
    }
    double S = 0.0, Sabs = 0.0;
    for (int j = 0; j < NU && ok; ++j) {
      S += cvec[j];
      Sabs += fabs(cvec[j]);
    }
    ok = ok && isfinite(S) && fabs(S) > 1e-8 * Sabs;
    for (int j = 0; j < NU; ++j) gam[j] = ok ? cvec[j] / S : 0.0;
    ok_s = ok ? 1 : 0;
  }
  __syncthreads();
  if (!ok_s) return false;
  // the estimate, node by node; a non-positive density rejects it
  int bad = 0;
  for (int n = tid; n < N; n += NT) {
    double rho = lbm::hsum(k.rho_ref);
    T v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < NU; ++j) acc += gam[j] * lbm::hsum(slot0[j * slot + size_t(i) * N + n]);
      v[i] = lbm::from_double<T>(acc);
      rho += acc;
    }
    if (!(rho > 0.0)) bad = 1;
#pragma unroll
    for (int i = 0; i < 9; ++i) cur[i * N + n] = v[i];
  }
  if (__syncthreads_or(bad)) {  // back to the last snapshot (x_{kMpeK+1} is the state before)
    const T* last = slot0 + size_t(kMpeK + 1) * slot;
    for (int e = tid; e < 9 * N; e += NT) cur[e] = last[e];
    __syncthreads();
    return false;
  }
  return true;
}

template <typename T, int MODE, bool UNIT, bool ACC, int NT>
__global__ void __launch_bounds__(NT) batch_kernel(const BatchArgs a) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[2][NW];  // mass partials of the state each iteration reads
  __shared__ double rmax[NW];
  __shared__ int s_col;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const RunParams run = *a.run;
  const int K = run.check_every;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_col = atomicAdd(a.counter, 1);
    __syncthreads();
    const int ci = s_col;
    if (ci >= a.ncols) break;
    const long long t_start = global_ns();
    const int c = a.order[ci];
    const BatchCol col = a.cols[c];
    const int nx = a.nx, ny = col.ny, N = nx * ny;
    T* psi_s = reinterpret_cast<T*>(sm_raw);
    double* rho_prev = reinterpret_cast<double*>(sm_raw + ((size_t(N) * sizeof(T) + 15) & ~size_t(15)));
    const lbm::PhysT<T> k = column_phys<T>(a, col);
    T* cur = static_cast<T*>(a.fA) + 9 * col.node_off;
    T* nxt = static_cast<T*>(a.fB) + 9 * col.node_off;

    {  // mass of the stored state, for <rho> of the first step
      lbm::Acc<T> acc;
      for (int n = tid; n < N; n += NT) {
        T g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = cur[i * N + n];
        acc.add9(g);
      }
      const double v = lbm::warp_sum(acc.value());
      if (lane == 0) red[0][warp] = v;
    }
    __syncthreads();

    int flag = 0;
    double res = MODE == lbm::MODE_STEP ? a.resid[c] : 0.0;
    double best = INFINITY;  // smallest residual of this run, for the stall test
    int stalled = 0;
    // extrapolation state (uniform over the CTA)
    const bool mpe = ACC && MODE == lbm::MODE_STEP && run.mpe_checks > 0 && run.snap != nullptr;
    int nsnap = 0, checks_since = 0;
    bool verify = false, skip_cycle = false;
    double res_before = 0.0;
    auto slot_ptr = [&](int j) { return static_cast<T*>(run.snap) + size_t(j) * size_t(run.slot) + 9 * col.node_off; };
    // FP64 partials of the stored mass of a state into red[q] (what the next step reads)
    auto remass = [&](const T* st, int q) {
      lbm::Acc<T> acc2;
      for (int n = tid; n < N; n += NT) {
        T g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = st[i * N + n];
        acc2.add9(g);
      }
      const double v = lbm::warp_sum(acc2.value());
      if (lane == 0) red[q][warp] = v;
      __syncthreads();
    };
    long long it = 0;
    const long long iters = MODE == lbm::MODE_STEP ? run.max_steps : 1;
    for (; it < iters; ++it) {
      const int p = int(it & 1);
      // <rho> - rho_ref from the FP64 mass partials: lane 0 of each warp forms it (GB300's
      // FP64 pipe is slow; the division alone is ~20 FP64 instructions) and broadcasts it
      T dmean;
      {
        T dm = lbm::cst<T>(0.0);
        if (lane == 0) {
          double msum = 0.0;
          for (int w2 = 0; w2 < NW; ++w2) msum += red[p][w2];  // same order in every warp
          dm = lbm::from_double<T>(msum / double(N));
        }
        dmean = bcast_lane0(dm);
      }
      const bool save = MODE == lbm::MODE_STEP && K >= 2 && ((it + 2) % K == 0);
      const bool chk = MODE == lbm::MODE_STEP && K >= 2 && ((it + 1) % K == 0);
      // (A) rho and psi of every node (Eqs. Density, EOS, InteractionPotential)
      for (int n = tid; n < N; n += NT) {
        const int x = n % nx, y = n / nx;
        T g[9];
        pull_col(cur, nx, ny, N, x, y, g);
        if (a.zh && (y == 0 || y == ny - 1)) lbm::zou_he(g, y == 0, dmean, k);
        const T rho = k.rho_ref + lbm::sum9(g);
        psi_s[n] = lbm::psi_of<T>(rho, k, flag);
        if (save) rho_prev[n] = sum9_fp64(g);
      }
      __syncthreads();
      // (B) forces, velocity, collision, store (Eqs. ShanChenForce, Gravity_1/2, Momentum,
      // OperatorMRT, LiFS)
      lbm::Acc<T> acc;
      double rm = 0.0;
      for (int n = tid; n < N; n += NT) {
        const int x = n % nx, y = n / nx;
        const int xl = x == 0 ? nx - 1 : x - 1, xr = x == nx - 1 ? 0 : x + 1;
        T g[9];
        pull_col(cur, nx, ny, N, x, y, g);
        if (a.zh && (y == 0 || y == ny - 1)) lbm::zou_he(g, y == 0, dmean, k);
        T Sx = lbm::cst<T>(0.0), Sy = lbm::cst<T>(0.0);
        if (y > 0 && y < ny - 1) {  // stencil w(1) = 1/3, w(2) = 1/12; zero on the wall rows
          const T* pc = psi_s + y * nx;
          const T* pn = pc + nx;
          const T* ps = pc - nx;
          const T E = pc[xr], Wt = pc[xl], Nn = pn[x], Ss = ps[x];
          const T NE = pn[xr], NW = pn[xl], SE = ps[xr], SWt = ps[xl];
          Sx = lbm::fmadd(lbm::cst<T>(1.0 / 3.0), E - Wt, lbm::cst<T>(1.0 / 12.0) * ((NE - NW) + (SE - SWt)));
          Sy = lbm::fmadd(lbm::cst<T>(1.0 / 3.0), Nn - Ss, lbm::cst<T>(1.0 / 12.0) * ((NE + NW) - (SE + SWt)));
        }
        T o[9], rho, ux, uy;
        lbm::collide_node<T, UNIT>(g, psi_s[n], Sx, Sy, dmean, k, o, rho, ux, uy, flag);
        if (MODE == lbm::MODE_STEP) {
#pragma unroll
          for (int i = 0; i < 9; ++i) nxt[i * N + n] = o[i];
          acc.add9(o);
          if (chk) rm = fmax(rm, fabs(sum9_fp64(g) - rho_prev[n]));
        } else {
          const long long idx = col.node_off + n;
          if (a.rho_out) a.rho_out[idx] = lbm::hsum(rho);
          if (a.ux_out) a.ux_out[idx] = lbm::hsum(ux);
          if (a.uy_out) a.uy_out[idx] = lbm::hsum(uy);
        }
      }
      if (MODE != lbm::MODE_STEP) break;
      const double v = lbm::warp_sum(acc.value());
      const double m = warp_max(rm);
      if (lane == 0) {
        red[p ^ 1][warp] = v;
        rmax[warp] = m;
      }
      __syncthreads();
      T* t = cur;
      cur = nxt;
      nxt = t;
      if (chk) {
        double r = 0.0;
        for (int w2 = 0; w2 < NW; ++w2) r = fmax(r, rmax[w2]);
        res = r;
        if (!(r > run.tol)) {  // converged (uniform decision)
          ++it;
          break;
        }
        if (r < 0.99 * best) {
          best = r;
          stalled = 0;
        } else if (run.stall_checks > 0 && r < kStallBelow<T> && ++stalled >= run.stall_checks) {
          // no gain near the precision's rounding floor (transients above it may plateau)
          ++it;
          break;
        }
        if (ACC && mpe) {
          const int q = (it + 1) & 1;  // partials the next iteration reads
          if (verify) {
            // the first check after an extrapolation: a larger change than before it means
            // the estimate is worse - go back to the last snapshot
            verify = false;
            if (r > res_before) {
              const T* last = slot_ptr(kMpeK + 1);
              for (int e = tid; e < 9 * N; e += NT) cur[e] = last[e];
              __syncthreads();
              remass(cur, q);
              skip_cycle = true;
              nsnap = 0;
              checks_since = 0;
            }
          }
          if (++checks_since >= run.mpe_checks) {
            checks_since = 0;
            T* dst = slot_ptr(nsnap);
            for (int e = tid; e < 9 * N; e += NT) dst[e] = cur[e];
            __syncthreads();
            if (++nsnap == kMpeK + 2) {
              nsnap = 0;
              if (skip_cycle) {
                skip_cycle = false;
              } else if (mpe_extrapolate<T, NT>(run, N, cur, slot_ptr(0), tid, lane, warp, k)) {
                remass(cur, q);
                verify = true;
                res_before = r;
              }
            }
          }
        }
      }
    }
    if (MODE == lbm::MODE_STEP) {
      T* A = static_cast<T*>(a.fA) + 9 * col.node_off;
      if (cur != A)  // the state ends in the second buffer: copy it back
        for (int e = tid; e < 9 * N; e += NT) A[e] = cur[e];
    }
    const int any = __syncthreads_or(flag);
    if (tid == 0 && MODE == lbm::MODE_STEP) {
      a.steps[c] += it;
      a.resid[c] = res;
      if (any) a.status[c] |= lbm::STATUS_NONPHYS;
      a.col_ns[c] += global_ns() - t_start;
    }
  }
}

// The rest state of every column's stored density field rho = sum_i f*_i (lbm_batch_rest_state):
// the forces of Eqs. ShanChenForce and Gravity_1 / Gravity_2 from rho, pre-collision
// populations with the moments of the rest equilibrium f_eq(rho, 0) except the momentum -F/2
// (so that the velocity of Eq. Momentum vanishes), and one collision (collide_node, Eqs.
// OperatorMRT, LiFS); written in place. psi of the column is staged in shared memory first.
// One CTA of 256 threads per column at a time.
template <typename T, bool UNIT>
__global__ void __launch_bounds__(256) batch_rest_kernel(const BatchArgs a) {
  constexpr int NT = 256, NW = NT / 32;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* psi_s = reinterpret_cast<T*>(sm_raw);
  for (int c = blockIdx.x; c < a.ncols; c += gridDim.x) {
    const BatchCol col = a.cols[c];
    const int nx = a.nx, ny = col.ny, N = nx * ny;
    const lbm::PhysT<T> k = column_phys<T>(a, col);
    T* cur = static_cast<T*>(a.fA) + 9 * col.node_off;
    int flag = 0;
    lbm::Acc<T> acc;  // FP64 mass of the stored state, for <rho> of Eq. Gravity_2
    for (int n = tid; n < N; n += NT) {
      T g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = cur[i * N + n];
      acc.add9(g);
      psi_s[n] = lbm::psi_of<T>(k.rho_ref + lbm::sum9(g), k, flag);
    }
    const double v = lbm::warp_sum(acc.value());
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double msum = 0.0;
    for (int w = 0; w < NW; ++w) msum += red[w];
    const T dmean = lbm::from_double<T>(msum / double(N));
    for (int n = tid; n < N; n += NT) {
      const int x = n % nx, y = n / nx;
      const int xl = x == 0 ? nx - 1 : x - 1, xr = x == nx - 1 ? 0 : x + 1;
      T g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = cur[i * N + n];
      const T dr = lbm::sum9(g);
      T Sx = lbm::cst<T>(0.0), Sy = lbm::cst<T>(0.0);
      if (y > 0 && y < ny - 1) {  // as in batch_kernel: w(1) = 1/3, w(2) = 1/12, zero on the wall rows
        const T* pc = psi_s + y * nx;
        const T* pn = pc + nx;
        const T* ps = pc - nx;
        const T E = pc[xr], Wt = pc[xl], Nn = pn[x], Ss = ps[x];
        const T NE = pn[xr], NW2 = pn[xl], SE = ps[xr], SWt = ps[xl];
        Sx = lbm::fmadd(lbm::cst<T>(1.0 / 3.0), E - Wt, lbm::cst<T>(1.0 / 12.0) * ((NE - NW2) + (SE - SWt)));
        Sy = lbm::fmadd(lbm::cst<T>(1.0 / 3.0), Nn - Ss, lbm::cst<T>(1.0 / 12.0) * ((NE + NW2) - (SE + SWt)));
      }
      // F = F_int + F_g as collide_node forms it
      const T base = (k.form == 2) ? (dr - dmean) : (k.rho_ref + dr);
      const T nGpsi = k.negG * psi_s[n];
      const T Fx = lbm::fmadd(nGpsi, Sx, base * k.gx);
      const T Fy = lbm::fmadd(nGpsi, Sy, base * k.gy);
      // deviations with the moments (dr, e = -2 dr, eps = dr, j = -F/2, q = 0, p_xx = p_xy = 0):
      // w_i dr plus the momentum part j/6 along each link (M^-1 with q = 0)
      const T ax = lbm::cst<T>(-1.0 / 12.0) * Fx, ay = lbm::cst<T>(-1.0 / 12.0) * Fy;  // j/6
      const T r9 = lbm::cst<T>(1.0 / 9.0) * dr, r36 = lbm::cst<T>(1.0 / 36.0) * dr;
      T pre[9];
      pre[0] = lbm::cst<T>(4.0 / 9.0) * dr;
      pre[1] = r9 + ax;
      pre[3] = r9 - ax;
      pre[2] = r9 + ay;
      pre[4] = r9 - ay;
      pre[5] = r36 + (ax + ay);
      pre[7] = r36 - (ax + ay);
      pre[6] = r36 + (ay - ax);
      pre[8] = r36 - (ay - ax);
      T o[9], rho, ux, uy;
      lbm::collide_node<T, UNIT>(pre, psi_s[n], Sx, Sy, dmean, k, o, rho, ux, uy, flag);
#pragma unroll
      for (int i = 0; i < 9; ++i) cur[i * N + n] = o[i];
    }
    if (__syncthreads_or(flag) && tid == 0) a.status[c] |= lbm::STATUS_NONPHYS;
  }
}

// g_i = w_i (rho0 - rho_ref) for every column
template <typename T>
__global__ void batch_init_kernel(const BatchCol* cols, int ncols, int nx, const double* rho0, T* f) {
  for (int c = blockIdx.x; c < ncols; c += gridDim.x) {
    const BatchCol col = cols[c];
    const int N = nx * col.ny;
    T* fc = f + 9 * col.node_off;
    const double* r = rho0 + col.node_off;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
      const double d = r[n] - col.rho_ref;
#pragma unroll
      for (int i = 0; i < 9; ++i) fc[i * N + n] = lbm::from_double<T>(lbm::w_of(i) * d);
    }
  }
}

// absolute populations of every column (to_double) or back (from_double)
template <typename T>
__global__ void batch_state_kernel(const BatchCol* cols, int ncols, int nx, T* f, double* out, bool to_double) {
  for (int c = blockIdx.x; c < ncols; c += gridDim.x) {
    const BatchCol col = cols[c];
    const int N = nx * col.ny;
    T* fc = f + 9 * col.node_off;
    double* oc = out + 9 * col.node_off;
    for (int e = threadIdx.x; e < 9 * N; e += blockDim.x) {
      const double w = lbm::w_of(e / N) * col.rho_ref;
      if (to_double)
        oc[e] = lbm::hsum(fc[e]) + w;
      else
        fc[e] = lbm::from_double<T>(oc[e] - w);
    }
  }
}

thread_local char g_berr[512] = "";

int bfail(int code, const char* msg) {
  snprintf(g_berr, sizeof(g_berr), "%s", msg);
  lbm::set_last_error(g_berr);
  return code;
}

}  // namespace

struct lbm_batch {
  lbm_params p{};
  int ncols = 0, nx = 0, max_ny = 0;
  long long total_nodes = 0;
  size_t s = 4;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<BatchCol> cols;
  BatchCol* cols_d = nullptr;
  int* order_d = nullptr;
  void* fA = nullptr;
  void* fB = nullptr;
  int* counter = nullptr;
  RunParams* run_d = nullptr;
  long long* steps_d = nullptr;
  double* resid_d = nullptr;
  int* status_d = nullptr;
  long long* ns_d = nullptr;  // per column device nanoseconds, summed over runs
  int grid = 0;
  size_t smem = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_acc = false;  // the captured launch is the extrapolating kernel
  int graph_threads = 0;   // and its block size
  int grid_acc = 0;        // its resident grid
  int threads = kDefaultThreads;  // block size (one CTA per column at a time)
  int nsm = 0;
  int mpe_checks = 0;      // extrapolation cycle (residual checks per snapshot); 0: off
  void* snap = nullptr;    // kMpeK + 2 snapshot slots of 9 * total_nodes reals
};

namespace {

template <typename T, int MODE, bool UNIT, bool ACC>
void* batch_fn(int threads) {
  switch (threads) {
    case 128: return reinterpret_cast<void*>(&batch_kernel<T, MODE, UNIT, ACC, 128>);
    case 512: return reinterpret_cast<void*>(&batch_kernel<T, MODE, UNIT, ACC, 512>);
    default: return reinterpret_cast<void*>(&batch_kernel<T, MODE, UNIT, ACC, 256>);
  }
}

template <typename T>
void* pick_typed(int mode, bool unit, bool acc, int threads) {
  if (mode == lbm::MODE_MOMENTS) return batch_fn<T, lbm::MODE_MOMENTS, false, false>(threads);
  if (acc)
    return unit ? batch_fn<T, lbm::MODE_STEP, true, true>(threads) : batch_fn<T, lbm::MODE_STEP, false, true>(threads);
  return unit ? batch_fn<T, lbm::MODE_STEP, true, false>(threads) : batch_fn<T, lbm::MODE_STEP, false, false>(threads);
}

// the extrapolating kernel only when the batch is set to extrapolate (it holds more registers)
void* pick_kernel(int precision, int mode, bool unit, bool acc, int threads) {
  if (precision == LBM_FP32) return pick_typed<float>(mode, unit, acc, threads);
  if (precision == LBM_DOUBLE_FLOAT) return pick_typed<lbm::dd>(mode, unit, acc, threads);
  return pick_typed<double>(mode, unit, acc, threads);
}

// one kernel launch over the batch's state in its storage type
template <template <typename> class K, typename... Args>
void launch_typed(int precision, int grid, cudaStream_t s, void* f, Args... args) {
  if (precision == LBM_FP32)
    K<float>::launch(grid, s, static_cast<float*>(f), args...);
  else if (precision == LBM_DOUBLE_FLOAT)
    K<lbm::dd>::launch(grid, s, static_cast<lbm::dd*>(f), args...);
  else
    K<double>::launch(grid, s, static_cast<double*>(f), args...);
}
template <typename T>
struct InitLaunch {
  static void launch(int grid, cudaStream_t s, T* f, const BatchCol* cols, int ncols, int nx, const double* rho0) {
    batch_init_kernel<T><<<grid, 256, 0, s>>>(cols, ncols, nx, rho0, f);
  }
};
template <typename T>
struct StateLaunch {
  static void launch(int grid, cudaStream_t s, T* f, const BatchCol* cols, int ncols, int nx, double* out, bool to_double) {
    batch_state_kernel<T><<<grid, 256, 0, s>>>(cols, ncols, nx, f, out, to_double);
  }
};

BatchArgs make_args(const lbm_batch* b) {
  BatchArgs a{};
  a.cols = b->cols_d;
  a.order = b->order_d;
  a.ncols = b->ncols;
  a.nx = b->nx;
  a.fA = b->fA;
  a.fB = b->fB;
  a.a = b->p.a;
  a.b = b->p.b;
  a.G = b->p.G;
  a.sig_e = b->p.sigma / (b->p.tau_e - 0.5);
  a.sig_vs = b->p.sigma / (b->p.tau_varsigma - 0.5);
  a.s_e = 1.0 / b->p.tau_e;
  a.s_vs = 1.0 / b->p.tau_varsigma;
  a.s_j = 1.0 / b->p.tau_j;
  a.s_q = 1.0 / b->p.tau_q;
  a.s_nu = 1.0 / b->p.tau_nu;
  a.run = b->run_d;
  a.counter = b->counter;
  a.steps = b->steps_d;
  a.resid = b->resid_d;
  a.status = b->status_d;
  a.col_ns = b->ns_d;
  a.zh = b->p.wall == LBM_WALL_ZOU_HE;
  return a;
}

bool unit_tau(const lbm_params& p) {
  return p.tau_e == 1.0 && p.tau_varsigma == 1.0 && p.tau_j == 1.0 && p.tau_q == 1.0 && p.tau_nu == 1.0;
}

bool accelerated(const lbm_batch* b) { return b->snap != nullptr && b->mpe_checks > 0; }

cudaError_t launch(const lbm_batch* b, int mode, BatchArgs args) {
  const bool acc = mode == lbm::MODE_STEP && accelerated(b);
  void* fn = pick_kernel(b->p.precision, mode, unit_tau(b->p), acc, b->threads);
  void* kargs[] = {&args};
  return cudaLaunchKernel(fn, dim3(acc ? b->grid_acc : b->grid), dim3(b->threads), kargs, b->smem, b->stream);
}

// persistent grids of the plain and the extrapolating kernel at the batch's block size:
// resident CTAs on every SM, capped so that the columns in flight keep their two buffers
// in L2 (about 96 MB)
void size_grids(lbm_batch* b) {
  const double avg_bytes = 2.0 * 9.0 * double(b->s) * double(b->total_nodes) / double(b->ncols);
  const int l2_cap = std::max(b->nsm, int(96.0e6 / avg_bytes));
  for (bool acc : {false, true}) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, pick_kernel(b->p.precision, lbm::MODE_STEP, unit_tau(b->p), acc, b->threads), b->threads, b->smem);
    (acc ? b->grid_acc : b->grid) = std::max(1, std::min({b->nsm * std::max(per_sm, 1), l2_cap, b->ncols}));
  }
}

void free_batch(lbm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* ptr : {(void*)b->cols_d, (void*)b->order_d, b->fA, b->fB, (void*)b->counter, (void*)b->run_d,
                    (void*)b->steps_d, (void*)b->resid_d, (void*)b->status_d, (void*)b->ns_d, b->snap})
    if (ptr) cudaFree(ptr);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // namespace

extern "C" {

int lbm_batch_init(const lbm_params* p, const lbm_column* cols, int ncols, const double* rho0, int rho0_where,
                   void* stream, lbm_batch** out) {
  if (!p || !cols || !rho0 || !out || ncols <= 0) return bfail(LBM_EINVAL, "p, cols, rho0, out must be set and ncols > 0");
  *out = nullptr;
  // validate the shared parameters with a representative column
  lbm_params q = *p;
  q.ny = cols[0].ny;
  q.T = cols[0].T;
  q.gravity_form = cols[0].gravity_form;
  if (q.precision == LBM_DOUBLE_FLOAT) q.precision = LBM_FP64;  // batches only; validated like FP64
  char err[512];
  int rc = lbm::validate_params(&q, err);
  if (rc) return bfail(rc, err);
  if (p->thermal) return bfail(LBM_EINVAL, "batched columns are isothermal (thermal must be 0)");
  if (p->nx > 64) return bfail(LBM_EINVAL, "batched columns are at most 64 nodes wide");
  if (rho0_where != LBM_HOST && rho0_where != LBM_DEVICE) return bfail(LBM_EINVAL, "rho0_where must be LBM_HOST or LBM_DEVICE");
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(LBM_ENOMEM, "out of host memory");
  b->p = *p;
  b->ncols = ncols;
  b->nx = p->nx;
  b->s = p->precision == LBM_FP32 ? 4 : 8;
  auto fail = [&](int code, const char* msg) {
    free_batch(b);
    return bfail(code, msg);
  };
  long long off = 0;
  b->cols.resize(ncols);
  for (int c = 0; c < ncols; ++c) {
    const lbm_column& in = cols[c];
    q.ny = in.ny;
    q.T = in.T;
    q.gx = in.gx;
    q.gy = in.gy;
    q.gravity_form = in.gravity_form;
    if ((rc = lbm::validate_params(&q, err))) return fail(rc, err);
    if (double(p->nx) * in.ny * ((p->precision == LBM_FP32 ? 4 : 8) + 8) + 16 > 200.0 * 1024)
      return fail(LBM_EINVAL, "column too large for the batch kernel's shared memory (nx ny (sizeof(real) + 8) <= 200 KiB)");
    BatchCol& bc = b->cols[c];
    bc.ny = in.ny;
    bc.form = in.gravity_form;
    bc.node_off = off;
    bc.RT = p->R * in.T;
    bc.gx = in.gx;
    bc.gy = in.gy;
    bc.rho_ref = 0.0;
    off += (long long)p->nx * in.ny;
    b->max_ny = std::max(b->max_ny, in.ny);
  }
  b->total_nodes = off;
  // deviation reference per column: the mean of its rho0 in FP32, 0 in FP64 (or p->rho_ref)
  std::vector<double> rho_h;
  const double* rho_src = rho0;
  if (rho0_where == LBM_DEVICE && p->precision != LBM_FP64 && std::isnan(p->rho_ref)) {
    rho_h.resize(size_t(off));
    if (cudaMemcpy(rho_h.data(), rho0, size_t(off) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(LBM_ECUDA, "copy of rho0");
    rho_src = rho_h.data();
  }
  for (int c = 0; c < ncols; ++c) {
    BatchCol& bc = b->cols[c];
    if (!std::isnan(p->rho_ref)) {
      bc.rho_ref = p->rho_ref;
    } else if (p->precision != LBM_FP64) {
      const long long n = (long long)p->nx * bc.ny;
      double s = 0.0;
      for (long long i = 0; i < n; ++i) s += rho_src[bc.node_off + i];
      bc.rho_ref = s / double(n);
    }
  }
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {  // graph capture needs a stream other than the legacy default one
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(LBM_ECUDA, "stream");
    b->own_stream = true;
  }
  const size_t state = size_t(off) * 9 * b->s;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  alloc((void**)&b->cols_d, sizeof(BatchCol) * ncols);
  alloc((void**)&b->order_d, sizeof(int) * ncols);
  alloc(&b->fA, state);
  alloc(&b->fB, state);
  alloc((void**)&b->counter, sizeof(int));
  alloc((void**)&b->run_d, sizeof(RunParams));
  alloc((void**)&b->steps_d, sizeof(long long) * ncols);
  alloc((void**)&b->resid_d, sizeof(double) * ncols);
  alloc((void**)&b->status_d, sizeof(int) * ncols);
  alloc((void**)&b->ns_d, sizeof(long long) * ncols);
  if (e != cudaSuccess) return fail(LBM_ENOMEM, "device allocation for the batch failed");
  // tallest columns first (longest work first balances the work-stealing queue)
  std::vector<int> order(ncols);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cols[x].ny > cols[y].ny; });
  std::vector<double> inf(ncols, INFINITY);
  e = cudaMemcpyAsync(b->cols_d, b->cols.data(), sizeof(BatchCol) * ncols, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->order_d, order.data(), sizeof(int) * ncols, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->steps_d, 0, sizeof(long long) * ncols, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->resid_d, inf.data(), sizeof(double) * ncols, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->status_d, 0, sizeof(int) * ncols, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ns_d, 0, sizeof(long long) * ncols, b->stream);
  // rho0 on the device: a host rho0 is staged through the second buffer (8 bytes per node
  // fit in its 9 * sizeof(real) bytes per node)
  double* rho_d = const_cast<double*>(rho0);
  if (e == cudaSuccess && rho0_where == LBM_HOST) {
    e = cudaMemcpyAsync(b->fB, rho0, size_t(off) * 8, cudaMemcpyHostToDevice, b->stream);
    rho_d = static_cast<double*>(b->fB);
  }
  if (e == cudaSuccess && rho_d) {
    launch_typed<InitLaunch>(p->precision, std::min(ncols, 4096), b->stream, b->fA, (const BatchCol*)b->cols_d, ncols,
                             b->nx, (const double*)rho_d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  b->smem = ((size_t(b->nx) * size_t(b->max_ny) * b->s + 15) & ~size_t(15)) + size_t(b->nx) * size_t(b->max_ny) * 8;
  for (int nt : kThreadChoices)
    for (int mode : {lbm::MODE_STEP, lbm::MODE_MOMENTS})
      for (bool u : {false, true})
        for (bool acc : {false, true}) {
          e = cudaFuncSetAttribute(pick_kernel(p->precision, mode, u, acc, nt),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(b->smem));
          if (e != cudaSuccess) return fail(LBM_ECUDA, "batch kernel shared memory limit");
        }
  size_grids(b);
  *out = b;
  return LBM_OK;
}

int lbm_batch_set_acceleration(lbm_batch* b, int checks) {
  if (!b) return bfail(LBM_EINVAL, "batch is NULL");
  if (checks < 0 || checks == 1) return bfail(LBM_EINVAL, "checks must be 0 (off) or >= 2");
  if (checks > 0 && !b->snap) {
    const size_t bytes = size_t(kMpeK + 2) * 9 * size_t(b->total_nodes) * b->s;
    cudaError_t e = cudaMalloc(&b->snap, bytes);
    if (e != cudaSuccess) {
      b->snap = nullptr;
      return bfail(LBM_ENOMEM, "cudaMalloc of the extrapolation snapshots failed");
    }
  }
  b->mpe_checks = checks;
  return LBM_OK;
}

int lbm_batch_set_threads(lbm_batch* b, int threads) {
  if (!b) return bfail(LBM_EINVAL, "batch is NULL");
  if (std::find(std::begin(kThreadChoices), std::end(kThreadChoices), threads) == std::end(kThreadChoices))
    return bfail(LBM_EINVAL, "threads must be 128, 256 or 512");
  b->threads = threads;
  size_grids(b);
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int steps, int* threads, double* us) {
  lbm::TraceRange trace("lbm_batch_autotune");
  if (!b) return bfail(LBM_EINVAL, "batch is NULL");
  if (steps < 1) return bfail(LBM_EINVAL, "steps must be >= 1");
  // a copy of the current state, so that b's state and results stay as they are
  lbm_batch* t = nullptr;
  int rc = lbm_batch_convert(b, b->p.precision, &t);
  if (rc) return rc;
  t->mpe_checks = b->mpe_checks;
  t->snap = nullptr;  // timed without extrapolation snapshots: the plain kernel's block size
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best_us = 0.0;
  int best = b->threads;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    t->threads = kThreadChoices[i];
    size_grids(t);
    float ms = 0.f;
    // every column `steps` steps (tol < 0: no column stops early), after a 2-step warm-up
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
      const RunParams rp{-1.0, pass == 0 ? 2LL : (long long)steps, 100, 0, 0, nullptr, 9 * t->total_nodes};
      e = cudaMemcpyAsync(t->run_d, &rp, sizeof(rp), cudaMemcpyHostToDevice, t->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(t->counter, 0, sizeof(int), t->stream);
      if (e == cudaSuccess && pass == 1) e = cudaEventRecord(e0, t->stream);
      if (e == cudaSuccess) e = launch(t, lbm::MODE_STEP, make_args(t));
      if (e == cudaSuccess && pass == 1) e = cudaEventRecord(e1, t->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    const double v = 1e3 * double(ms) / steps;
    if (threads) threads[i] = kThreadChoices[i];
    if (us) us[i] = v;
    if (i == 0 || v < best_us) {
      best_us = v;
      best = kThreadChoices[i];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  lbm_batch_destroy(t);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  return lbm_batch_set_threads(b, best);
}

int lbm_batch_run(lbm_batch* b, double tol, int64_t max_steps, int check_every, double* seconds) {
  return lbm_batch_run_stall(b, tol, max_steps, check_every, 0, seconds);
}

int lbm_batch_run_stall(lbm_batch* b, double tol, int64_t max_steps, int check_every, int stall_checks,
                        double* seconds) {
  lbm::TraceRange trace("lbm_batch_run");
  if (!b) return bfail(LBM_EINVAL, "batch is NULL");
  if (max_steps < 0 || check_every < 2 || !(tol >= 0) || stall_checks < 0)
    return bfail(LBM_EINVAL, "need max_steps >= 0, check_every >= 2, tol >= 0, stall_checks >= 0");
  RunParams rp{tol, (long long)max_steps, check_every, stall_checks, b->snap ? b->mpe_checks : 0, b->snap,
               9 * b->total_nodes};
  cudaError_t e = cudaMemcpyAsync(b->run_d, &rp, sizeof(rp), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && b->graph && (b->graph_acc != accelerated(b) || b->graph_threads != b->threads)) {
    // the kernel choice changed
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (e == cudaSuccess && !b->graph) {  // capture [counter reset -> persistent kernel] once
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream);
      cudaError_t e2 = launch(b, lbm::MODE_STEP, make_args(b));
      e = cudaStreamEndCapture(b->stream, &g);
      if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (e == cudaSuccess) {
      b->graph_acc = accelerated(b);
      b->graph_threads = b->threads;
    }
    if (g) cudaGraphDestroy(g);
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess && seconds) {
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
  if (e == cudaSuccess && seconds) e = cudaEventRecord(t1, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess && seconds) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, t0, t1);
    *seconds = ms * 1e-3;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_results(const lbm_batch* b, int64_t* steps, double* residual, int* status) {
  if (!b) return bfail(LBM_EINVAL, "batch is NULL");
  cudaError_t e = cudaSuccess;
  if (steps) e = cudaMemcpyAsync(steps, b->steps_d, sizeof(long long) * b->ncols, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess && residual)
    e = cudaMemcpyAsync(residual, b->resid_d, sizeof(double) * b->ncols, cudaMemcpyDeviceToHost, b->stream);
  std::vector<int> st(b->ncols);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st.data(), b->status_d, sizeof(int) * b->ncols, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  bool bad = false;
  for (int c = 0; c < b->ncols; ++c) {
    const int code = (st[c] & lbm::STATUS_NONPHYS) ? LBM_ENONPHYS : LBM_OK;
    bad |= code != LBM_OK;
    if (status) status[c] = code;
  }
  return bad ? bfail(LBM_ENONPHYS, "at least one column became non-physical") : LBM_OK;
}

int lbm_batch_column_seconds(const lbm_batch* b, double* seconds) {
  if (!b || !seconds) return bfail(LBM_EINVAL, "batch and seconds must not be NULL");
  std::vector<long long> ns(b->ncols);
  cudaError_t e = cudaMemcpyAsync(ns.data(), b->ns_d, sizeof(long long) * b->ncols, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  for (int c = 0; c < b->ncols; ++c) seconds[c] = 1e-9 * double(ns[c]);
  return LBM_OK;
}

int lbm_batch_moments(lbm_batch* b, double* rho, double* ux, double* uy, int where) {
  if (!b) return bfail(LBM_EINVAL, "batch is NULL");
  if (where != LBM_HOST && where != LBM_DEVICE) return bfail(LBM_EINVAL, "where must be LBM_HOST or LBM_DEVICE");
  const size_t bytes = size_t(b->total_nodes) * 8;
  double* d[3] = {rho, ux, uy};
  double* tmp[3] = {nullptr, nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  if (where == LBM_HOST)  // staged through freshly allocated device buffers
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
      if (d[i]) e = cudaMalloc(&tmp[i], bytes);
  BatchArgs a = make_args(b);
  a.rho_out = where == LBM_HOST ? tmp[0] : rho;
  a.ux_out = where == LBM_HOST ? tmp[1] : ux;
  a.uy_out = where == LBM_HOST ? tmp[2] : uy;
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = launch(b, lbm::MODE_MOMENTS, a);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    if (where == LBM_HOST && d[i]) e = cudaMemcpyAsync(d[i], tmp[i], bytes, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  for (double* t : tmp)
    if (t) cudaFree(t);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_rest_state(lbm_batch* b) {
  if (!b) return bfail(LBM_EINVAL, "batch is NULL");
  const BatchArgs a = make_args(b);
  const size_t smem = size_t(b->nx) * size_t(b->max_ny) * b->s;  // psi of the tallest column
  const int grid = std::min(b->ncols, 4096);
  const bool unit = unit_tau(b->p);
  void* fn;
  if (b->p.precision == LBM_FP32)
    fn = unit ? (void*)&batch_rest_kernel<float, true> : (void*)&batch_rest_kernel<float, false>;
  else if (b->p.precision == LBM_DOUBLE_FLOAT)
    fn = unit ? (void*)&batch_rest_kernel<lbm::dd, true> : (void*)&batch_rest_kernel<lbm::dd, false>;
  else
    fn = unit ? (void*)&batch_rest_kernel<double, true> : (void*)&batch_rest_kernel<double, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  void* kargs[] = {const_cast<BatchArgs*>(&a)};
  if (e == cudaSuccess) e = cudaLaunchKernel(fn, dim3(grid), dim3(256), kargs, smem, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_get_state(lbm_batch* b, double* f, int where) {
  if (!b || !f || (where != LBM_HOST && where != LBM_DEVICE)) return bfail(LBM_EINVAL, "bad batch, f or where");
  const size_t bytes = size_t(b->total_nodes) * 9 * 8;
  double* dst = f;
  cudaError_t e = cudaSuccess;
  if (where == LBM_HOST) e = cudaMalloc(&dst, bytes);
  const int g = std::min(b->ncols, 4096);
  if (e == cudaSuccess) {
    launch_typed<StateLaunch>(b->p.precision, g, b->stream, b->fA, (const BatchCol*)b->cols_d, b->ncols, b->nx, dst,
                              true);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && where == LBM_HOST) e = cudaMemcpyAsync(f, dst, bytes, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (where == LBM_HOST && dst) cudaFree(dst);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_convert(const lbm_batch* src, int precision, lbm_batch** out) {
  lbm::TraceRange trace("lbm_batch_convert");
  if (!src || !out || (precision != LBM_FP32 && precision != LBM_FP64 && precision != LBM_DOUBLE_FLOAT))
    return bfail(LBM_EINVAL, "bad arguments");
  *out = nullptr;
  // the new batch starts from src's state: absolute populations through a device buffer
  const size_t n9 = size_t(src->total_nodes) * 9;
  double* abs_d = nullptr;
  if (cudaMalloc(&abs_d, n9 * 8) != cudaSuccess) return bfail(LBM_ENOMEM, "conversion buffer");
  lbm_batch* s = const_cast<lbm_batch*>(src);
  int rc = lbm_batch_get_state(s, abs_d, LBM_DEVICE);
  std::vector<lbm_column> cols(src->ncols);
  for (int c = 0; c < src->ncols; ++c) {
    cols[c].ny = src->cols[c].ny;
    cols[c].gravity_form = src->cols[c].form;
    cols[c].T = src->cols[c].RT / src->p.R;
    cols[c].gx = src->cols[c].gx;
    cols[c].gy = src->cols[c].gy;
  }
  // rho0 placeholder: the column means (only the deviation reference uses it)
  std::vector<double> rho0(size_t(src->total_nodes));
  for (int c = 0; c < src->ncols; ++c)
    std::fill(rho0.begin() + src->cols[c].node_off, rho0.begin() + src->cols[c].node_off + src->nx * src->cols[c].ny,
              src->cols[c].rho_ref);
  lbm_params p = src->p;
  p.precision = precision;
  if (rc == LBM_OK) rc = lbm_batch_init(&p, cols.data(), src->ncols, rho0.data(), LBM_HOST, src->own_stream ? nullptr : src->stream, out);
  if (rc == LBM_OK) {
    lbm_batch* b = *out;
    b->threads = src->threads;
    size_grids(b);
    for (int c = 0; c < b->ncols; ++c) b->cols[c].rho_ref = precision == LBM_FP64 && std::isnan(src->p.rho_ref) ? 0.0 : src->cols[c].rho_ref;
    cudaError_t e = cudaMemcpyAsync(b->cols_d, b->cols.data(), sizeof(BatchCol) * b->ncols, cudaMemcpyHostToDevice, b->stream);
    const int g = std::min(b->ncols, 4096);
    if (e == cudaSuccess) {
      launch_typed<StateLaunch>(precision, g, b->stream, b->fA, (const BatchCol*)b->cols_d, b->ncols, b->nx, abs_d,
                                false);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->steps_d, src->steps_d, sizeof(long long) * b->ncols, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->ns_d, src->ns_d, sizeof(long long) * b->ncols, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
      lbm_batch_destroy(b);
      *out = nullptr;
      rc = bfail(LBM_ECUDA, cudaGetErrorString(e));
    }
  }
  cudaFree(abs_d);
  return rc;
}

int lbm_batch_destroy(lbm_batch* b) {
  if (b && b->stream) cudaStreamSynchronize(b->stream);
  free_batch(b);
  return LBM_OK;
}

}  // extern "C"
