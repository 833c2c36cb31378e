// Internal declarations shared by the host API (lbm_api.cu) and the kernels
// (lbm_kernels.cu) of liblbm. Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "lbm.h"

namespace lbm {

// Sticky device status bits (OR-ed by kernels, mapped to LBM_E* on the host).
enum : int { STATUS_NONPHYS = 1, STATUS_TIMEOUT = 2 };

// Physical constants of one step, FP64 masters (converted to the kernel's real type).
struct StepPhys {
  double rho_ref;          // populations are stored as g_i = f_i - w_i rho_ref
  double RT, R, a, b;      // Eq. EOS: R T, R, a, b
  double G;                // Eqs. ShanChenForce / InteractionPotential
  double s_e, s_vs, s_j, s_q, s_nu;   // diagonal of Lambda (Eq. RelaxationMatrix): 1/tau
  double sig_e, sig_vs;    // sigma/(tau_e - 1/2), sigma/(tau_varsigma - 1/2) of Eq. LiFS
  double gx, gy;           // gravity
  int form;                // 1: rho g (Eq. Gravity_1), 2: (rho - <rho>) g (Eq. Gravity_2)
  int wall;                // LBM_WALL_BOUNCE_BACK or LBM_WALL_ZOU_HE
};

// Tiling of the fused step: CTA b covers band (b % nbands) of width band_w along x
// and strip (b / nbands) of strip_h rows, counted from row y_begin.
struct StepTiling {
  int nx, ny;                // buffer rows and columns (the state is real[9][ny][nx])
  int band_w, nbands, strip_h, nstrips;
  int threads, smem_bytes;
  int variant;               // index into the kernel's tile variants (0 = default)
  // Rows the step collides and writes: [y_begin, y_end). Rows ylo and yhi are the wall
  // rows (halfway bounce-back beyond them, Zou-He on them, no Shan-Chen force there);
  // a buffer row outside [ylo, yhi] is never read. A whole domain: 0, ny, 0, ny - 1. A
  // slab of a larger domain with ghost rows: its own rows, and ylo / yhi at its own first /
  // last row where it meets a wall, else at the buffer's edge (the ghost rows are read,
  // not written).
  int y_begin, y_end, ylo, yhi;
  double n_total;            // nodes of the whole domain: <rho> = (sum of rho) / n_total
};

enum StepMode : int { MODE_STEP = 0, MODE_MOMENTS = 1 };

struct StepIO {
  const void* fin;         // real[9][ny][nx], state after the previous step
  void* fout;              // real[9][ny][nx], state after this step (MODE_STEP)
  const double* part_in;   // FP64 partial sums of sum_i g_i of fin, npart_in entries
  int npart_in;
  double* part_out;        // one FP64 partial per CTA of sum_i g_i of fout (MODE_STEP)
  int* status;             // sticky device status word
  double* rho_out;         // MODE_MOMENTS outputs, [y][x] doubles (may be NULL); thermal FP64
  double* ux_out;          // MODE_STEP: this step's rho, u for the energy equation (required)
  double* uy_out;
  float* rho32;            // thermal FP32 MODE_STEP (barrier-free tile): this step's rho, u as
  float* ux32;             // floats, [y][x] (required there, unused elsewhere)
  float* uy32;
  const void* Tfield;      // thermal variant: real[ny][nx] temperature (NULL: uniform T)
};

// ---- launch wrappers (lbm_kernels.cu). All are asynchronous on `stream`.
int stages(int precision, int variant);  // pipeline depth (rows in shared memory) of a tile variant
int step_num_variants(int precision);
// has the thermal and Zou-He wall kernels (io.Tfield set, StepPhys::wall = LBM_WALL_ZOU_HE)
bool step_variant_extended(int precision, int variant);
// widest x band one CTA covers, threads per CTA, dynamic shared bytes of a tile variant
bool step_variant_info(int precision, int variant, int* band_w, int* threads, int* smem);
int step_max_ctas_per_sm(int precision, int variant, int threads, int smem_bytes);
cudaError_t step_prepare(int precision);  // sets the dynamic shared memory limit
cudaError_t launch_step(int precision, int mode, const StepTiling& t, const StepPhys& ph,
                        const StepIO& io, cudaStream_t stream);

// initial state and the FP64 partial sums of its stored values into part[0..npart)
cudaError_t launch_init(int precision, const double* rho0, void* f, int nx, int ny, double rho_ref, double* part,
                        int npart, cudaStream_t stream);
cudaError_t launch_partials(int precision, const void* f, int nx, int ny, double* part, int npart,
                            cudaStream_t stream);
// out[0] = sum of part[0..npart) in a fixed order
cudaError_t launch_sum_partials(const double* part, int npart, double* out, cudaStream_t stream);
// one population plane of n values: out = plane + add / plane = in - sub
cudaError_t launch_plane_to_double(int precision, const void* plane, double* out, size_t n, double add,
                                   cudaStream_t stream);
cudaError_t launch_plane_from_double(int precision, const double* in, void* plane, size_t n, double sub,
                                     cudaStream_t stream);
// max |a - b| over n (b may be NULL: max |a|); max sqrt(ux^2+uy^2)
cudaError_t launch_max_abs_diff(const double* a, const double* b, size_t n, double* out, cudaStream_t stream);
cudaError_t launch_max_speed(const double* ux, const double* uy, size_t n, double* out, cudaStream_t stream);
cudaError_t launch_row_means(const double* rho, int nx, int ny, double* rowmean, cudaStream_t stream);
// out[0] = first crossing height of rowmean through level (NaN if none); out[1] = max; out[2] = min
cudaError_t launch_profile_scan(const double* rowmean, int ny, double level, double* out, cudaStream_t stream);

// ---- thermal variant (lbm_thermal.cu): Eq. Energy_Equation on a real[ny][nx] field
// One Heun step in one launch: Tout = Tin + (k1 + k2)/2 with k1 = L(Tin), k2 = L(Tin + k1),
// rho, ux, uy ([y][x] real: float for precision 1, double for 2) held fixed. Tin and Tout
// are distinct real[ny][nx] fields. wall_nodes: rows 0 and ny - 1 keep their temperature
// (Zou-He walls); else wall ghosts.
cudaError_t launch_energy_step(int precision, int nx, int ny, int wall_nodes, double R, double b, double c_v,
                               double kappa, double T_bot, double T_top, const void* rho, const void* ux,
                               const void* uy, const void* Tin, void* Tout, cudaStream_t stream);
// Tf = T_bot + (T_top - T_bot)(y + 1/2)/ny, or T_bot + (T_top - T_bot) y/(ny - 1) with wall nodes
cudaError_t launch_linear_T(int precision, int nx, int ny, double T_bot, double T_top, int wall_nodes, void* Tf,
                            cudaStream_t stream);

// ---- NVTX range over the rest of a host scope (init, step, moments, reductions, state I/O,
// batch runs): named intervals on a profiler's timeline, no cost without a tool attached
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// ---- host helpers of lbm_api.cu shared with other entry points (same behaviour as lbm_init's)
int validate_params(const lbm_params* p, char* err);  // err: 512 bytes
StepPhys phys_from_params(const lbm_params& p, double rho_ref);
// step_prepare once per device and precision (thread-safe; a failure is not remembered):
// every grid plan needs it first, since the occupancy query depends on the limit it sets
int prepare_step_kernels(int dev, int precision, char* err);
// resident step CTAs per SM of a tile variant on the current device (at least 1), asked
// once per device, precision and variant after prepare_step_kernels
int step_ctas_per_sm(int precision, int variant, int threads, int smem_bytes, int* per_sm, char* err);
int plan_step_tiling(const lbm_params& p, int nsm, StepTiling* t, char* err);  // default variant
void set_last_error(const char* msg);  // text returned by lbm_last_error(NULL)

}  // namespace lbm
