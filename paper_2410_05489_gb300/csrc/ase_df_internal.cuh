// Internal declarations shared by the CUDA translation units of the ASE-DF library.
//
// Method (arXiv 2410.05489): per face, adaptive stencil extension (Sec. 3, Algorithm 1)
// driven by the discontinuity feedback factor (Sec. 3.1, Eq. 3.2), WENOZ-AO(5,3) with DF
// damping as the fallback (Sec. 3.2), Gauss-point states (Sec. 2.1), local
// Lax-Friedrichs flux and discontinuity strength per Gauss point (Sec. 2.3, Sec. 3.1),
// flux difference (Sec. 2.1, Eq. 2.3) and SSP-RK3 (Sec. 2.3).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ase_df.h"

namespace asedf {

// Raises a kernel's dynamic shared-memory limit once per device (the attribute belongs to
// the function on the current device): `done` holds one bit per device ordinal (< 64) for
// which it is set.  Safe to call from several host threads.
template <typename Kernel>
inline cudaError_t ensure_smem_limit(Kernel kern, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit != 0ull && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && bit != 0ull) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Streaming multiprocessors of the current device (cached per device ordinal < 64).
inline int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 152;
  if (dev < 64) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

// Evaluation points of a reconstruction polynomial on its cell [-1, 0]:
//   0: xi = 0 (the "plus" face), 1: xi = -1 (the "minus" face), 2..: Gauss points.
constexpr int kMaxPts = 6;

// Reconstruction tables of one scheme order, built on the host by exact rational
// inversion of the cell-average moment problem (see ase_df_tables.cpp).
struct Tables {
  // lin[b][p][t]: weight of W_{t-4} in the value at point p of the linear polynomial of
  // the centred (2b+3)-cell stencil (b = 0..3 for 3, 5, 7, 9 cells).
  double lin[4][kMaxPts][9];
  // sub[k][p][j]: weight of the j-th cell (offsets k-2+j) of sub-stencil S3_{k-1} in its
  // undamped quadratic's value at point p.
  double sub[3][kMaxPts][3];
  // cq[k][q][j]: coefficient of xi^(q+1) of that quadratic (for the smoothness indicator).
  double cq[3][2][3];
  double gw[4];   // Gauss weights on [0, 1]
  double hgw[4];  // gw / 2 (the 1/2 of the Lax-Friedrichs flux folded in)
  // symmetric Gauss-point pairs of the order-r linear branch: for the point pair
  // (eta_g, -1 - eta_g), g < G/2, value = E +- O with E = se[g][0] W_0 + sum_t se[g][t] (W_t + W_-t)
  // and O = sum_t so[g][t] (W_t - W_-t), t = 1..k; the middle point of odd G uses se only.
  double se[2][5];
  double so[2][5];
  double d5, d3[3];  // linear weights of WENOZ-AO(5,3) (Sec. 3.2, d_Hi = d_Lo = 0.85)
  double eps;        // 1e-6 (Sec. 3.2)
};

// Derivative weights (d/dxi) of the same polynomials at the same points, for the
// gas-kinetic flux (which needs the slopes of the reconstructed states).
struct DTables {
  double dlin[4][kMaxPts][9];
  double dsub[3][kMaxPts][3];
};

// Positivity repair of a stage update (the paper's transition to first order for
// positivity): at most this many passes per RK stage.
constexpr int kRepairPasses = 8;

// Device-resident solver status.
struct DevState {
  unsigned long long max_speed_bits;  // atomicMax over the bit patterns of non-negative doubles
  double dt;        // the step of the current SSP-RK3 step
  double t;         // time
  double last_dt;
  unsigned int flags;
  unsigned int pad;
  // cnt[0]: cells the stage update left non-physical; cnt[p]: cells newly non-physical
  // after repair pass p.  Cleared by the x-face sweep of every stage.
  unsigned int cnt[kRepairPasses + 1];
  // rbad[p]: cells still non-physical after repair pass p (marked before or not).
  unsigned int rbad[kRepairPasses + 1];
  unsigned long long repaired_total;  // cells marked by the repair since the last reset
  unsigned long long frozen_total;    // cells left without a flux update (last resort)
  // Branch histogram of the sweeps (ase_df_hist_*): per face and side, the branch of
  // Algorithm 1 taken by the normal and (2D) the tangential reconstruction, and the Gauss
  // points that took first-order states; slots as kBranchSlots.
  unsigned long long hist[8];
  // Grid barrier of the single-launch repair (repair_all_kernel): arrivals and generation.
  // bar_count is 0 between barriers; ase_df_reset clears both.
  unsigned int bar_count, bar_gen;
};

// Slots of the branch histogram: linear 9th, 7th, 5th order, WENOZ-AO(5,3)+DF, linear 3rd
// order, DF-damped 3rd order, first-order Gauss point.
constexpr int kBranchSlots = 7;

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW_BAND = 2, BC_REFLECT = 3, BC_WALL_AFTER = 4, BC_MOVING_SHOCK = 5 };

// Grid and boundary description handed to the kernels.
struct GridInfo {
  int nx, ny;         // cells (ny = 1 in 1D)
  int bc[4];          // x-lo, x-hi, y-lo, y-hi
  int band_j0, band_j1;  // rows whose ghost cells at x < 0 take the inflow state
  double inflow_cons[4];
  double gamma;
  double gm1, gg1;    // gamma - 1 and gamma (gamma - 1), for the flux kernels
  double gm1_hgw[4] = {0.0, 0.0, 0.0, 0.0};  // (gamma - 1) x half Gauss weight of each point
  double thres;
  // BC_WALL_AFTER (y-lo): columns i < wall_i0 (centre x below wall_x) have fixed ghosts
  int wall_i0 = 0;
  // BC_MOVING_SHOCK (y-hi): ghost centre x0 + (i + 1/2) dx below shock_x0 + shock_speed t
  // takes inflow_cons, otherwise state_b_cons
  double x0 = 0.0, dx = 0.0, shock_x0 = 0.0, shock_speed = 0.0;
  double state_b_cons[4] = {0.0, 0.0, 0.0, 0.0};
};

struct SweepArgs {
  const double* W;        // [C][ny][nx]
  const double* s_norm;   // sigma of the faces normal to the sweep
  const double* s_tan;    // sigma of the faces along the sweep lines (2D)
  double* F;              // face fluxes of this direction
  double* s_out;          // sigma_out of this direction
  DevState* st;
  double tfrac = 0.0;     // the stage's time is st->t + tfrac st->dt (time-dependent ghosts)
  unsigned long long* hist = nullptr;  // branch histogram (kBranchSlots counters) or nullptr
};

struct CombineArgs {
  unsigned char* mark;  // per cell: 0, or the pass (1..) in which it was found non-physical
  const double* Fx;   // [C][ny][nx+1]
  const double* Fy;   // [C][ny+1][nx] (2D)
  const double* Wn;   // W^n
  const double* Ws;   // stage input W^(s)
  double* out;        // W^(s+1) (or L for stage 0)
  DevState* st;
  double inv_dx, inv_dy;
  double dt_fixed;    // > 0: this dt; otherwise the CFL dt (stage 1 computes it)
  double cfl, t_end, inflow_speed;
  int stage;          // 0: out = L; 1, 2, 3: SSP-RK3 stages
};

struct RepairArgs {
  unsigned char* mark;
  const double* Fx;
  const double* Fy;
  const double* Wn;
  const double* Ws;
  double* out;
  double* sx_out;     // sigma of the stage (faces switched to first order get 1e30)
  double* sy_out;
  DevState* st;
  double inv_dx, inv_dy;
  double dt_fixed;
  int stage;
  int pass;           // 1..kRepairPasses
  double tfrac = 0.0; // the stage's time is st->t + tfrac dt (time-dependent ghosts)
};

struct SpeedArgs {
  const double* W;
  DevState* st;
  double inv_dx, inv_dy;
};

// Sets g.gm1_hgw from the tables of the problem's order (call after g.gm1 and the tables
// are known).
inline void set_flux_weights(GridInfo& g, const Tables& t) {
  for (int q = 0; q < 4; ++q) g.gm1_hgw[q] = g.gm1 * t.hgw[q];
}

// A validated problem and what the kernels derive from it; shared by ase_df_init and
// ase_df_residual_noalloc, so that both accept the same problems and describe them to the
// kernels identically.
struct ProblemSetup {
  ase_df_params p;       // normalised: ny = 1 and outflow y-sides in 1D
  int C, K;              // components, stencil half-width (r - 1) / 2
  double dx, dy, inv_dx, inv_dy;
  double inflow_speed;   // (|u|+c)/dx (+ (|v|+c)/dy) of the inflow band's state, else 0
  GridInfo g;
};

// Validates *p and fills *out (host arithmetic only, no allocation).  On failure returns
// the status and writes a message into err[0 .. err_len) (err may be NULL).
ase_df_status setup_problem(const ase_df_params* p, ProblemSetup* out, char* err, size_t err_len);

// The process-wide message buffer that ase_df_last_error(NULL) returns (512 bytes).
char* init_error_buffer();

// Host-side launchers, one set per scheme order (ase_df_sweep.cu is compiled once per
// order).  dim = 1 or 2; dir = 0 (x-faces) or 1 (y-faces).
cudaError_t launch_sweep_r3(int dim, int dir, const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s);
cudaError_t launch_sweep_r5(int dim, int dir, const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s);
cudaError_t launch_sweep_r7(int dim, int dir, const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s);
cudaError_t launch_sweep_r9(int dim, int dir, const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s);

cudaError_t launch_combine(int dim, const GridInfo& g, const CombineArgs& a, cudaStream_t s);
cudaError_t launch_max_speed(int dim, const GridInfo& g, const SpeedArgs& a, cudaStream_t s);
// All repair passes and the freeze of one stage in one cooperative launch (returns at once
// when the stage update was physical everywhere; a grid barrier between passes).
cudaError_t launch_repair_all(int dim, const GridInfo& g, const RepairArgs& a, cudaStream_t s);
// A grid barrier that cannot complete (self-test of the bounded wait): raises
// ASE_DF_FLAG_SYNC after about a second, then clears the barrier's arrival count.
cudaError_t launch_wait_selftest(DevState* st, cudaStream_t s);
cudaError_t launch_state_kernel(DevState* st, int op, double t, cudaStream_t s);

// Tables of scheme order r (host, exact rational arithmetic, no allocation); false only if a
// moment matrix were singular, which the fixed stencils rule out.
bool build_tables(int r, int ndim, Tables* out);
bool build_dtables(int r, int ndim, DTables* out);

}  // namespace asedf
