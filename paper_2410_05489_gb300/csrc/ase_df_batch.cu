// Batched solves: many independent 1D/2D problems of mixed order, advanced together.
//
// One persistent launch per sweep direction per RK stage serves every tile of every
// problem: CTAs (a chosen number per SM) pull work items (problem, tile) from a list
// ordered by cost (largest tiles first) through an atomic counter and run the same
// fused face-sweep tile as the one-problem kernel, dispatching on the problem's order
// and dimension.  The flux difference / SSP-RK3 combination, the positivity repair and
// the CFL reduction run over lists of cell chunks, each chunk belonging to one problem;
// every problem has its own device status (CFL dt, time, flags).  A whole step is
// captured once into a CUDA graph and replayed (ase_df_batch_run).  The schedule (CTAs
// per SM for the sweeps, item ordering, chunk size) is set by ase_df_batch_set_schedule;
// the Python package's autotuner times the candidates and caches the choice per device.
//
// Memory: the caller owns the packed state arrays (layout from ase_df_batch_layout);
// the batch owns the packed scratch (RK stage states, face fluxes, sigma ping-pong,
// repair marks), the problem descriptors and the work lists.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ase_df.h"
#include "ase_df_combine_body.cuh"
#include "ase_df_sweep_body.cuh"

namespace asedf {
namespace {

// Device descriptor of one problem of a batch.
struct BatchProblem {
  GridInfo g;
  int ndim, variant;        // variant = (ndim - 1) * 4 + (order - 3) / 2
  long long w_off, sx_off, sy_off, fx_off, fy_off, cell_off;
  double inv_dx, inv_dy, cfl, t_end, inflow_speed;
};

// Base pointers of the packed arrays of one launch.
struct BatchPtrs {
  double *W, *sx, *sy;                       // caller's packed state and sigma
  double *W1, *W2, *sxa, *sya, *sxb, *syb;   // scratch, same layouts as W / sx / sy
  double *zsx, *zsy;                         // zero sigma (priming)
  double *Fx, *Fy;
  unsigned char* mark;
};

struct StagePtrs {
  const double *Ws, *sxin, *syin;
  double *sxout, *syout, *out;
};

// Stage 0 = priming (sigma from zero sigma), 1..3 = SSP-RK3 stages.
__device__ __forceinline__ StagePtrs stage_ptrs(const BatchPtrs& P, const BatchProblem& pb, int stage) {
  StagePtrs s;
  const long long w = pb.w_off, x = pb.sx_off, y = pb.sy_off;
  if (stage == 0) {
    s.Ws = P.W + w; s.sxin = P.zsx + x; s.syin = P.zsy + y; s.sxout = P.sx + x; s.syout = P.sy + y; s.out = nullptr;
  } else if (stage == 1) {
    s.Ws = P.W + w; s.sxin = P.sx + x; s.syin = P.sy + y; s.sxout = P.sxa + x; s.syout = P.sya + y; s.out = P.W1 + w;
  } else if (stage == 2) {
    s.Ws = P.W1 + w; s.sxin = P.sxa + x; s.syin = P.sya + y; s.sxout = P.sxb + x; s.syout = P.syb + y; s.out = P.W2 + w;
  } else {
    s.Ws = P.W2 + w; s.sxin = P.sxb + x; s.syin = P.syb + y; s.sxout = P.sx + x; s.syout = P.sy + y; s.out = P.W + w;
  }
  return s;
}

constexpr int kNT = 256;

// One out-of-line copy per variant (order, dimension, direction, tile lines), so that each
// gets its own register allocation.
template <int R, int DIM, int DIR, int TT = (DIM == 2) ? 64 : 1>
__device__ __noinline__ void tile_call(const GridInfo& g, const SweepArgs& a, const Tables& T, int a0, int b0,
                                       double* smem) {
  sweep_tile<R, DIM, DIR, TT>(g, a, T, a0, b0, TT, smem);
}

// 2D tile of 8 faces x tt lines (64: two faces per thread, 32: one)
template <int R, int DIR>
__device__ __forceinline__ void tile_call_2d(int tt, const GridInfo& g, const SweepArgs& a, const Tables& T, int a0,
                                             int b0, double* smem) {
  if (tt == 32) tile_call<R, 2, DIR, 32>(g, a, T, a0, b0, smem);
  else tile_call<R, 2, DIR, 64>(g, a, T, a0, b0, smem);
}

template <int DIR>
__global__ void __launch_bounds__(kNT, 2)
batch_sweep_kernel(const BatchProblem* __restrict__ probs, const int4* __restrict__ items, int nitems,
                   unsigned int* counter, const BatchPtrs P, int stage, const Tables* __restrict__ tabs,
                   DevState* states) {
  extern __shared__ double smem[];
  __shared__ Tables sT;
  __shared__ int s_item[2];  // the current work item and the next one (fetched during the tile)
  __shared__ int s_variant;
  if (threadIdx.x == 0) {
    s_variant = -1;
    s_item[0] = (int)atomicAdd(counter, 1u);
  }
  int k = 0;
  while (true) {
    // the previous tile is done with smem, and s_item[k] holds this tile's item (written by
    // thread 0 before this barrier, after every thread had read the slot's previous value)
    __syncthreads();
    const int it = s_item[k];
    if (it >= nitems) break;
    if (threadIdx.x == 0) s_item[k ^ 1] = (int)atomicAdd(counter, 1u);  // read after the next barrier
    k ^= 1;
    const int4 w = items[it];  // problem, a0, b0, lines of a 2D tile
    const BatchProblem& pb = probs[w.x];
    const int variant = pb.variant;
    if (variant != s_variant) {  // stage this order's tables in shared memory
      const double* src = reinterpret_cast<const double*>(tabs + variant);
      double* dst = reinterpret_cast<double*>(&sT);
      for (int e = threadIdx.x; e < (int)(sizeof(Tables) / sizeof(double)); e += kNT) dst[e] = src[e];
      __syncthreads();
      if (threadIdx.x == 0) s_variant = variant;
      __syncthreads();
    }
    const StagePtrs sp = stage_ptrs(P, pb, stage);
    SweepArgs a;
    a.W = sp.Ws;
    a.s_norm = (DIR == 0) ? sp.sxin : sp.syin;
    a.s_tan = (DIR == 0) ? sp.syin : sp.sxin;
    a.F = (DIR == 0) ? P.Fx + pb.fx_off : P.Fy + pb.fy_off;
    a.s_out = (DIR == 0) ? sp.sxout : sp.syout;
    a.st = states + w.x;
    if (DIR == 0 && w.y == 0 && w.z == 0 && threadIdx.x <= kRepairPasses) {
      a.st->cnt[threadIdx.x] = 0u;  // repair counters of this problem's stage
      a.st->rbad[threadIdx.x] = 0u;
    }
    const GridInfo g = pb.g;
    if (DIR == 0) {
      switch (variant) {
        case 0: tile_call<3, 1, 0>(g, a, sT, w.y, w.z, smem); break;
        case 1: tile_call<5, 1, 0>(g, a, sT, w.y, w.z, smem); break;
        case 2: tile_call<7, 1, 0>(g, a, sT, w.y, w.z, smem); break;
        case 3: tile_call<9, 1, 0>(g, a, sT, w.y, w.z, smem); break;
        case 4: tile_call_2d<3, 0>(w.w, g, a, sT, w.y, w.z, smem); break;
        case 5: tile_call_2d<5, 0>(w.w, g, a, sT, w.y, w.z, smem); break;
        case 6: tile_call_2d<7, 0>(w.w, g, a, sT, w.y, w.z, smem); break;
        default: tile_call_2d<9, 0>(w.w, g, a, sT, w.y, w.z, smem); break;
      }
    } else {
      switch (variant) {
        case 4: tile_call_2d<3, 1>(w.w, g, a, sT, w.y, w.z, smem); break;
        case 5: tile_call_2d<5, 1>(w.w, g, a, sT, w.y, w.z, smem); break;
        case 6: tile_call_2d<7, 1>(w.w, g, a, sT, w.y, w.z, smem); break;
        default: tile_call_2d<9, 1>(w.w, g, a, sT, w.y, w.z, smem); break;
      }
    }
  }
}

// chunk = (problem, first cell, last cell, -)
__global__ void __launch_bounds__(256) batch_combine_kernel(const BatchProblem* __restrict__ probs,
                                                            const int4* __restrict__ chunks, int nchunks,
                                                            const BatchPtrs P, int stage, DevState* states) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int4 ch = chunks[c];
    const BatchProblem& pb = probs[ch.x];
    const StagePtrs sp = stage_ptrs(P, pb, stage);
    CombineArgs a;
    a.mark = P.mark + pb.cell_off;
    a.Fx = P.Fx + pb.fx_off;
    a.Fy = P.Fy + pb.fy_off;
    a.Wn = P.W + pb.w_off;
    a.Ws = sp.Ws;
    a.out = sp.out;
    a.st = states + ch.x;
    a.inv_dx = pb.inv_dx;
    a.inv_dy = pb.inv_dy;
    a.dt_fixed = 0.0;
    a.cfl = pb.cfl;
    a.t_end = pb.t_end;
    a.inflow_speed = pb.inflow_speed;
    a.stage = stage;
    const bool leader = (ch.y == 0 && threadIdx.x == 0);
    if (pb.ndim == 1) combine_range<1>(pb.g, a, (size_t)ch.y + threadIdx.x, (size_t)ch.z, blockDim.x, leader);
    else combine_range<2>(pb.g, a, (size_t)ch.y + threadIdx.x, (size_t)ch.z, blockDim.x, leader);
  }
}

__device__ __forceinline__ RepairArgs repair_args(const BatchPtrs& P, const BatchProblem& pb, int stage, int pass,
                                                  DevState* st) {
  const StagePtrs sp = stage_ptrs(P, pb, stage);
  RepairArgs r;
  r.mark = P.mark + pb.cell_off;
  r.Fx = P.Fx + pb.fx_off;
  r.Fy = P.Fy + pb.fy_off;
  r.Wn = P.W + pb.w_off;
  r.Ws = sp.Ws;
  r.out = sp.out;
  r.sx_out = sp.sxout;
  r.sy_out = sp.syout;
  r.st = st;
  r.inv_dx = pb.inv_dx;
  r.inv_dy = pb.inv_dy;
  r.dt_fixed = 0.0;
  r.stage = stage;
  r.pass = pass;
  return r;
}

__global__ void __launch_bounds__(256) batch_repair_kernel(const BatchProblem* __restrict__ probs,
                                                           const int4* __restrict__ chunks, int nchunks,
                                                           const BatchPtrs P, int stage, int pass, DevState* states) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int4 ch = chunks[c];
    const BatchProblem& pb = probs[ch.x];
    const RepairArgs r = repair_args(P, pb, stage, pass, states + ch.x);
    if (pass > 0) {
      if (pb.ndim == 1) repair_range<1>(pb.g, r, (size_t)ch.y + threadIdx.x, (size_t)ch.z, blockDim.x);
      else repair_range<2>(pb.g, r, (size_t)ch.y + threadIdx.x, (size_t)ch.z, blockDim.x);
    } else {  // pass 0: the last resort
      if (pb.ndim == 1) freeze_range<1>(pb.g, r, (size_t)ch.y + threadIdx.x, (size_t)ch.z, blockDim.x);
      else freeze_range<2>(pb.g, r, (size_t)ch.y + threadIdx.x, (size_t)ch.z, blockDim.x);
    }
  }
}

__global__ void __launch_bounds__(256) batch_max_speed_kernel(const BatchProblem* __restrict__ probs,
                                                              const int4* __restrict__ chunks, int nchunks,
                                                              const BatchPtrs P, DevState* states) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int4 ch = chunks[c];
    const BatchProblem& pb = probs[ch.x];
    SpeedArgs a;
    a.W = P.W + pb.w_off;
    a.st = states + ch.x;
    a.inv_dx = pb.inv_dx;
    a.inv_dy = pb.inv_dy;
    if (pb.ndim == 1) max_speed_range<1>(pb.g, a, (size_t)ch.y + threadIdx.x, (size_t)ch.z, blockDim.x);
    else max_speed_range<2>(pb.g, a, (size_t)ch.y + threadIdx.x, (size_t)ch.z, blockDim.x);
  }
}

// Work counters of the step's sweep launches and the CFL maxima of every problem.
__global__ void batch_reset_kernel(unsigned int* counters, int ncounters, DevState* states, int nprob, int full) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncounters) counters[i] = 0u;
  if (i < nprob) {
    states[i].max_speed_bits = 0ull;
    if (full) {
      states[i].flags = 0u;
      states[i].t = 0.0;
      states[i].dt = 0.0;
      states[i].last_dt = 0.0;
      states[i].repaired_total = 0ull;
      states[i].frozen_total = 0ull;
    }
  }
}

}  // namespace
}  // namespace asedf

using namespace asedf;

struct ase_df_batch {
  int n = 0;
  int nsm = 0;
  int any2d = 0;
  std::vector<ase_df_params> params;
  std::vector<long long> w_off, sx_off, sy_off, fx_off, fy_off, cell_off;
  std::vector<int4> items_x, items_y;  // host copies (cost order)
  std::vector<long long> item_cost_x, item_cost_y;
  BatchProblem* d_prob = nullptr;
  DevState* d_state = nullptr;
  Tables* d_tabs = nullptr;
  int4* d_items_x = nullptr;
  int4* d_items_y = nullptr;
  int4* d_chunks = nullptr;
  int nchunks = 0;
  unsigned int* d_counters = nullptr;  // [8]: prime x/y, stages 1..3 x/y
  BatchPtrs P{};
  size_t smem_bytes = 0;
  // schedule
  int ctas_per_sm = 2, order_by_cost = 1, chunk_cells = 16384;
  int tile_lines[4] = {64, 64, 64, 64};  // lines of the 2D tiles of orders 3, 5, 7, 9
  // graph of one step
  cudaGraphExec_t graph = nullptr;
  double *g_W = nullptr, *g_sx = nullptr, *g_sy = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  char err[512] = "";
};

static char g_batch_err[512] = "";

static ase_df_status bfail(ase_df_batch* b, ase_df_status s, const char* fmt, ...) {
  char* dst = b ? b->err : g_batch_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return s;
}

static ase_df_status bcuda(ase_df_batch* b, cudaError_t e, const char* where) {
  return bfail(b, ASE_DF_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Validation of one problem, as ase_df_init does it.
static bool valid_problem(ase_df_params& p, char* why, size_t nwhy) {
  if (p.ndim != 1 && p.ndim != 2) { snprintf(why, nwhy, "ndim must be 1 or 2"); return false; }
  if (p.order != 3 && p.order != 5 && p.order != 7 && p.order != 9) { snprintf(why, nwhy, "bad order"); return false; }
  if (p.ndim == 1) p.ny = 1;
  if (p.nx < 1 || p.ny < 1 || p.nx > (1 << 20) || p.ny > (1 << 20)) { snprintf(why, nwhy, "bad grid size"); return false; }
  if (!(p.x1 > p.x0) || (p.ndim == 2 && !(p.y1 > p.y0))) { snprintf(why, nwhy, "empty domain"); return false; }
  if (!(p.gamma > 1.0) || !(p.sigma_thres > 0.0) || !(p.cfl > 0.0)) { snprintf(why, nwhy, "bad gamma / sigma_thres / cfl"); return false; }
  for (int s = 0; s < 4; ++s) {
    if (p.bc[s] < 0 || p.bc[s] > 3 || (p.bc[s] == ASE_DF_BC_INFLOW_BAND && s != 0)) { snprintf(why, nwhy, "bad boundary code"); return false; }
    if (p.ndim == 1 && s >= 2) p.bc[s] = ASE_DF_BC_OUTFLOW;
  }
  const int64_t need = (p.order + 1) / 2;
  if (((p.bc[0] == ASE_DF_BC_REFLECT || p.bc[1] == ASE_DF_BC_REFLECT) && p.nx < need) ||
      (p.ndim == 2 && (p.bc[2] == ASE_DF_BC_REFLECT || p.bc[3] == ASE_DF_BC_REFLECT) && p.ny < need)) {
    snprintf(why, nwhy, "a reflecting wall needs (order+1)/2 cells in its direction");
    return false;
  }
  if ((p.bc[0] == ASE_DF_BC_PERIODIC) != (p.bc[1] == ASE_DF_BC_PERIODIC) ||
      (p.ndim == 2 && (p.bc[2] == ASE_DF_BC_PERIODIC) != (p.bc[3] == ASE_DF_BC_PERIODIC))) {
    snprintf(why, nwhy, "periodic boundaries must come in pairs");
    return false;
  }
  if (p.bc[0] == ASE_DF_BC_INFLOW_BAND && !(p.inflow_state[0] > 0.0 && p.inflow_state[3] > 0.0)) {
    snprintf(why, nwhy, "inflow state must have rho > 0 and p > 0");
    return false;
  }
  return true;
}

static void fill_grid(const ase_df_params& p, BatchProblem& d) {
  std::memset(&d, 0, sizeof(d));
  const int C = (p.ndim == 1) ? 3 : 4;
  GridInfo& g = d.g;
  g.nx = (int)p.nx;
  g.ny = (int)p.ny;
  for (int s = 0; s < 4; ++s) g.bc[s] = p.bc[s];
  g.band_j0 = 1;
  g.band_j1 = 0;
  const double dx = (p.x1 - p.x0) / (double)p.nx;
  const double dy = (p.ndim == 2) ? (p.y1 - p.y0) / (double)p.ny : 1.0;
  d.inv_dx = 1.0 / dx;
  d.inv_dy = (p.ndim == 2) ? 1.0 / dy : 0.0;
  if (p.bc[0] == ASE_DF_BC_INFLOW_BAND) {
    int j0 = -1, j1 = -2;
    for (int j = 0; j < g.ny; ++j) {
      const double yc = p.y0 + ((double)j + 0.5) * dy;
      if (yc > p.inflow_lo && yc < p.inflow_hi) {
        if (j0 < 0) j0 = j;
        j1 = j;
      }
    }
    if (j0 >= 0) { g.band_j0 = j0; g.band_j1 = j1; }
    const double rho = p.inflow_state[0], u = p.inflow_state[1], v = p.inflow_state[2], pr = p.inflow_state[3];
    g.inflow_cons[0] = rho;
    g.inflow_cons[1] = rho * u;
    if (C == 4) {
      g.inflow_cons[2] = rho * v;
      g.inflow_cons[3] = pr / (p.gamma - 1.0) + 0.5 * rho * (u * u + v * v);
    } else {
      g.inflow_cons[2] = pr / (p.gamma - 1.0) + 0.5 * rho * u * u;
    }
    const double c = std::sqrt(p.gamma * pr / rho);
    d.inflow_speed = (std::fabs(u) + c) * d.inv_dx + (p.ndim == 2 ? (std::fabs(v) + c) * d.inv_dy : 0.0);
  }
  g.gamma = p.gamma;
  g.gm1 = p.gamma - 1.0;
  g.gg1 = p.gamma * (p.gamma - 1.0);
  g.thres = p.sigma_thres;
  d.ndim = p.ndim;
  d.variant = (p.ndim - 1) * 4 + (p.order - 3) / 2;
  d.cfl = p.cfl;
  d.t_end = p.t_end;
}

// Relative FP64 cost of one face of a sweep tile (the algorithmic flops per face).
static long long face_cost(int ndim, int r) {
  const int C = (ndim == 2) ? 4 : 3;
  const int G = (ndim == 2) ? (r == 3 ? 1 : (r - 1) / 2) : 1;
  const int phi = (ndim == 2) ? 70 : 54;
  return 2LL * C * (2 * r - 1) + (ndim == 2 ? 2LL * C * G * (2 * r - 1) : 0) + G * (phi + 2 * C + 1) + 1;
}

static void build_items(ase_df_batch* b) {
  b->items_x.clear();
  b->items_y.clear();
  std::vector<std::pair<long long, int4>> wx, wy;
  for (int i = 0; i < b->n; ++i) {
    const ase_df_params& p = b->params[i];
    const long long fc = face_cost(p.ndim, p.order);
    if (p.ndim == 1) {
      const int TN = Tile<3, 1>::TN;
      for (long long a0 = 0; a0 <= p.nx; a0 += TN) {
        const long long nf = std::min<long long>(TN, p.nx + 1 - a0);
        wx.push_back({fc * nf, make_int4(i, (int)a0, 0, 0)});
      }
    } else {
      const int TN = Tile<3, 2>::TN, TT = b->tile_lines[(p.order - 3) / 2];
      for (long long b0 = 0; b0 < p.ny; b0 += TT)
        for (long long a0 = 0; a0 <= p.nx; a0 += TN) {
          const long long nf = std::min<long long>(TN, p.nx + 1 - a0) * std::min<long long>(TT, p.ny - b0);
          wx.push_back({fc * nf, make_int4(i, (int)a0, (int)b0, TT)});
        }
      for (long long b0 = 0; b0 < p.nx; b0 += TT)
        for (long long a0 = 0; a0 <= p.ny; a0 += TN) {
          const long long nf = std::min<long long>(TN, p.ny + 1 - a0) * std::min<long long>(TT, p.nx - b0);
          wy.push_back({fc * nf, make_int4(i, (int)a0, (int)b0, TT)});
        }
    }
  }
  if (b->order_by_cost) {
    // 2D before 1D and higher orders first, then larger cost first within an order: a CTA's
    // consecutive items seldom change order (each change restages that order's tables behind
    // two barriers), and the cheapest items come last, where they even out the tail (measured
    // +0.7 % on the 512-problem set against cost order alone)
    const ase_df_batch* bb = b;
    auto rank = [bb](const int4& w) { return bb->params[w.x].ndim * 16 + bb->params[w.x].order; };
    auto cmp = [rank](const std::pair<long long, int4>& a, const std::pair<long long, int4>& c) {
      const int ra = rank(a.second), rc = rank(c.second);
      return ra != rc ? ra > rc : a.first > c.first;
    };
    std::stable_sort(wx.begin(), wx.end(), cmp);
    std::stable_sort(wy.begin(), wy.end(), cmp);
  }
  for (auto& w : wx) b->items_x.push_back(w.second);
  for (auto& w : wy) b->items_y.push_back(w.second);
}

static std::vector<int4> build_chunks(const ase_df_batch* b) {
  std::vector<int4> ch;
  for (int i = 0; i < b->n; ++i) {
    const long long ncell = b->params[i].nx * b->params[i].ny;
    for (long long f = 0; f < ncell; f += b->chunk_cells)
      ch.push_back(make_int4(i, (int)f, (int)std::min<long long>(ncell, f + b->chunk_cells), 0));
  }
  return ch;
}

static ase_df_status upload_schedule(ase_df_batch* b) {
  build_items(b);
  std::vector<int4> ch = build_chunks(b);
  if (b->d_items_x) cudaFree(b->d_items_x);
  if (b->d_items_y) cudaFree(b->d_items_y);
  if (b->d_chunks) cudaFree(b->d_chunks);
  b->d_items_x = b->d_items_y = b->d_chunks = nullptr;
  size_t nx = std::max<size_t>(1, b->items_x.size()), ny = std::max<size_t>(1, b->items_y.size());
  if (cudaMalloc(&b->d_items_x, nx * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&b->d_items_y, ny * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&b->d_chunks, ch.size() * sizeof(int4)) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, ASE_DF_E_NOMEM, "work lists");
  }
  cudaError_t e = cudaMemcpy(b->d_items_x, b->items_x.data(), b->items_x.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->items_y.empty())
    e = cudaMemcpy(b->d_items_y, b->items_y.data(), b->items_y.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_chunks, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(b, e, "work list upload");
  b->nchunks = (int)ch.size();
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return ASE_DF_OK;
}

static int chunk_grid(const ase_df_batch* b) { return std::max(1, std::min(b->nchunks, b->nsm * 8)); }

static cudaError_t launch_sweeps(ase_df_batch* b, int stage, cudaStream_t s) {
  const int counter_base = 2 * stage;
  const int grid_x = std::max(1, std::min((int)b->items_x.size(), b->nsm * b->ctas_per_sm));
  batch_sweep_kernel<0><<<grid_x, kNT, b->smem_bytes, s>>>(b->d_prob, b->d_items_x, (int)b->items_x.size(),
                                                          b->d_counters + counter_base, b->P, stage, b->d_tabs,
                                                          b->d_state);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || b->items_y.empty()) return e;
  const int grid_y = std::max(1, std::min((int)b->items_y.size(), b->nsm * b->ctas_per_sm));
  batch_sweep_kernel<1><<<grid_y, kNT, b->smem_bytes, s>>>(b->d_prob, b->d_items_y, (int)b->items_y.size(),
                                                          b->d_counters + counter_base + 1, b->P, stage, b->d_tabs,
                                                          b->d_state);
  return cudaGetLastError();
}

static cudaError_t batch_step_launches(ase_df_batch* b, cudaStream_t s) {
  const int nthr = std::max(b->n, 8);
  batch_reset_kernel<<<(nthr + 255) / 256, 256, 0, s>>>(b->d_counters, 8, b->d_state, b->n, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int cg = chunk_grid(b);
  batch_max_speed_kernel<<<cg, 256, 0, s>>>(b->d_prob, b->d_chunks, b->nchunks, b->P, b->d_state);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int stage = 1; stage <= 3; ++stage) {
    if ((e = launch_sweeps(b, stage, s)) != cudaSuccess) return e;
    batch_combine_kernel<<<cg, 256, 0, s>>>(b->d_prob, b->d_chunks, b->nchunks, b->P, stage, b->d_state);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int pass = 1; pass <= kRepairPasses; ++pass) {
      batch_repair_kernel<<<cg, 256, 0, s>>>(b->d_prob, b->d_chunks, b->nchunks, b->P, stage, pass, b->d_state);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    batch_repair_kernel<<<cg, 256, 0, s>>>(b->d_prob, b->d_chunks, b->nchunks, b->P, stage, 0, b->d_state);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static ase_df_status set_user(ase_df_batch* b, const double* W, const double* sx, const double* sy) {
  if (!W || !sx || (b->any2d && !sy)) return bfail(b, ASE_DF_E_INVAL, "NULL state or sigma pointer");
  b->P.W = const_cast<double*>(W);
  b->P.sx = const_cast<double*>(sx);
  b->P.sy = const_cast<double*>(sy ? sy : b->P.zsy);
  return ASE_DF_OK;
}

extern "C" {

ase_df_status ase_df_batch_init(const ase_df_params* p, int32_t n, ase_df_batch** out) {
  if (!out) return bfail(nullptr, ASE_DF_E_INVAL, "out is NULL");
  *out = nullptr;
  if (!p || n < 1) return bfail(nullptr, ASE_DF_E_INVAL, "need at least one problem");
  ase_df_batch* b = new (std::nothrow) ase_df_batch();
  if (!b) return bfail(nullptr, ASE_DF_E_NOMEM, "host allocation");
  b->n = n;
  b->params.assign(p, p + n);
  long long w = 0, x = 0, y = 0, fx = 0, fy = 0, cells = 0;
  for (int i = 0; i < n; ++i) {
    char why[128];
    if (!valid_problem(b->params[i], why, sizeof(why))) {
      delete b;
      return bfail(nullptr, ASE_DF_E_INVAL, "problem %d: %s", i, why);
    }
    const ase_df_params& q = b->params[i];
    const int C = (q.ndim == 1) ? 3 : 4;
    if ((double)C * (double)(q.nx + 1) * (double)(q.ny + 1) >= 2147483648.0) {
      delete b;
      return bfail(nullptr, ASE_DF_E_BOUNDS, "problem %d too large", i);
    }
    b->w_off.push_back(w);
    b->sx_off.push_back(x);
    b->sy_off.push_back(y);
    b->fx_off.push_back(fx);
    b->fy_off.push_back(fy);
    b->cell_off.push_back(cells);
    w += (long long)C * q.nx * q.ny;
    x += q.ny * (q.nx + 1);
    y += (q.ndim == 2) ? (q.ny + 1) * q.nx : 0;
    fx += (long long)C * q.ny * (q.nx + 1);
    fy += (q.ndim == 2) ? (long long)C * (q.ny + 1) * q.nx : 0;
    cells += q.nx * q.ny;
    if (q.ndim == 2) b->any2d = 1;
  }
  b->w_off.push_back(w);
  b->sx_off.push_back(x);
  b->sy_off.push_back(y);
  if (cells >= 2147483648LL) {
    delete b;
    return bfail(nullptr, ASE_DF_E_BOUNDS, "more than 2^31 cells in a batch");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  // device descriptors and tables
  std::vector<BatchProblem> desc(n);
  for (int i = 0; i < n; ++i) {
    fill_grid(b->params[i], desc[i]);
    desc[i].w_off = b->w_off[i];
    desc[i].sx_off = b->sx_off[i];
    desc[i].sy_off = b->sy_off[i];
    desc[i].fx_off = b->fx_off[i];
    desc[i].fy_off = b->fy_off[i];
    desc[i].cell_off = b->cell_off[i];
  }
  std::vector<Tables> tabs(8);
  for (int v = 0; v < 8; ++v) build_tables(3 + 2 * (v % 4), 1 + v / 4, &tabs[v]);
  for (int i = 0; i < n; ++i) set_flux_weights(desc[i].g, tabs[desc[i].variant]);
  const size_t yw = (size_t)std::max<long long>(1, y);
  struct { void** ptr; size_t bytes; } allocs[] = {
    {(void**)&b->d_prob, sizeof(BatchProblem) * n}, {(void**)&b->d_state, sizeof(DevState) * n},
    {(void**)&b->d_tabs, sizeof(Tables) * 8}, {(void**)&b->d_counters, sizeof(unsigned int) * 8},
    {(void**)&b->P.W1, sizeof(double) * w}, {(void**)&b->P.W2, sizeof(double) * w},
    {(void**)&b->P.sxa, sizeof(double) * x}, {(void**)&b->P.sxb, sizeof(double) * x},
    {(void**)&b->P.sya, sizeof(double) * yw}, {(void**)&b->P.syb, sizeof(double) * yw},
    {(void**)&b->P.zsx, sizeof(double) * x}, {(void**)&b->P.zsy, sizeof(double) * yw},
    {(void**)&b->P.Fx, sizeof(double) * fx}, {(void**)&b->P.Fy, sizeof(double) * std::max<long long>(1, fy)},
    {(void**)&b->P.mark, (size_t)cells},
  };
  for (auto& a : allocs) {
    if (cudaMalloc(a.ptr, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      ase_df_batch_destroy(b);
      return bfail(nullptr, ASE_DF_E_NOMEM, "device allocation of %zu bytes failed", a.bytes);
    }
  }
  cudaError_t e = cudaMemcpy(b->d_prob, desc.data(), sizeof(BatchProblem) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tabs, tabs.data(), sizeof(Tables) * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_state, 0, sizeof(DevState) * n);
  if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, sizeof(unsigned int) * 8);
  if (e == cudaSuccess) e = cudaMemset(b->P.zsx, 0, sizeof(double) * x);
  if (e == cudaSuccess) e = cudaMemset(b->P.zsy, 0, sizeof(double) * yw);
  if (e != cudaSuccess) {
    ase_df_batch_destroy(b);
    return bfail(nullptr, ASE_DF_E_CUDA, "batch init: %s", cudaGetErrorString(e));
  }
  b->smem_bytes = std::max(Tile<9, 2>::smem_doubles, Tile<9, 1>::smem_doubles) * sizeof(double);
  e = cudaFuncSetAttribute(batch_sweep_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_sweep_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes);
  if (e != cudaSuccess) {
    ase_df_batch_destroy(b);
    return bfail(nullptr, ASE_DF_E_CUDA, "batch smem attribute: %s", cudaGetErrorString(e));
  }
  ase_df_status st = upload_schedule(b);
  if (st != ASE_DF_OK) {
    ase_df_batch_destroy(b);
    return bfail(nullptr, st, "batch work lists");
  }
  *out = b;
  return ASE_DF_OK;
}

void ase_df_batch_destroy(ase_df_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  void* ptrs[] = {b->d_prob, b->d_state, b->d_tabs, b->d_items_x, b->d_items_y, b->d_chunks, b->d_counters,
                  b->P.W1, b->P.W2, b->P.sxa, b->P.sya, b->P.sxb, b->P.syb, b->P.zsx, b->P.zsy, b->P.Fx,
                  b->P.Fy, b->P.mark};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

const char* ase_df_batch_last_error(const ase_df_batch* b) { return b ? b->err : g_batch_err; }

ase_df_status ase_df_batch_layout(const ase_df_batch* b, int64_t* w_off, int64_t* sx_off, int64_t* sy_off) {
  if (!b) return ASE_DF_E_INVAL;
  for (int i = 0; i <= b->n; ++i) {
    if (w_off) w_off[i] = b->w_off[i];
    if (sx_off) sx_off[i] = b->sx_off[i];
    if (sy_off) sy_off[i] = b->sy_off[i];
  }
  return ASE_DF_OK;
}

ase_df_status ase_df_batch_prime_sigma(ase_df_batch* b, const double* W, double* sx, double* sy, void* stream) {
  if (!b) return ASE_DF_E_INVAL;
  ase_df_status st = set_user(b, W, sx, sy);
  if (st != ASE_DF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  const int nthr = std::max(b->n, 8);
  batch_reset_kernel<<<(nthr + 255) / 256, 256, 0, s>>>(b->d_counters, 8, b->d_state, b->n, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_sweeps(b, 0, s);
  if (e == cudaSuccess) {  // then a clean status (time 0), as ase_df_reset after priming
    batch_reset_kernel<<<(nthr + 255) / 256, 256, 0, s>>>(b->d_counters, 8, b->d_state, b->n, 1);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return bcuda(b, e, "batch prime");
  return ASE_DF_OK;
}

ase_df_status ase_df_batch_step(ase_df_batch* b, double* W, double* sx, double* sy, void* stream) {
  if (!b) return ASE_DF_E_INVAL;
  ase_df_status st = set_user(b, W, sx, sy);
  if (st != ASE_DF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  cudaError_t e = batch_step_launches(b, s);
  if (e != cudaSuccess) return bcuda(b, e, "batch step");
  return ASE_DF_OK;
}

ase_df_status ase_df_batch_run(ase_df_batch* b, double* W, double* sx, double* sy, int32_t nsteps, void* stream) {
  if (!b) return ASE_DF_E_INVAL;
  if (nsteps < 0) return bfail(b, ASE_DF_E_INVAL, "nsteps < 0");
  ase_df_status st = set_user(b, W, sx, sy);
  if (st != ASE_DF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  if (nsteps == 0) return ASE_DF_OK;
  if (!b->graph || b->g_W != W || b->g_sx != sx || b->g_sy != sy) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaError_t e;
    if (!b->cap_stream && (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bcuda(b, e, "capture stream");
    if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return bcuda(b, e, "begin capture");
    cudaError_t le = batch_step_launches(b, b->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return bcuda(b, le != cudaSuccess ? le : e, "batch capture");
    }
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bcuda(b, e, "graph instantiate");
    }
    b->g_W = W;
    b->g_sx = sx;
    b->g_sy = sy;
  }
  for (int32_t i = 0; i < nsteps; ++i) {
    cudaError_t e = cudaGraphLaunch(b->graph, s);
    if (e != cudaSuccess) return bcuda(b, e, "graph launch");
  }
  return ASE_DF_OK;
}

ase_df_status ase_df_batch_get_status(ase_df_batch* b, uint32_t* flags, double* t, double* last_dt) {
  if (!b) return ASE_DF_E_INVAL;
  cudaError_t e = cudaStreamSynchronize(b->last_stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch status sync");
  std::vector<DevState> h(b->n);
  e = cudaMemcpy(h.data(), b->d_state, sizeof(DevState) * b->n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bcuda(b, e, "batch status copy");
  bool bad = false;
  for (int i = 0; i < b->n; ++i) {
    if (flags) flags[i] = h[i].flags;
    if (t) t[i] = h[i].t;
    if (last_dt) last_dt[i] = h[i].last_dt;
    if (h[i].flags & ASE_DF_FLAG_NONPHYSICAL) bad = true;
  }
  return bad ? bfail(b, ASE_DF_E_NONPHYSICAL, "a problem reports a non-physical state") : ASE_DF_OK;
}

ase_df_status ase_df_batch_set_schedule(ase_df_batch* b, int32_t ctas_per_sm, int32_t order_by_cost,
                                        int32_t chunk_cells) {
  if (!b) return ASE_DF_E_INVAL;
  if (ctas_per_sm < 1 || ctas_per_sm > 2 || chunk_cells < 256 || chunk_cells > (1 << 24))
    return bfail(b, ASE_DF_E_INVAL, "schedule out of range (ctas_per_sm 1..2, chunk_cells 256..2^24)");
  const bool relist = (order_by_cost != 0) != (b->order_by_cost != 0) || chunk_cells != b->chunk_cells;
  b->ctas_per_sm = ctas_per_sm;
  b->order_by_cost = order_by_cost != 0;
  b->chunk_cells = chunk_cells;
  if (relist) {
    cudaDeviceSynchronize();
    return upload_schedule(b);
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return ASE_DF_OK;
}

ase_df_status ase_df_batch_set_tiles(ase_df_batch* b, const int32_t* lines) {
  if (!b || !lines) return ASE_DF_E_INVAL;
  for (int k = 0; k < 4; ++k)
    if (lines[k] != 32 && lines[k] != 64) return bfail(b, ASE_DF_E_INVAL, "tile lines must be 32 or 64");
  bool changed = false;
  for (int k = 0; k < 4; ++k) {
    changed |= b->tile_lines[k] != lines[k];
    b->tile_lines[k] = lines[k];
  }
  if (!changed) return ASE_DF_OK;
  cudaDeviceSynchronize();
  return upload_schedule(b);
}

}  // extern "C"
