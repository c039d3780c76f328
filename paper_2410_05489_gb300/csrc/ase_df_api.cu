// C ABI of the ASE-DF library (declared in include/ase_df.h): validation, context and
// scratch management, and the launch sequences of one residual and of one SSP-RK3 step.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ase_df.h"
#include "ase_df_adjoint.cuh"
#include "ase_df_gks.cuh"
#include "ase_df_internal.cuh"

using namespace asedf;

struct ase_df_ctx {
  ase_df_params p;
  int C, K, dim;
  GridInfo g;
  Tables tab;
  DTables dtab;             // derivative weights (gas-kinetic path)
  double dx, dy, inv_dx, inv_dy, inflow_speed;
  // device scratch owned by the context
  double *Fx, *Fy;          // face fluxes
  double *W1, *W2;          // RK stage states
  double *sxa, *sya, *sxb, *syb;  // sigma ping-pong
  double *zsx, *zsy;        // zero sigma (priming)
  unsigned char* mark;      // per-cell marks of the positivity repair
  DevState* st;
  // adjoint scratch (allocated by the first adjoint call)
  double* adj;              // per-direction kernel scratch (adj_scratch_doubles)
  double *Ab1, *Ab2, *Abn;  // stage adjoints of the SSP-RK3 step adjoint
  double *s0bx, *s0by, *s1bx, *s1by, *s2bx, *s2by;  // sigma adjoints of the stages
  // gas-kinetic scratch (allocated by the first gas-kinetic call)
  double *Fxt, *Fyt;        // time derivatives of the face fluxes
  double *L0, *Lt0;         // L(W^n), L_t(W^n) of an S2O4 step
  // CUDA graph of one step (ase_df_run)
  cudaGraphExec_t graph_exec;
  double* g_W;
  double* g_sx;
  double* g_sy;
  double g_dt;
  cudaStream_t cap_stream;
  cudaStream_t last_stream;
  // 2D: the stream and events of the y-sweep, which runs beside the x-sweep (face_fluxes)
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  // kernel timing (ase_df_profile_*)
  bool prof_on;
  bool hist_on;             // branch histogram of the sweeps (ase_df_hist_*)
  bool g_hist;              // hist_on when the step graph was captured
  std::vector<cudaEvent_t>* prof_ev;  // pairs (start, stop)
  std::vector<int>* prof_kind;
  char err[512];
};

static const size_t kProfMax = 65536;

// Records an event pair around one launch when profiling is on (never during capture).
struct ProfScope {
  ase_df_ctx* c;
  cudaStream_t s;
  int kind;
  cudaEvent_t e1;
  bool on;
  ProfScope(ase_df_ctx* c_, cudaStream_t s_, int kind_) : c(c_), s(s_), kind(kind_), e1(nullptr), on(false) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (!c->prof_on || cs != cudaStreamCaptureStatusNone || c->prof_kind->size() >= kProfMax) return;
    cudaEvent_t e0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return;
    cudaEventRecord(e0, s);
    c->prof_ev->push_back(e0);
    on = true;
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(e1, s);
    c->prof_ev->push_back(e1);
    c->prof_kind->push_back(kind);
  }
};

static void prof_clear(ase_df_ctx* c) {
  if (!c->prof_ev) return;
  for (cudaEvent_t e : *c->prof_ev) cudaEventDestroy(e);
  c->prof_ev->clear();
  c->prof_kind->clear();
}

static char g_init_err[512] = "";

static ase_df_status fail(ase_df_ctx* c, ase_df_status s, const char* fmt, ...) {
  char* dst = c ? c->err : g_init_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return s;
}

static ase_df_status cuda_fail(ase_df_ctx* c, cudaError_t e, const char* where) {
  return fail(c, ASE_DF_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static double sound_speed_sum(const ase_df_params& p, double inv_dx, double inv_dy) {
  const double rho = p.inflow_state[0], u = p.inflow_state[1], v = p.inflow_state[2], pr = p.inflow_state[3];
  const double c = std::sqrt(p.gamma * pr / rho);
  double s = (std::fabs(u) + c) * inv_dx;
  if (p.ndim == 2) s += (std::fabs(v) + c) * inv_dy;
  return s;
}

// primitive (rho, u, v, p) -> conservative (rho, rho u, [rho v], E)
static void to_conservative(const double* q, double gamma, int C, double* out) {
  const double rho = q[0], u = q[1], v = q[2], pr = q[3];
  out[0] = rho;
  out[1] = rho * u;
  if (C == 4) {
    out[2] = rho * v;
    out[3] = pr / (gamma - 1.0) + 0.5 * rho * (u * u + v * v);
  } else {
    out[2] = pr / (gamma - 1.0) + 0.5 * rho * u * u;
  }
}

namespace asedf {

char* init_error_buffer() { return g_init_err; }

ase_df_status setup_problem(const ase_df_params* pin, ProblemSetup* out, char* err, size_t err_len) {
  auto bad = [&](ase_df_status st, const char* fmt, auto... args) {
    if (err && err_len) snprintf(err, err_len, fmt, args...);
    return st;
  };
  if (!pin) return bad(ASE_DF_E_INVAL, "params is NULL");
  ase_df_params p = *pin;
  if (p.ndim != 1 && p.ndim != 2) return bad(ASE_DF_E_INVAL, "ndim must be 1 or 2 (got %d)", p.ndim);
  if (p.order != 3 && p.order != 5 && p.order != 7 && p.order != 9)
    return bad(ASE_DF_E_INVAL, "order must be 3, 5, 7 or 9 (got %d)", p.order);
  if (p.ndim == 1) p.ny = 1;
  if (p.nx < 1 || p.ny < 1) return bad(ASE_DF_E_INVAL, "nx, ny must be >= 1");
  if (p.nx > (1 << 20) || p.ny > (1 << 20)) return bad(ASE_DF_E_BOUNDS, "nx, ny must be <= 2^20");
  const int C = (p.ndim == 1) ? 3 : 4;
  if ((double)C * (double)(p.nx + 1) * (double)(p.ny + 1) >= 2147483648.0)
    return bad(ASE_DF_E_BOUNDS, "C*(nx+1)*(ny+1) must be < 2^31");
  if (!(p.x1 > p.x0) || (p.ndim == 2 && !(p.y1 > p.y0))) return bad(ASE_DF_E_INVAL, "empty domain");
  if (!(p.gamma > 1.0) || !std::isfinite(p.gamma)) return bad(ASE_DF_E_INVAL, "gamma must be > 1");
  if (!(p.sigma_thres > 0.0)) return bad(ASE_DF_E_INVAL, "sigma_thres must be > 0");
  if (!(p.cfl > 0.0)) return bad(ASE_DF_E_INVAL, "cfl must be > 0");
  for (int s = 0; s < 4; ++s) {
    if (p.bc[s] < 0 || p.bc[s] > 5) return bad(ASE_DF_E_INVAL, "bad boundary code %d", p.bc[s]);
    if (p.bc[s] == ASE_DF_BC_INFLOW_BAND && s != 0)
      return bad(ASE_DF_E_INVAL, "the inflow band is supported on x-lo only");
    if (p.bc[s] == ASE_DF_BC_WALL_AFTER && (s != 2 || p.ndim != 2))
      return bad(ASE_DF_E_INVAL, "the split wall is supported on y-lo of a 2D grid only");
    if (p.bc[s] == ASE_DF_BC_MOVING_SHOCK && (s != 3 || p.ndim != 2))
      return bad(ASE_DF_E_INVAL, "the moving-shock boundary is supported on y-hi of a 2D grid only");
    if (p.ndim == 1 && s >= 2) p.bc[s] = ASE_DF_BC_OUTFLOW;
  }
  {
    const int64_t need = (p.order + 1) / 2;
    if ((p.bc[0] == ASE_DF_BC_REFLECT || p.bc[1] == ASE_DF_BC_REFLECT) && p.nx < need)
      return bad(ASE_DF_E_INVAL, "a reflecting x-wall needs nx >= %lld", (long long)need);
    if (p.ndim == 2 && (p.bc[2] == ASE_DF_BC_REFLECT || p.bc[3] == ASE_DF_BC_REFLECT ||
                        p.bc[2] == ASE_DF_BC_WALL_AFTER) && p.ny < need)
      return bad(ASE_DF_E_INVAL, "a reflecting y-wall needs ny >= %lld", (long long)need);
  }
  if ((p.bc[0] == ASE_DF_BC_PERIODIC) != (p.bc[1] == ASE_DF_BC_PERIODIC))
    return bad(ASE_DF_E_INVAL, "periodic boundaries must come in pairs (x)");
  if (p.ndim == 2 && (p.bc[2] == ASE_DF_BC_PERIODIC) != (p.bc[3] == ASE_DF_BC_PERIODIC))
    return bad(ASE_DF_E_INVAL, "periodic boundaries must come in pairs (y)");
  const bool uses_inflow = p.bc[0] == ASE_DF_BC_INFLOW_BAND || p.bc[2] == ASE_DF_BC_WALL_AFTER ||
                           p.bc[3] == ASE_DF_BC_MOVING_SHOCK;
  if (uses_inflow && !(p.inflow_state[0] > 0.0 && p.inflow_state[3] > 0.0))
    return bad(ASE_DF_E_INVAL, "inflow state must have rho > 0 and p > 0");
  if (p.bc[3] == ASE_DF_BC_MOVING_SHOCK) {
    if (!(p.state_b[0] > 0.0 && p.state_b[3] > 0.0))
      return bad(ASE_DF_E_INVAL, "state_b must have rho > 0 and p > 0");
    if (!std::isfinite(p.shock_x0) || !std::isfinite(p.shock_speed))
      return bad(ASE_DF_E_INVAL, "shock_x0 and shock_speed must be finite");
  }
  if (p.bc[2] == ASE_DF_BC_WALL_AFTER && !std::isfinite(p.wall_x))
    return bad(ASE_DF_E_INVAL, "wall_x must be finite");

  ProblemSetup& o = *out;
  o = ProblemSetup{};
  o.p = p;
  o.C = C;
  o.K = (p.order - 1) / 2;
  o.dx = (p.x1 - p.x0) / (double)p.nx;
  o.dy = (p.ndim == 2) ? (p.y1 - p.y0) / (double)p.ny : 1.0;
  o.inv_dx = 1.0 / o.dx;
  o.inv_dy = (p.ndim == 2) ? 1.0 / o.dy : 0.0;
  o.inflow_speed = 0.0;
  GridInfo& g = o.g;
  g.nx = (int)p.nx;
  g.ny = (int)p.ny;
  for (int s = 0; s < 4; ++s) g.bc[s] = p.bc[s];
  g.band_j0 = 1;
  g.band_j1 = 0;  // empty
  if (p.bc[0] == ASE_DF_BC_INFLOW_BAND) {
    // rows whose centre y0 + (j + 1/2) dy lies strictly inside (inflow_lo, inflow_hi)
    int j0 = -1, j1 = -2;
    for (int j = 0; j < g.ny; ++j) {
      const double yc = p.y0 + ((double)j + 0.5) * o.dy;
      if (yc > p.inflow_lo && yc < p.inflow_hi) {
        if (j0 < 0) j0 = j;
        j1 = j;
      }
    }
    if (j0 >= 0) { g.band_j0 = j0; g.band_j1 = j1; }
    o.inflow_speed = sound_speed_sum(p, o.inv_dx, o.inv_dy);
  }
  if (uses_inflow) to_conservative(p.inflow_state, p.gamma, C, g.inflow_cons);
  if (p.bc[3] == ASE_DF_BC_MOVING_SHOCK) to_conservative(p.state_b, p.gamma, C, g.state_b_cons);
  g.x0 = p.x0;
  g.dx = o.dx;
  g.shock_x0 = p.shock_x0;
  g.shock_speed = p.shock_speed;
  if (p.bc[2] == ASE_DF_BC_WALL_AFTER) {
    // the first column whose centre x0 + (i + 1/2) dx is at or past wall_x; ghost columns
    // reach k + 1 cells beyond the grid, so the search is confined to that range
    const int lo = -(o.K + 2), hi = g.nx + o.K + 2;
    auto centre = [&](int i) { return p.x0 + ((double)i + 0.5) * o.dx; };
    const double est = std::floor((p.wall_x - p.x0) / o.dx - 0.5) - 2.0;
    int i0 = (int)std::max((double)lo, std::min((double)hi, est));
    while (i0 > lo && centre(i0) >= p.wall_x) --i0;
    while (i0 < hi && centre(i0) < p.wall_x) ++i0;
    g.wall_i0 = i0;
  }
  g.gamma = p.gamma;
  g.gm1 = p.gamma - 1.0;
  g.gg1 = p.gamma * (p.gamma - 1.0);
  g.thres = p.sigma_thres;
  return ASE_DF_OK;
}

}  // namespace asedf

extern "C" {

ase_df_status ase_df_init(const ase_df_params* pin, ase_df_ctx** out) {
  if (!out) return fail(nullptr, ASE_DF_E_INVAL, "out is NULL");
  *out = nullptr;
  ProblemSetup ps;
  {
    const ase_df_status v = setup_problem(pin, &ps, g_init_err, sizeof(g_init_err));
    if (v != ASE_DF_OK) return v;
  }
  const ase_df_params& p = ps.p;
  const int C = ps.C;

  ase_df_ctx* c = new (std::nothrow) ase_df_ctx;
  if (!c) return fail(nullptr, ASE_DF_E_NOMEM, "host allocation failed");
  std::memset(c, 0, sizeof(*c));
  c->prof_ev = new (std::nothrow) std::vector<cudaEvent_t>();
  c->prof_kind = new (std::nothrow) std::vector<int>();
  if (!c->prof_ev || !c->prof_kind) {
    delete c->prof_ev;
    delete c->prof_kind;
    delete c;
    return fail(nullptr, ASE_DF_E_NOMEM, "host allocation failed");
  }
  c->p = p;
  c->C = C;
  c->K = ps.K;
  c->dim = p.ndim;
  c->dx = ps.dx;
  c->dy = ps.dy;
  c->inv_dx = ps.inv_dx;
  c->inv_dy = ps.inv_dy;
  c->inflow_speed = ps.inflow_speed;
  c->g = ps.g;
  const GridInfo& g = c->g;
  build_tables(p.order, p.ndim, &c->tab);
  build_dtables(p.order, p.ndim, &c->dtab);
  set_flux_weights(c->g, c->tab);

  const size_t nW = (size_t)C * g.nx * g.ny;
  const size_t nFx = (size_t)C * g.ny * (g.nx + 1);
  const size_t nFy = (p.ndim == 2) ? (size_t)C * (g.ny + 1) * g.nx : 1;
  const size_t nsx = (size_t)g.ny * (g.nx + 1);
  const size_t nsy = (p.ndim == 2) ? (size_t)(g.ny + 1) * g.nx : 1;
  struct { double** ptr; size_t n; } allocs[] = {
    {&c->Fx, nFx}, {&c->Fy, nFy}, {&c->W1, nW}, {&c->W2, nW}, {&c->sxa, nsx}, {&c->sya, nsy},
    {&c->sxb, nsx}, {&c->syb, nsy}, {&c->zsx, nsx}, {&c->zsy, nsy},
  };
  for (auto& a : allocs) {
    if (cudaMalloc((void**)a.ptr, a.n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      ase_df_destroy(c);
      return fail(nullptr, ASE_DF_E_NOMEM, "device allocation of %zu bytes failed", a.n * sizeof(double));
    }
  }
  if (cudaMalloc((void**)&c->mark, (size_t)g.nx * g.ny) != cudaSuccess) {
    cudaGetLastError();
    ase_df_destroy(c);
    return fail(nullptr, ASE_DF_E_NOMEM, "device allocation of the repair marks failed");
  }
  if (cudaMalloc((void**)&c->st, sizeof(DevState)) != cudaSuccess) {
    cudaGetLastError();
    ase_df_destroy(c);
    return fail(nullptr, ASE_DF_E_NOMEM, "device allocation of the status word failed");
  }
  cudaError_t e = cudaMemset(c->zsx, 0, nsx * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->zsy, 0, nsy * sizeof(double));
  if (e == cudaSuccess && p.ndim == 2) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && p.ndim == 2) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && p.ndim == 2) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemset(c->st, 0, sizeof(DevState));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    ase_df_destroy(c);
    return fail(nullptr, ASE_DF_E_CUDA, "init: %s", cudaGetErrorString(e));
  }
  *out = c;
  return ASE_DF_OK;
}

void ase_df_destroy(ase_df_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  double* ptrs[] = {c->Fx,  c->Fy,  c->W1,   c->W2,   c->sxa,  c->sya,  c->sxb,  c->syb,  c->zsx, c->zsy,
                    c->adj, c->Ab1, c->Ab2,  c->Abn,  c->s0bx, c->s0by, c->s1bx, c->s1by, c->s2bx, c->s2by,
                    c->Fxt, c->Fyt, c->L0,   c->Lt0};
  for (double* q : ptrs)
    if (q) cudaFree(q);
  if (c->st) cudaFree(c->st);
  if (c->mark) cudaFree(c->mark);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  prof_clear(c);
  delete c->prof_ev;
  delete c->prof_kind;
  delete c;
}

const char* ase_df_last_error(const ase_df_ctx* c) { return c ? c->err : g_init_err; }

}  // extern "C"

// ---------------------------------------------------------------------------------
// launch sequences
// ---------------------------------------------------------------------------------
static cudaError_t sweep(ase_df_ctx* c, int dir, const double* W, const double* sx, const double* sy,
                         double* F, double* s_out, cudaStream_t s, double tfrac) {
  SweepArgs a;
  a.tfrac = tfrac;
  a.W = W;
  a.s_norm = (dir == 0) ? sx : sy;
  a.s_tan = (dir == 0) ? sy : sx;
  a.F = F;
  a.s_out = s_out;
  a.st = c->st;
  a.hist = c->hist_on ? c->st->hist : nullptr;
  ProfScope prof(c, s, dir);
  switch (c->p.order) {
    case 3: return launch_sweep_r3(c->dim, dir, c->g, a, c->tab, s);
    case 5: return launch_sweep_r5(c->dim, dir, c->g, a, c->tab, s);
    case 7: return launch_sweep_r7(c->dim, dir, c->g, a, c->tab, s);
    default: return launch_sweep_r9(c->dim, dir, c->g, a, c->tab, s);
  }
}

// Face fluxes of both directions of W with sigma_in = (sx, sy), sigma_out -> (sxo, syo);
// time-dependent ghosts at the device time t + tfrac dt.  The two sweeps read the same
// inputs and write separate outputs, so in 2D the y-sweep runs on the context's side stream
// (forked from and joined back to s, also under graph capture): its tiles take the SMs that
// the x-sweep's last tiles leave.  With kernel timing on, the sweeps run one after the other
// so that each launch is timed alone.
static cudaError_t face_fluxes(ase_df_ctx* c, const double* W, const double* sx, const double* sy,
                               double* sxo, double* syo, cudaStream_t s, double tfrac = 0.0) {
  if (c->dim == 1 || c->prof_on) {
    cudaError_t e = sweep(c, 0, W, sx, sy, c->Fx, sxo, s, tfrac);
    if (e != cudaSuccess || c->dim == 1) return e;
    return sweep(c, 1, W, sx, sy, c->Fy, syo, s, tfrac);
  }
  cudaError_t e = cudaEventRecord(c->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  if (e != cudaSuccess) return e;
  cudaError_t ex = sweep(c, 0, W, sx, sy, c->Fx, sxo, s, tfrac);
  cudaError_t ey = sweep(c, 1, W, sx, sy, c->Fy, syo, c->side, tfrac);
  // the join is made whatever happened, so that s never runs ahead of the side stream
  e = cudaEventRecord(c->ev_join, c->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
  return ex != cudaSuccess ? ex : (ey != cudaSuccess ? ey : e);
}

// Time offsets of the SSP-RK3 stage values (Sec. 2.3): W^n at t, W^(1) at t + dt, W^(2) at
// t + dt/2; stage s's fluxes and repair see the boundaries at the time of its input.
static double rk_tfrac(int stage) { return stage == 2 ? 1.0 : (stage == 3 ? 0.5 : 0.0); }

// Stage combination (or L for stage 0); for stages 1..3 followed by the positivity
// repair passes, which get the stage's sigma_out (sxo, syo).
static cudaError_t combine(ase_df_ctx* c, int stage, const double* Wn, const double* Ws, double* out,
                           double dt_fixed, cudaStream_t s, double* sxo = nullptr, double* syo = nullptr) {
  cudaError_t e = cudaSuccess;
  CombineArgs a;
  a.mark = c->mark;
  a.Fx = c->Fx;
  a.Fy = c->Fy;
  a.Wn = Wn;
  a.Ws = Ws;
  a.out = out;
  a.st = c->st;
  a.inv_dx = c->inv_dx;
  a.inv_dy = c->inv_dy;
  a.dt_fixed = dt_fixed;
  a.cfl = c->p.cfl;
  a.t_end = c->p.t_end;
  a.inflow_speed = c->inflow_speed;
  a.stage = stage;
  {
    ProfScope prof(c, s, 2);
    e = launch_combine(c->dim, c->g, a, s);
  }
  if (e != cudaSuccess || stage == 0) return e;
  RepairArgs r;
  r.mark = c->mark;
  r.Fx = c->Fx;
  r.Fy = c->Fy;
  r.Wn = Wn;
  r.Ws = Ws;
  r.out = out;
  r.sx_out = sxo;
  r.sy_out = syo;
  r.st = c->st;
  r.inv_dx = c->inv_dx;
  r.inv_dy = c->inv_dy;
  r.dt_fixed = dt_fixed;
  r.stage = stage;
  r.tfrac = rk_tfrac(stage);
  r.pass = 1;
  ProfScope prof(c, s, 4);
  return launch_repair_all(c->dim, c->g, r, s);
}

static ase_df_status check_ptrs(ase_df_ctx* c, const void* W, const void* sx, const void* sy) {
  if (!c) return ASE_DF_E_INVAL;
  if (!W || !sx) return fail(c, ASE_DF_E_INVAL, "NULL state or sigma pointer");
  if (c->dim == 2 && !sy) return fail(c, ASE_DF_E_INVAL, "sy must not be NULL in 2D");
  return ASE_DF_OK;
}

static ase_df_status step_launches(ase_df_ctx* c, double* W, double* sx, double* sy, double dt,
                                   cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!(dt > 0.0)) {
    SpeedArgs sa;
    sa.W = W;
    sa.st = c->st;
    sa.inv_dx = c->inv_dx;
    sa.inv_dy = c->inv_dy;
    {
      ProfScope prof(c, s, 3);
      e = launch_max_speed(c->dim, c->g, sa, s);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "max_speed");
  }
  const double dtf = (dt > 0.0) ? dt : 0.0;
  // stage 1
  if ((e = face_fluxes(c, W, sx, sy, c->sxa, c->sya, s)) != cudaSuccess) return cuda_fail(c, e, "stage 1 sweep");
  if ((e = combine(c, 1, W, W, c->W1, dtf, s, c->sxa, c->sya)) != cudaSuccess) return cuda_fail(c, e, "stage 1 combine");
  // stage 2
  if ((e = face_fluxes(c, c->W1, c->sxa, c->sya, c->sxb, c->syb, s, rk_tfrac(2))) != cudaSuccess) return cuda_fail(c, e, "stage 2 sweep");
  if ((e = combine(c, 2, W, c->W1, c->W2, dtf, s, c->sxb, c->syb)) != cudaSuccess) return cuda_fail(c, e, "stage 2 combine");
  // stage 3: sigma_out lands in the caller's sx / sy, W^{n+1} in W
  if ((e = face_fluxes(c, c->W2, c->sxb, c->syb, sx, sy, s, rk_tfrac(3))) != cudaSuccess) return cuda_fail(c, e, "stage 3 sweep");
  if ((e = combine(c, 3, W, c->W2, W, dtf, s, sx, sy)) != cudaSuccess) return cuda_fail(c, e, "stage 3 combine");
  return ASE_DF_OK;
}

extern "C" {

ase_df_status ase_df_residual(ase_df_ctx* c, const double* W, const double* sx_in, const double* sy_in,
                              double* L, double* sx_out, double* sy_out, void* stream) {
  ase_df_status r = check_ptrs(c, W, sx_in, sy_in);
  if (r != ASE_DF_OK) return r;
  if (!L || !sx_out || (c->dim == 2 && !sy_out)) return fail(c, ASE_DF_E_INVAL, "NULL output pointer");
  if (sx_out == sx_in || (c->dim == 2 && sy_out == sy_in))
    return fail(c, ASE_DF_E_INVAL, "sigma_out must not alias sigma_in");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  cudaError_t e = face_fluxes(c, W, sx_in, sy_in, sx_out, sy_out, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "residual sweep");
  e = combine(c, 0, W, W, L, 0.0, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "residual combine");
  return ASE_DF_OK;
}

ase_df_status ase_df_prime_sigma(ase_df_ctx* c, const double* W, double* sx, double* sy, void* stream) {
  ase_df_status r = check_ptrs(c, W, sx, sy);
  if (r != ASE_DF_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  cudaError_t e = face_fluxes(c, W, c->zsx, c->zsy, sx, sy, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "prime_sigma");
  return ASE_DF_OK;
}

ase_df_status ase_df_copy_face_fluxes(ase_df_ctx* c, double* Fx, double* Fy, void* stream) {
  if (!c || !Fx || (c->dim == 2 && !Fy)) return c ? fail(c, ASE_DF_E_INVAL, "NULL pointer") : ASE_DF_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nFx = (size_t)c->C * c->g.ny * (c->g.nx + 1);
  cudaError_t e = cudaMemcpyAsync(Fx, c->Fx, nFx * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && c->dim == 2) {
    const size_t nFy = (size_t)c->C * (c->g.ny + 1) * c->g.nx;
    e = cudaMemcpyAsync(Fy, c->Fy, nFy * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "copy_face_fluxes");
  return ASE_DF_OK;
}

ase_df_status ase_df_step(ase_df_ctx* c, double* W, double* sx, double* sy, double dt, void* stream) {
  ase_df_status r = check_ptrs(c, W, sx, sy);
  if (r != ASE_DF_OK) return r;
  if (!std::isfinite(dt)) return fail(c, ASE_DF_E_INVAL, "dt is not finite");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return step_launches(c, W, sx, sy, dt, s);
}

ase_df_status ase_df_run(ase_df_ctx* c, double* W, double* sx, double* sy, double dt, int32_t nsteps,
                         void* stream) {
  ase_df_status r = check_ptrs(c, W, sx, sy);
  if (r != ASE_DF_OK) return r;
  if (nsteps < 0) return fail(c, ASE_DF_E_INVAL, "nsteps < 0");
  if (!std::isfinite(dt)) return fail(c, ASE_DF_E_INVAL, "dt is not finite");
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  if (nsteps == 0) return ASE_DF_OK;
  const double dtkey = (dt > 0.0) ? dt : 0.0;
  if (!c->graph_exec || c->g_W != W || c->g_sx != sx || c->g_sy != sy || c->g_dt != dtkey ||
      c->g_hist != c->hist_on) {
    if (c->graph_exec) {
      cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
    }
    if (!c->cap_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(c, e, "capture stream");
    }
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
    ase_df_status st = step_launches(c, W, sx, sy, dtkey, c->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (st != ASE_DF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->graph_exec = nullptr;
      return cuda_fail(c, e, "graph instantiate");
    }
    c->g_W = W;
    c->g_sx = sx;
    c->g_sy = sy;
    c->g_dt = dtkey;
    c->g_hist = c->hist_on;
  }
  for (int32_t i = 0; i < nsteps; ++i) {
    cudaError_t e = cudaGraphLaunch(c->graph_exec, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
  }
  return ASE_DF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------------
static ase_df_status ensure_adjoint(ase_df_ctx* c) {
  if (c->adj) return ASE_DF_OK;
  const GridInfo& g = c->g;
  size_t nadj = adj_scratch_doubles(c->dim, c->p.order, g.nx, g.ny);
  if (c->dim == 2) nadj += adj_scratch_doubles(c->dim, c->p.order, g.ny, g.nx);
  const size_t nW = (size_t)c->C * g.nx * g.ny;
  const size_t nsx = (size_t)g.ny * (g.nx + 1);
  const size_t nsy = (c->dim == 2) ? (size_t)(g.ny + 1) * g.nx : 1;
  struct { double** ptr; size_t n; } allocs[] = {
    {&c->adj, nadj}, {&c->Ab1, nW}, {&c->Ab2, nW}, {&c->Abn, nW}, {&c->s0bx, nsx}, {&c->s0by, nsy},
    {&c->s1bx, nsx}, {&c->s1by, nsy}, {&c->s2bx, nsx}, {&c->s2by, nsy},
  };
  for (auto& a : allocs) {
    if (cudaMalloc((void**)a.ptr, a.n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      for (auto& b : allocs) {
        if (*b.ptr) cudaFree(*b.ptr);
        *b.ptr = nullptr;
      }
      return fail(c, ASE_DF_E_NOMEM, "device allocation of %zu bytes of adjoint scratch failed", a.n * sizeof(double));
    }
  }
  return ASE_DF_OK;
}

// Wbar += J_W^T (lscale Lbar) + ..., sbi += J_sigma^T ... for both directions.  In 2D the
// face and normal kernels of the y-direction run on the side stream beside those of the
// x-direction (each direction has its own scratch); the gathers of both directions into
// the shared outputs then run as one launch on s, which adds the x-direction's sums first,
// as the serial order does (with kernel timing on, everything is serial on s).
static cudaError_t residual_adjoint(ase_df_ctx* c, const double* W, const double* sx, const double* sy,
                                    const double* Lbar, double lscale, const double* sbo_x, const double* sbo_y,
                                    double* Wbar, double* sbi_x, double* sbi_y, cudaStream_t s) {
  const GridInfo& g = c->g;
  const int K = c->K, KT = (c->dim == 2) ? K : 0, C = c->C;
  AdjArgs aa[2];
  SweepArgs sa[2];
  double* scratch = c->adj;
  for (int dir = 0; dir < c->dim; ++dir) {
    const size_t n = (dir == 0) ? g.nx : g.ny, m = (dir == 0) ? g.ny : g.nx;
    const size_t nf = (n + 1) * m, ni = (n + 2) * (m + 2 * KT);
    AdjArgs& A = aa[dir];
    A.Lbar = Lbar;
    A.lscale = lscale;
    A.sbar_out = (dir == 0) ? sbo_x : sbo_y;
    A.Tbar = scratch;
    A.Cbar = A.Tbar + (size_t)2 * (2 * KT + 1) * C * nf;
    A.Stb = A.Cbar + (size_t)2 * C * nf;
    A.Nbar = A.Stb + (c->dim == 2 ? 8 * nf : 0);
    A.Snb = A.Nbar + (size_t)(2 * K + 1) * C * ni;
    scratch += adj_scratch_doubles(c->dim, c->p.order, (long long)n, (long long)m);
    A.Wbar = Wbar;
    A.sbar_norm = (dir == 0) ? sbi_x : sbi_y;
    A.sbar_tan = (c->dim == 2) ? ((dir == 0) ? sbi_y : sbi_x) : nullptr;
    A.inv_h = (dir == 0) ? c->inv_dx : c->inv_dy;
    SweepArgs& a = sa[dir];
    a.W = W;
    a.s_norm = (dir == 0) ? sx : sy;
    a.s_tan = (dir == 0) ? sy : sx;
    a.F = nullptr;
    a.s_out = nullptr;
    a.st = c->st;
  }
  auto launch = [&](int dir, int phase, cudaStream_t st) -> cudaError_t {
    switch (c->p.order) {
      case 3: return launch_adjoint_r3(c->dim, dir, phase, g, sa[dir], aa[dir], c->tab, st);
      case 5: return launch_adjoint_r5(c->dim, dir, phase, g, sa[dir], aa[dir], c->tab, st);
      case 7: return launch_adjoint_r7(c->dim, dir, phase, g, sa[dir], aa[dir], c->tab, st);
      default: return launch_adjoint_r9(c->dim, dir, phase, g, sa[dir], aa[dir], c->tab, st);
    }
  };
  if (c->dim == 1 || c->prof_on) {
    for (int dir = 0; dir < c->dim; ++dir) {
      cudaError_t e = launch(dir, 3, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = cudaEventRecord(c->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  if (e != cudaSuccess) return e;
  const cudaError_t ex = launch(0, 1, s);
  const cudaError_t ey = launch(1, 1, c->side);
  // the join is made whatever happened, so that s never runs ahead of the side stream
  e = cudaEventRecord(c->ev_join, c->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
  if (ex != cudaSuccess) return ex;
  if (ey != cudaSuccess) return ey;
  if (e != cudaSuccess) return e;
  switch (c->p.order) {
    case 3: return launch_adjoint_gathers_2d_r3(g, aa[0], aa[1], s);
    case 5: return launch_adjoint_gathers_2d_r5(g, aa[0], aa[1], s);
    case 7: return launch_adjoint_gathers_2d_r7(g, aa[0], aa[1], s);
    default: return launch_adjoint_gathers_2d_r9(g, aa[0], aa[1], s);
  }
}

extern "C" {

ase_df_status ase_df_residual_adjoint(ase_df_ctx* c, const double* W, const double* sx_in, const double* sy_in,
                                      const double* Lbar, const double* sxbar_out, const double* sybar_out,
                                      double* Wbar, double* sxbar_in, double* sybar_in, void* stream) {
  ase_df_status r = check_ptrs(c, W, sx_in, sy_in);
  if (r != ASE_DF_OK) return r;
  if (!Wbar) return fail(c, ASE_DF_E_INVAL, "Wbar is NULL");
  for (int b = 0; b < 4; ++b)
    if (c->g.bc[b] >= BC_REFLECT) return fail(c, ASE_DF_E_INVAL, "the adjoint does not support walls or the moving-shock boundary");
  if (Wbar == W || Wbar == Lbar || (sxbar_in && (sxbar_in == sx_in || sxbar_in == sxbar_out)) ||
      (c->dim == 2 && sybar_in && (sybar_in == sy_in || sybar_in == sybar_out)))
    return fail(c, ASE_DF_E_INVAL, "adjoint outputs must not alias the inputs");
  if ((r = ensure_adjoint(c)) != ASE_DF_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  cudaError_t e = residual_adjoint(c, W, sx_in, sy_in, Lbar, 1.0, sxbar_out, c->dim == 2 ? sybar_out : nullptr,
                                   Wbar, sxbar_in, c->dim == 2 ? sybar_in : nullptr, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "residual adjoint");
  return ASE_DF_OK;
}

ase_df_status ase_df_step_adjoint(ase_df_ctx* c, const double* W, const double* sx, const double* sy, double dt,
                                  double* Wbar, double* sxbar, double* sybar, void* stream) {
  ase_df_status r = check_ptrs(c, W, sx, sy);
  if (r != ASE_DF_OK) return r;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, ASE_DF_E_INVAL, "the step adjoint needs a fixed dt > 0");
  for (int b = 0; b < 4; ++b)
    if (c->g.bc[b] >= BC_REFLECT) return fail(c, ASE_DF_E_INVAL, "the adjoint does not support walls or the moving-shock boundary");
  if (!Wbar || !sxbar || (c->dim == 2 && !sybar)) return fail(c, ASE_DF_E_INVAL, "NULL adjoint pointer");
  if (Wbar == W || sxbar == sx || (c->dim == 2 && sybar == sy))
    return fail(c, ASE_DF_E_INVAL, "adjoint arrays must not alias the state");
  if ((r = ensure_adjoint(c)) != ASE_DF_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const GridInfo& g = c->g;
  const size_t nW = (size_t)c->C * g.nx * g.ny;
  const size_t nsx = (size_t)g.ny * (g.nx + 1);
  const size_t nsy = (c->dim == 2) ? (size_t)(g.ny + 1) * g.nx : 0;
  double* sybar_ = (c->dim == 2) ? sybar : nullptr;
  double* s0by = (c->dim == 2) ? c->s0by : nullptr;
  double* s1by = (c->dim == 2) ? c->s1by : nullptr;
  double* s2by = (c->dim == 2) ? c->s2by : nullptr;
  cudaError_t e;
  // stages 1 and 2 of the forward step: W1, sigma1 (sxa, sya), W2, sigma2 (sxb, syb)
  if ((e = face_fluxes(c, W, sx, sy, c->sxa, c->sya, s)) != cudaSuccess) return cuda_fail(c, e, "adjoint: stage 1 sweep");
  if ((e = combine(c, 1, W, W, c->W1, dt, s, c->sxa, c->sya)) != cudaSuccess) return cuda_fail(c, e, "adjoint: stage 1 combine");
  if ((e = face_fluxes(c, c->W1, c->sxa, c->sya, c->sxb, c->syb, s, rk_tfrac(2))) != cudaSuccess) return cuda_fail(c, e, "adjoint: stage 2 sweep");
  if ((e = combine(c, 2, W, c->W1, c->W2, dt, s, c->sxb, c->syb)) != cudaSuccess) return cuda_fail(c, e, "adjoint: stage 2 combine");
  // stage 3: W^{n+1} = W^n / 3 + 2/3 W2 + 2/3 dt L(W2, sigma2), sigma3 = sigma_out(W2, sigma2)
  e = launch_axpby(c->Abn, 1.0 / 3.0, Wbar, 0.0, nullptr, nW, s);
  if (e == cudaSuccess) e = launch_axpby(c->Ab2, 2.0 / 3.0, Wbar, 0.0, nullptr, nW, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->s2bx, 0, nsx * sizeof(double), s);
  if (e == cudaSuccess && nsy) e = cudaMemsetAsync(c->s2by, 0, nsy * sizeof(double), s);
  if (e == cudaSuccess)
    e = residual_adjoint(c, c->W2, c->sxb, c->syb, Wbar, 2.0 / 3.0 * dt, sxbar, sybar_, c->Ab2, c->s2bx, s2by, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint: stage 3");
  // stage 2: W2 = 3/4 W^n + 1/4 W1 + 1/4 dt L(W1, sigma1), sigma2 = sigma_out(W1, sigma1)
  e = launch_axpby(c->Abn, 1.0, c->Abn, 0.75, c->Ab2, nW, s);
  if (e == cudaSuccess) e = launch_axpby(c->Ab1, 0.25, c->Ab2, 0.0, nullptr, nW, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->s1bx, 0, nsx * sizeof(double), s);
  if (e == cudaSuccess && nsy) e = cudaMemsetAsync(c->s1by, 0, nsy * sizeof(double), s);
  if (e == cudaSuccess)
    e = residual_adjoint(c, c->W1, c->sxa, c->sya, c->Ab2, 0.25 * dt, c->s2bx, s2by, c->Ab1, c->s1bx, s1by, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint: stage 2");
  // stage 1: W1 = W^n + dt L(W^n, sigma^n), sigma1 = sigma_out(W^n, sigma^n)
  e = launch_axpby(c->Abn, 1.0, c->Abn, 1.0, c->Ab1, nW, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->s0bx, 0, nsx * sizeof(double), s);
  if (e == cudaSuccess && nsy) e = cudaMemsetAsync(c->s0by, 0, nsy * sizeof(double), s);
  if (e == cudaSuccess) e = residual_adjoint(c, W, sx, sy, c->Ab1, dt, c->s1bx, s1by, c->Abn, c->s0bx, s0by, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint: stage 1");
  e = cudaMemcpyAsync(Wbar, c->Abn, nW * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sxbar, c->s0bx, nsx * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && nsy) e = cudaMemcpyAsync(sybar, c->s0by, nsy * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint: copy out");
  return ASE_DF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// gas-kinetic path (Sec. 2.2)
// ---------------------------------------------------------------------------------
static ase_df_status ensure_gks(ase_df_ctx* c) {
  if (c->Fxt) return ASE_DF_OK;
  const GridInfo& g = c->g;
  const size_t nW = (size_t)c->C * g.nx * g.ny;
  const size_t nFx = (size_t)c->C * g.ny * (g.nx + 1);
  const size_t nFy = (c->dim == 2) ? (size_t)c->C * (g.ny + 1) * g.nx : 1;
  struct { double** ptr; size_t n; } allocs[] = {{&c->Fxt, nFx}, {&c->Fyt, nFy}, {&c->L0, nW}, {&c->Lt0, nW}};
  for (auto& a : allocs) {
    if (cudaMalloc((void**)a.ptr, a.n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      for (auto& b : allocs) {
        if (*b.ptr) cudaFree(*b.ptr);
        *b.ptr = nullptr;
      }
      return fail(c, ASE_DF_E_NOMEM, "device allocation of %zu bytes of gas-kinetic scratch failed",
                  a.n * sizeof(double));
    }
  }
  return ASE_DF_OK;
}

static cudaError_t gks_face_fluxes(ase_df_ctx* c, const double* W, const double* sx, const double* sy,
                                   double* sxo, double* syo, double dt_fixed, cudaStream_t s,
                                   double tfrac = 0.0) {
  // as face_fluxes: in 2D the y-sweep runs on the side stream unless kernel timing is on
  const bool fork = c->dim == 2 && !c->prof_on;
  if (fork) {
    cudaError_t e = cudaEventRecord(c->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    if (e != cudaSuccess) return e;
  }
  cudaError_t err = cudaSuccess;
  for (int dir = 0; dir < c->dim && err == cudaSuccess; ++dir) {
    const cudaStream_t sd = (fork && dir == 1) ? c->side : s;
    GksSweepArgs a;
    a.tfrac = tfrac;
    a.W = W;
    a.s_norm = (dir == 0) ? sx : sy;
    a.s_tan = (dir == 0) ? sy : sx;
    a.F = (dir == 0) ? c->Fx : c->Fy;
    a.Ft = (dir == 0) ? c->Fxt : c->Fyt;
    a.s_out = (dir == 0) ? sxo : syo;
    a.st = c->st;
    a.dt_fixed = dt_fixed;
    a.inv_dn = (dir == 0) ? c->inv_dx : c->inv_dy;
    a.inv_dt = (dir == 0) ? c->inv_dy : c->inv_dx;
    a.c1 = c->p.gks_c1 > 0.0 ? c->p.gks_c1 : 0.05;
    a.c2 = c->p.gks_c2 > 0.0 ? c->p.gks_c2 : 1.0;
    ProfScope prof(c, sd, dir);
    switch (c->p.order) {
      case 3: err = launch_gks_sweep_r3(c->dim, dir, c->g, a, c->tab, c->dtab, sd); break;
      case 5: err = launch_gks_sweep_r5(c->dim, dir, c->g, a, c->tab, c->dtab, sd); break;
      case 7: err = launch_gks_sweep_r7(c->dim, dir, c->g, a, c->tab, c->dtab, sd); break;
      default: err = launch_gks_sweep_r9(c->dim, dir, c->g, a, c->tab, c->dtab, sd); break;
    }
  }
  if (fork) {  // the join is made whatever happened, so that s never runs ahead of the side stream
    cudaError_t e = cudaEventRecord(c->ev_join, c->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
    if (err == cudaSuccess) err = e;
  }
  return err;
}

static cudaError_t gks_combine(ase_df_ctx* c, int stage, const double* Wn, double* out, double* Lt_out,
                               double dt_fixed, cudaStream_t s) {
  GksCombineArgs a;
  a.Fx = c->Fx;
  a.Fxt = c->Fxt;
  a.Fy = c->Fy;
  a.Fyt = c->Fyt;
  a.Wn = Wn;
  a.out = out;
  a.Lt_out = Lt_out;
  a.L0 = c->L0;
  a.Lt0 = c->Lt0;
  a.st = c->st;
  a.inv_dx = c->inv_dx;
  a.inv_dy = c->inv_dy;
  a.dt_fixed = dt_fixed;
  a.stage = stage;
  ProfScope prof(c, s, 2);
  return launch_gks_combine(c->dim, c->g, a, s);
}

extern "C" {

ase_df_status ase_df_gks_residual(ase_df_ctx* c, const double* W, const double* sx_in, const double* sy_in, double dt,
                                  double* L, double* Lt, double* sx_out, double* sy_out, void* stream) {
  ase_df_status r = check_ptrs(c, W, sx_in, sy_in);
  if (r != ASE_DF_OK) return r;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, ASE_DF_E_INVAL, "the gas-kinetic flux needs dt > 0");
  if (!L || !Lt || !sx_out || (c->dim == 2 && !sy_out)) return fail(c, ASE_DF_E_INVAL, "NULL output pointer");
  if (sx_out == sx_in || (c->dim == 2 && sy_out == sy_in))
    return fail(c, ASE_DF_E_INVAL, "sigma_out must not alias sigma_in");
  if ((r = ensure_gks(c)) != ASE_DF_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  cudaError_t e = gks_face_fluxes(c, W, sx_in, sy_in, sx_out, sy_out, dt, s);
  if (e == cudaSuccess) e = gks_combine(c, 0, W, L, Lt, dt, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "gas-kinetic residual");
  return ASE_DF_OK;
}

ase_df_status ase_df_gks_step(ase_df_ctx* c, double* W, double* sx, double* sy, double dt, void* stream) {
  ase_df_status r = check_ptrs(c, W, sx, sy);
  if (r != ASE_DF_OK) return r;
  if (!std::isfinite(dt)) return fail(c, ASE_DF_E_INVAL, "dt is not finite");
  if ((r = ensure_gks(c)) != ASE_DF_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  cudaError_t e = cudaSuccess;
  const double dtf = (dt > 0.0) ? dt : 0.0;
  if (!(dt > 0.0)) {
    SpeedArgs sa;
    sa.W = W;
    sa.st = c->st;
    sa.inv_dx = c->inv_dx;
    sa.inv_dy = c->inv_dy;
    ProfScope prof(c, s, 3);
    e = launch_max_speed(c->dim, c->g, sa, s);
  }
  if (e == cudaSuccess) e = launch_gks_dt(c->st, dtf, c->p.cfl, c->p.t_end, c->inflow_speed, s);
  // stage 1: W* = W^n + dt/2 L + dt^2/8 L_t, sigma -> sxa, sya
  if (e == cudaSuccess) e = gks_face_fluxes(c, W, sx, sy, c->sxa, c->sya, dtf, s);
  if (e == cudaSuccess) e = gks_combine(c, 1, W, c->W1, nullptr, dtf, s);
  // stage 2: W^{n+1} from L(W^n), L_t(W^n) and L_t(W*); its sigma lands in sx, sy
  if (e == cudaSuccess) e = gks_face_fluxes(c, c->W1, c->sxa, c->sya, sx, sy, dtf, s, 0.5);  // W* at t + dt/2
  if (e == cudaSuccess) e = gks_combine(c, 2, W, W, nullptr, dtf, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "gas-kinetic step");
  return ASE_DF_OK;
}

ase_df_status ase_df_get_status(ase_df_ctx* c, uint32_t* flags, double* last_dt, double* t) {
  if (!c) return ASE_DF_E_INVAL;
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_status sync");
  DevState h;
  e = cudaMemcpy(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_status copy");
  if (flags) *flags = h.flags;
  if (last_dt) *last_dt = h.last_dt;
  if (t) *t = h.t;
  if (h.flags & ASE_DF_FLAG_SYNC) return fail(c, ASE_DF_E_TIMEOUT, "a grid barrier on the device gave up waiting");
  if (h.flags & ASE_DF_FLAG_NONPHYSICAL) return fail(c, ASE_DF_E_NONPHYSICAL, "non-physical state on the device");
  return ASE_DF_OK;
}

ase_df_status ase_df_selftest_wait(ase_df_ctx* c, void* stream) {
  if (!c) return ASE_DF_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  cudaError_t e = launch_wait_selftest(c->st, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "wait self-test");
  return ASE_DF_OK;
}

ase_df_status ase_df_profile_enable(ase_df_ctx* c, int32_t enable) {
  if (!c) return ASE_DF_E_INVAL;
  if (enable) {
    cudaDeviceSynchronize();
    prof_clear(c);
  }
  c->prof_on = enable != 0;
  return ASE_DF_OK;
}

ase_df_status ase_df_hist_enable(ase_df_ctx* c, int32_t enable) {
  if (!c) return ASE_DF_E_INVAL;
  c->hist_on = enable != 0;
  return ASE_DF_OK;
}

ase_df_status ase_df_hist_read(ase_df_ctx* c, uint64_t* counts) {
  if (!c || !counts) return c ? fail(c, ASE_DF_E_INVAL, "NULL pointer") : ASE_DF_E_INVAL;
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (e == cudaSuccess && c->side) e = cudaStreamSynchronize(c->side);
  if (e != cudaSuccess) return cuda_fail(c, e, "hist_read sync");
  unsigned long long h[kBranchSlots];
  e = cudaMemcpy(h, c->st->hist, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->st->hist, 0, sizeof(h));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "hist_read copy");
  for (int k = 0; k < kBranchSlots; ++k) counts[k] = h[k];
  return ASE_DF_OK;
}

ase_df_status ase_df_profile_read(ase_df_ctx* c, double* ms, int64_t* n) {
  if (!c || !ms || !n) return c ? fail(c, ASE_DF_E_INVAL, "NULL pointer") : ASE_DF_E_INVAL;
  for (int k = 0; k < 5; ++k) { ms[k] = 0.0; n[k] = 0; }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "profile_read sync");
  for (size_t i = 0; i < c->prof_kind->size(); ++i) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, (*c->prof_ev)[2 * i], (*c->prof_ev)[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "profile_read elapsed");
    const int k = (*c->prof_kind)[i];
    ms[k] += t;
    n[k] += 1;
  }
  return ASE_DF_OK;
}

ase_df_status ase_df_get_repair_stats(ase_df_ctx* c, uint32_t* last_stage, uint64_t* total,
                                      uint64_t* frozen) {
  if (!c) return ASE_DF_E_INVAL;
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_repair_stats sync");
  DevState h;
  e = cudaMemcpy(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_repair_stats copy");
  if (last_stage)
    for (int k = 0; k <= kRepairPasses; ++k) {
      last_stage[k] = h.cnt[k];
      last_stage[kRepairPasses + 1 + k] = h.rbad[k];
    }
  if (total) *total = h.repaired_total;
  if (frozen) *frozen = h.frozen_total;
  return ASE_DF_OK;
}

ase_df_status ase_df_reset(ase_df_ctx* c, double t, void* stream) {
  if (!c) return ASE_DF_E_INVAL;
  cudaError_t e = launch_state_kernel(c->st, 0, t, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reset");
  c->last_stream = (cudaStream_t)stream;
  return ASE_DF_OK;
}

}  // extern "C"
