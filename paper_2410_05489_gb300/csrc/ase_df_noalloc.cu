// ase_df_residual_noalloc: the residual entry point for callers that cannot allocate
// device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaFree are off limits -- inside a
// region being captured into a CUDA graph by someone else, a real-time loop that must
// not synchronise the device (cudaFree does), or a host framework that owns every
// device byte through its own pool and forbids other allocations.  ase_df_init cannot
// serve them, because the context allocates its scratch.
//
// How: the face fluxes that ase_df_residual keeps in context-owned scratch live here in
// one file-scope __device__ array of fixed size instead.  Every GPU that loads this
// library holds that array (16 MiB) until the process exits.  Host code cannot use the
// array's name as a device address; the first call on each device looks the address
// up with cudaGetSymbolAddress (with that device current) and caches it, so make that
// first call before any stream capture.  The kernels are the same ones ase_df_residual
// launches.  The reconstruction tables are built on the stack by exact rational
// arithmetic (no heap, no device allocation).
//
// Sharing: every call uses the same array, and it keeps the last call's contents.
// The face fluxes are fully rewritten by each call; the status word is cleared at the
// start of each call.  Calls that overlap on the GPU (different streams, or different
// host threads) race on the array and must not be issued.

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/ase_df.h"
#include "ase_df_internal.cuh"

namespace asedf {
namespace {

// 2^21 doubles = 16 MiB: the status word (first 256 bytes) and the face fluxes
// Fx [C][ny][nx+1] and Fy [C][ny+1][nx].
constexpr size_t kScratchDoubles = size_t(1) << 21;
constexpr size_t kStatusDoubles = 32;  // 256 bytes reserved for DevState

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// The status code is the whole error report (this entry point has no context to hold
// a message); the text documents each case at its call site.
ase_df_status nfail(ase_df_status s, const char* /*why*/, ...) { return s; }

// ---------------------------------------------------------------------------------
// Tables without heap memory: the same cell-average moment problem as the library's
// table builder, solved with fixed-size 128-bit rational arrays on the stack.
// ---------------------------------------------------------------------------------
typedef __int128 i128;

struct Q {
  i128 n, d;
};

i128 qgcd(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}
Q qmk(i128 n, i128 d) {
  if (d < 0) { n = -n; d = -d; }
  i128 g = qgcd(n, d);
  if (g == 0) g = 1;
  return Q{n / g, d / g};
}
Q qadd(Q a, Q b) { return qmk(a.n * b.d + b.n * a.d, a.d * b.d); }
Q qsub(Q a, Q b) { return qmk(a.n * b.d - b.n * a.d, a.d * b.d); }
Q qmul(Q a, Q b) { return qmk(a.n * b.n, a.d * b.d); }
Q qdiv(Q a, Q b) { return qmk(a.n * b.d, a.d * b.n); }
long double qld(Q a) { return (long double)a.n / (long double)a.d; }

// inv[q][i]: coefficient of xi^q per unit average in stencil cell i (n <= 9 cells).
bool moment_inverse_fixed(const int* offs, int n, Q inv[9][9]) {
  Q A[9][18];
  for (int i = 0; i < n; ++i) {
    for (int q = 0; q < n; ++q) {
      i128 hi = 1, lo = 1;
      for (int e = 0; e < q + 1; ++e) { hi *= offs[i]; lo *= (offs[i] - 1); }
      A[i][q] = qmk(hi - lo, q + 1);
    }
    for (int j = 0; j < n; ++j) A[i][n + j] = qmk(i == j ? 1 : 0, 1);
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    while (piv < n && A[piv][col].n == 0) ++piv;
    if (piv == n) return false;
    for (int j = 0; j < 2 * n; ++j) { Q t = A[piv][j]; A[piv][j] = A[col][j]; A[col][j] = t; }
    Q pv = A[col][col];
    for (int j = 0; j < 2 * n; ++j) A[col][j] = qdiv(A[col][j], pv);
    for (int r = 0; r < n; ++r) {
      if (r == col || A[r][col].n == 0) continue;
      Q f = A[r][col];
      for (int j = 0; j < 2 * n; ++j) A[r][j] = qsub(A[r][j], qmul(f, A[col][j]));
    }
  }
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i) inv[q][i] = A[q][n + i];
  return true;
}

void gauss_legendre_fixed(int G, long double* t, long double* w) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < G; ++i) {
    long double x = cosl(pi * (i + 0.75L) / (G + 0.5L)), dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = x;
      for (int k = 2; k <= G; ++k) {
        long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = G * (x * p1 - p0) / (x * x - 1);
      long double dx = p1 / dp;
      x -= dx;
      if (fabsl(dx) < 1e-30L) break;
    }
    t[G - 1 - i] = 0.5L * (x + 1);
    w[G - 1 - i] = 1.0L / ((1 - x * x) * dp * dp);
  }
}

double point_weight(Q inv[9][9], int n, int i, int p, const long double* gt) {
  if (p <= 1) {  // xi = 0 or -1, exact
    Q s = qmk(0, 1), xp = qmk(1, 1), xi = qmk(p == 0 ? 0 : -1, 1);
    for (int q = 0; q < n; ++q) {
      s = qadd(s, qmul(xp, inv[q][i]));
      xp = qmul(xp, xi);
    }
    return (double)qld(s);
  }
  const long double xi = gt[p - 2] - 1.0L;
  long double s = 0;
  for (int q = n - 1; q >= 0; --q) s = s * xi + qld(inv[q][i]);
  return (double)s;
}

bool build_tables_fixed(int r, int ndim, Tables* T) {
  std::memset(T, 0, sizeof(Tables));
  const int G = (ndim == 2) ? (r == 3 ? 1 : (r - 1) / 2) : 1;
  long double gt[4], gwt[4];
  gauss_legendre_fixed(G, gt, gwt);
  for (int g = 0; g < G; ++g) {
    T->gw[g] = (double)gwt[g];
    T->hgw[g] = (double)(0.5L * gwt[g]);
  }
  const int npts = 2 + G;
  Q inv[9][9];
  for (int b = 0; b < 4; ++b) {
    const int h = b + 1, n = 2 * h + 1;
    int offs[9];
    for (int i = 0; i < n; ++i) offs[i] = i - h;
    if (!moment_inverse_fixed(offs, n, inv)) return false;
    for (int p = 0; p < npts; ++p)
      for (int i = 0; i < n; ++i) T->lin[b][p][4 - h + i] = point_weight(inv, n, i, p, gt);
  }
  {
    const int h = (r - 1) / 2, n = 2 * h + 1;
    int offs[9];
    for (int i = 0; i < n; ++i) offs[i] = i - h;
    if (!moment_inverse_fixed(offs, n, inv)) return false;
    for (int g = 0; g < (G + 1) / 2 && g < 2; ++g) {
      long double w[9];
      const long double xi = gt[g] - 1.0L;
      for (int i = 0; i < n; ++i) {
        long double sacc = 0;
        for (int q = n - 1; q >= 0; --q) sacc = sacc * xi + qld(inv[q][i]);
        w[i] = sacc;
      }
      T->se[g][0] = (double)w[h];
      for (int t = 1; t <= h; ++t) {
        T->se[g][t] = (double)(0.5L * (w[h + t] + w[h - t]));
        T->so[g][t] = (double)(0.5L * (w[h + t] - w[h - t]));
      }
    }
  }
  for (int k = 0; k < 3; ++k) {
    int offs[3] = {k - 2, k - 1, k};
    if (!moment_inverse_fixed(offs, 3, inv)) return false;
    for (int p = 0; p < npts; ++p)
      for (int j = 0; j < 3; ++j) T->sub[k][p][j] = point_weight(inv, 3, j, p, gt);
    for (int q = 0; q < 2; ++q)
      for (int j = 0; j < 3; ++j) T->cq[k][q][j] = (double)qld(inv[q + 1][j]);
  }
  T->d5 = (double)qld(qmk(85, 100));
  T->d3[0] = (double)qld(qmk(15 * 15, 100 * 100 * 2));
  T->d3[1] = (double)qld(qmk(15 * 85, 100 * 100));
  T->d3[2] = T->d3[0];
  T->eps = 1e-6;
  return true;
}

}  // namespace
}  // namespace asedf

using namespace asedf;

extern "C" ase_df_status ase_df_residual_noalloc(const ase_df_params* pin, const double* W,
                                                 const double* sx_in, const double* sy_in,
                                                 double* L, double* sx_out, double* sy_out,
                                                 void* stream) {
  if (!pin) return nfail(ASE_DF_E_INVAL, "params is NULL");
  ase_df_params p = *pin;
  if (p.ndim != 1 && p.ndim != 2) return nfail(ASE_DF_E_INVAL, "ndim must be 1 or 2");
  if (p.order != 3 && p.order != 5 && p.order != 7 && p.order != 9)
    return nfail(ASE_DF_E_INVAL, "order must be 3, 5, 7 or 9");
  if (p.ndim == 1) p.ny = 1;
  if (p.nx < 1 || p.ny < 1 || p.nx > (1 << 20) || p.ny > (1 << 20))
    return nfail(ASE_DF_E_INVAL, "nx, ny must be in [1, 2^20]");
  if (!(p.x1 > p.x0) || (p.ndim == 2 && !(p.y1 > p.y0))) return nfail(ASE_DF_E_INVAL, "empty domain");
  if (!(p.gamma > 1.0) || !(p.sigma_thres > 0.0)) return nfail(ASE_DF_E_INVAL, "gamma must be > 1, sigma_thres > 0");
  for (int s = 0; s < 4; ++s) {
    if (p.bc[s] < 0 || p.bc[s] > 2 || (p.bc[s] == ASE_DF_BC_INFLOW_BAND && s != 0))
      return nfail(ASE_DF_E_INVAL, "bad boundary code %d on side %d", p.bc[s], s);
    if (p.ndim == 1 && s >= 2) p.bc[s] = ASE_DF_BC_OUTFLOW;
  }
  if ((p.bc[0] == ASE_DF_BC_PERIODIC) != (p.bc[1] == ASE_DF_BC_PERIODIC) ||
      (p.ndim == 2 && (p.bc[2] == ASE_DF_BC_PERIODIC) != (p.bc[3] == ASE_DF_BC_PERIODIC)))
    return nfail(ASE_DF_E_INVAL, "periodic boundaries must come in pairs");
  if (!W || !sx_in || !L || !sx_out || (p.ndim == 2 && (!sy_in || !sy_out)))
    return nfail(ASE_DF_E_INVAL, "NULL array pointer");
  if (sx_out == sx_in || (p.ndim == 2 && sy_out == sy_in))
    return nfail(ASE_DF_E_INVAL, "sigma_out must not alias sigma_in");

  const int C = (p.ndim == 1) ? 3 : 4;
  const size_t nx = (size_t)p.nx, ny = (size_t)p.ny;
  const size_t nFx = (size_t)C * ny * (nx + 1);
  const size_t nFy = (p.ndim == 2) ? (size_t)C * (ny + 1) * nx : 0;
  if (kStatusDoubles + nFx + nFy > kScratchDoubles)
    return nfail(ASE_DF_E_BOUNDS,
                 "grid too large for the fixed scratch: needs %zu face-flux doubles, the limit is %zu "
                 "(2^21 doubles = 16 MiB minus the status word); use ase_df_init / ase_df_residual",
                 nFx + nFy, kScratchDoubles - kStatusDoubles);

  // once per device: the device address of the scratch array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(ASE_DF_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nfail(ASE_DF_E_BOUNDS, "device index %d >= %d", dev, kMaxDevices);
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* a = nullptr;
      e = cudaGetSymbolAddress(&a, g_scratch);
      if (e != cudaSuccess) return nfail(ASE_DF_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<double*>(a);
    }
    base = g_scratch_ptr[dev];
  }

  Tables tab;
  if (!build_tables_fixed(p.order, p.ndim, &tab)) return nfail(ASE_DF_E_INVAL, "table construction failed");

  GridInfo g;
  std::memset(&g, 0, sizeof(g));
  g.nx = (int)p.nx;
  g.ny = (int)p.ny;
  for (int s = 0; s < 4; ++s) g.bc[s] = p.bc[s];
  g.band_j0 = 1;
  g.band_j1 = 0;
  const double dx = (p.x1 - p.x0) / (double)p.nx;
  const double dy = (p.ndim == 2) ? (p.y1 - p.y0) / (double)p.ny : 1.0;
  if (p.bc[0] == ASE_DF_BC_INFLOW_BAND) {
    if (!(p.inflow_state[0] > 0.0 && p.inflow_state[3] > 0.0))
      return nfail(ASE_DF_E_INVAL, "inflow state must have rho > 0 and p > 0");
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
  }
  g.gamma = p.gamma;
  g.thres = p.sigma_thres;

  DevState* st = reinterpret_cast<DevState*>(base);
  double* Fx = base + kStatusDoubles;
  double* Fy = Fx + nFx;
  cudaStream_t s = (cudaStream_t)stream;

  e = launch_state_kernel(st, 0, 0.0, s);  // clear the status word of the previous call
  if (e != cudaSuccess) return nfail(ASE_DF_E_CUDA, "status reset: %s", cudaGetErrorString(e));
  for (int dir = 0; dir < p.ndim; ++dir) {
    SweepArgs a;
    a.W = W;
    a.s_norm = (dir == 0) ? sx_in : sy_in;
    a.s_tan = (dir == 0) ? sy_in : sx_in;
    a.F = (dir == 0) ? Fx : Fy;
    a.s_out = (dir == 0) ? sx_out : sy_out;
    a.st = st;
    switch (p.order) {
      case 3: e = launch_sweep_r3(p.ndim, dir, g, a, tab, s); break;
      case 5: e = launch_sweep_r5(p.ndim, dir, g, a, tab, s); break;
      case 7: e = launch_sweep_r7(p.ndim, dir, g, a, tab, s); break;
      default: e = launch_sweep_r9(p.ndim, dir, g, a, tab, s); break;
    }
    if (e != cudaSuccess) return nfail(ASE_DF_E_CUDA, "sweep: %s", cudaGetErrorString(e));
  }
  CombineArgs c;
  std::memset(&c, 0, sizeof(c));
  c.Fx = Fx;
  c.Fy = (p.ndim == 2) ? Fy : nullptr;
  c.Wn = W;
  c.Ws = W;
  c.out = L;
  c.st = st;
  c.inv_dx = 1.0 / dx;
  c.inv_dy = (p.ndim == 2) ? 1.0 / dy : 0.0;
  c.stage = 0;
  e = launch_combine(p.ndim, g, c, s);
  if (e != cudaSuccess) return nfail(ASE_DF_E_CUDA, "combine: %s", cudaGetErrorString(e));
  return ASE_DF_OK;
}
