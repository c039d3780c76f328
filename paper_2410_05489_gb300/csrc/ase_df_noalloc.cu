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
// array's name as a device address: each call looks the address up with
// cudaGetSymbolAddress (with the caller's device current) unless the stream is being
// captured, in which case it takes the address an earlier call on that device found.
// So the first call on each device must come before any stream capture, and a lookup
// outside capture also picks up a new address after cudaDeviceReset.  The problem is
// validated and described to the kernels by the same code as in ase_df_init, and the
// kernels are the ones ase_df_residual launches, so the results are the same bit for
// bit.  The reconstruction tables are built once per (dimension, order) by the library's
// exact rational builder, which uses fixed-size arrays only.
//
// Sharing: every call uses the same array, and it keeps the last call's contents.
// The face fluxes are fully rewritten by each call; the status word is cleared at the
// start of each call.  Calls that overlap on the GPU (different streams, or different
// host threads) race on the array and must not be issued.

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
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
static_assert(sizeof(DevState) <= kStatusDoubles * sizeof(double),
              "the status word must fit in the space reserved before the face fluxes");

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Tables per (dimension, order), built on first use.
Tables g_tables[2][4];
bool g_have_tables[2][4] = {{false}};

// The message goes to the buffer ase_df_last_error(NULL) returns.
ase_df_status nfail(ase_df_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(init_error_buffer(), 512, fmt, ap);
  va_end(ap);
  return s;
}

}  // namespace
}  // namespace asedf

using namespace asedf;

extern "C" ase_df_status ase_df_residual_noalloc(const ase_df_params* pin, const double* W,
                                                 const double* sx_in, const double* sy_in,
                                                 double* L, double* sx_out, double* sy_out,
                                                 void* stream) {
  ProblemSetup ps;
  {
    const ase_df_status v = setup_problem(pin, &ps, init_error_buffer(), 512);
    if (v != ASE_DF_OK) return v;
  }
  const ase_df_params& p = ps.p;
  if (p.bc[3] == ASE_DF_BC_MOVING_SHOCK)
    return nfail(ASE_DF_E_INVAL,
                 "the moving-shock boundary depends on the solver time, which only a context holds; "
                 "use ase_df_init / ase_df_reset / ase_df_residual");
  if (!W || !sx_in || !L || !sx_out || (p.ndim == 2 && (!sy_in || !sy_out)))
    return nfail(ASE_DF_E_INVAL, "NULL array pointer");
  if (sx_out == sx_in || (p.ndim == 2 && sy_out == sy_in))
    return nfail(ASE_DF_E_INVAL, "sigma_out must not alias sigma_in");

  const int C = ps.C;
  const size_t nx = (size_t)p.nx, ny = (size_t)p.ny;
  const size_t nFx = (size_t)C * ny * (nx + 1);
  const size_t nFy = (p.ndim == 2) ? (size_t)C * (ny + 1) * nx : 0;
  if (kStatusDoubles + nFx + nFy > kScratchDoubles)
    return nfail(ASE_DF_E_BOUNDS,
                 "grid too large for the fixed scratch: needs %zu face-flux doubles, the limit is %zu "
                 "(2^21 doubles = 16 MiB minus the status word); use ase_df_init / ase_df_residual",
                 nFx + nFy, kScratchDoubles - kStatusDoubles);

  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(ASE_DF_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nfail(ASE_DF_E_BOUNDS, "device index %d >= %d", dev, kMaxDevices);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;  // unknown: take the cached address, look nothing up
  }
  double* base = nullptr;
  const Tables* tab = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
      // the device address of the scratch array (it changes if the device was reset)
      void* a = nullptr;
      e = cudaGetSymbolAddress(&a, g_scratch);
      if (e != cudaSuccess) return nfail(ASE_DF_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<double*>(a);
    } else if (!g_scratch_ptr[dev]) {
      return nfail(ASE_DF_E_INVAL,
                   "the first call on device %d came during stream capture; make one call before capturing", dev);
    }
    base = g_scratch_ptr[dev];
    const int di = p.ndim - 1, oi = (p.order - 3) / 2;
    if (!g_have_tables[di][oi]) {
      if (!build_tables(p.order, p.ndim, &g_tables[di][oi]))
        return nfail(ASE_DF_E_INVAL, "table construction failed");
      g_have_tables[di][oi] = true;
    }
    tab = &g_tables[di][oi];
  }

  GridInfo g = ps.g;
  set_flux_weights(g, *tab);
  DevState* st = reinterpret_cast<DevState*>(base);
  double* Fx = base + kStatusDoubles;
  double* Fy = Fx + nFx;

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
      case 3: e = launch_sweep_r3(p.ndim, dir, g, a, *tab, s); break;
      case 5: e = launch_sweep_r5(p.ndim, dir, g, a, *tab, s); break;
      case 7: e = launch_sweep_r7(p.ndim, dir, g, a, *tab, s); break;
      default: e = launch_sweep_r9(p.ndim, dir, g, a, *tab, s); break;
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
  c.inv_dx = ps.inv_dx;
  c.inv_dy = ps.inv_dy;
  c.stage = 0;
  e = launch_combine(p.ndim, g, c, s);
  if (e != cudaSuccess) return nfail(ASE_DF_E_CUDA, "combine: %s", cudaGetErrorString(e));
  return ASE_DF_OK;
}
