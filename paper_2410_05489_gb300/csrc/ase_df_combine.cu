// Flux difference, SSP-RK3 stage combination, CFL wave-speed reduction and status
// kernels of the ASE-DF library (sm_103a, FP64).
//
//   L_ij = -(F_{i+1/2,j} - F_{i-1/2,j}) / dx - (G_{i,j+1/2} - G_{i,j-1/2}) / dy
// (Sec. 2.1, Eq. 2.3, with the Gauss-averaged face fluxes of the sweep kernels) and
//   W1 = W^n + dt L(W^n)
//   W2 = 3/4 W^n + 1/4 W1 + 1/4 dt L(W1)
//   W^{n+1} = 1/3 W^n + 2/3 W2 + 2/3 dt L(W2)          (Sec. 2.3, Eq. SSP-RK3).
//
// Positivity of a stage update (the paper falls back to a first-order scheme where
// positivity is at risk; here that is done a posteriori): the combine kernel marks every
// cell whose new average is non-physical; each repair pass gives every face of a marked
// cell the first-order Lax-Friedrichs flux of the stage's cell averages (and sigma 1e30)
// and updates again every cell next to such a face; cells that turn non-physical in a
// pass are marked for the next one.  All passes of a stage run in one cooperative launch
// with a grid barrier between them, which returns at once when the combine marked no
// cell and stops after a pass that marked none.  Last resort:
// a cell still non-physical after the passes keeps the stage's combination of W^n and
// W^(s) without the flux update (a convex combination of physical states); where
// rounding of a near-vacuum pressure still leaves p <= 0, E is raised so that
// p = 1e-13 of the kinetic energy density.  The cell is then not conservative in that
// stage, and ASE_DF_FLAG_FROZEN is raised.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "ase_df_adjoint.cuh"
#include "ase_df_combine_body.cuh"

namespace asedf {
namespace {

template <int DIM>
__global__ void __launch_bounds__(256) combine_kernel(const GridInfo g, const CombineArgs a) {
  const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  combine_range<DIM>(g, a, first, (size_t)g.nx * g.ny, stride, first == 0);
}

// Barrier over the CTAs of a cooperative launch (all co-resident), on the counters of the
// status word.  Thread 0 of each CTA arrives; the last arrival resets the count and
// advances the generation, the others wait for it.  The wait gives up after a bounded
// number of polls (about a second), raises ASE_DF_FLAG_SYNC and returns false, so that a
// barrier that cannot complete ends the kernel instead of holding the GPU.  `extra` raises the
// arrival count the barrier waits for (0 in the solver; 1 in the self-test of the wait, which
// can then never complete).
__device__ bool grid_barrier(DevState* st, unsigned int extra = 0u) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &st->bar_gen;
    const unsigned int g0 = *gen;
    __threadfence();  // this CTA's writes before the arrival
    ok = 1;
    if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1 + extra) {
      st->bar_count = 0u;
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      long long polls = 0;
      while (*gen == g0) {
        if (++polls > (1ll << 20)) {
          atomicOr(&st->flags, 0x10u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Repair passes 1..kRepairPasses and the freeze of one stage in one launch (cooperative:
// every CTA is resident).  Each pass is repair_range over the same cells per thread as the
// freeze, with a grid barrier between passes; the counters that decide whether another
// pass runs are read after the barrier, so every CTA takes the same decision.
template <int DIM>
__global__ void __launch_bounds__(256) repair_all_kernel(const GridInfo g, RepairArgs a) {
  if (__ldcg(&a.st->cnt[0]) == 0u) return;  // the stage update was physical everywhere
  const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  const size_t ncell = (size_t)g.nx * g.ny;
  for (int pass = 1; pass <= kRepairPasses; ++pass) {
    a.pass = pass;
    repair_range<DIM>(g, a, first, ncell, stride);
    if (!grid_barrier(a.st)) return;
    if (__ldcg(&a.st->cnt[pass]) == 0u) break;  // no cell turned non-physical in this pass
  }
  freeze_range<DIM>(g, a, first, ncell, stride);
}

// Self-test of the bounded wait: a barrier that expects one CTA more than the grid has.
__global__ void __launch_bounds__(256) wait_selftest_kernel(DevState* st) { grid_barrier(st, 1u); }

template <int DIM>
__global__ void __launch_bounds__(256) max_speed_kernel(const GridInfo g, const SpeedArgs a) {
  const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  max_speed_range<DIM>(g, a, first, (size_t)g.nx * g.ny, stride);
}

__global__ void state_kernel(DevState* st, int op, double t) {
  if (op == 0) {  // reset
    st->flags = 0u;
    st->t = t;
    st->dt = 0.0;
    st->last_dt = 0.0;
    st->max_speed_bits = 0ull;
    st->repaired_total = 0ull;
    st->frozen_total = 0ull;
    st->bar_count = 0u;
    st->bar_gen = 0u;
  } else if (op == 2) {  // the barrier's arrivals after a barrier that gave up
    st->bar_count = 0u;
  }
}

// out = a x + b y (the linear combinations of the SSP-RK3 adjoint)
__global__ void __launch_bounds__(256) axpby_kernel(double* out, double a, const double* x, double b,
                                                    const double* y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = y ? fma(b, y[i], a * x[i]) : a * x[i];
}

int grid_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  const size_t cap = 152 * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Threads per block of the per-cell kernels: 256, or 32 on grids of fewer than 256 cells per
// SM.  FP64 issues at 2 instructions per cycle per SM, so the per-cell FP64 work of a small
// grid runs faster spread thinly over many SMs than packed into a few 256-thread CTAs.
int cell_block(size_t n) { return n < (size_t)device_sm_count() * 256 ? 32 : 256; }

}  // namespace

cudaError_t launch_combine(int dim, const GridInfo& g, const CombineArgs& a, cudaStream_t s) {
  const size_t ncell = (size_t)g.nx * g.ny;
  const int nt = cell_block(ncell);
  if (dim == 1) combine_kernel<1><<<grid_for(ncell, nt), nt, 0, s>>>(g, a);
  else combine_kernel<2><<<grid_for(ncell, nt), nt, 0, s>>>(g, a);
  return cudaGetLastError();
}

template <int DIM>
cudaError_t repair_all_launch(const GridInfo& g, const RepairArgs& a, cudaStream_t s) {
  // resident CTAs of this kernel: its CTAs per SM (a property of the kernel on this
  // architecture, found once per dimension) times the current device's SMs
  static std::atomic<int> per_sm_cache{0};
  int per_sm = per_sm_cache.load();
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, repair_all_kernel<DIM>, 256, 0);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, per_sm);
    per_sm_cache.store(per_sm);
  }
  const int nres = per_sm * device_sm_count();
  const size_t ncell = (size_t)g.nx * g.ny;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::min<size_t>((size_t)nres, (ncell + 255) / 256));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, repair_all_kernel<DIM>, g, a);
}

cudaError_t launch_wait_selftest(DevState* st, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);  // two CTAs, both resident (cooperative launch)
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, wait_selftest_kernel, st);
  if (e != cudaSuccess) return e;
  state_kernel<<<1, 1, 0, s>>>(st, 2, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_repair_all(int dim, const GridInfo& g, const RepairArgs& a, cudaStream_t s) {
  return (dim == 1) ? repair_all_launch<1>(g, a, s) : repair_all_launch<2>(g, a, s);
}

cudaError_t launch_max_speed(int dim, const GridInfo& g, const SpeedArgs& a, cudaStream_t s) {
  const size_t ncell = (size_t)g.nx * g.ny;
  const int nt = cell_block(ncell);
  if (dim == 1) max_speed_kernel<1><<<grid_for(ncell, nt), nt, 0, s>>>(g, a);
  else max_speed_kernel<2><<<grid_for(ncell, nt), nt, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double* out, double a, const double* x, double b, const double* y, size_t n,
                         cudaStream_t s) {
  axpby_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t launch_state_kernel(DevState* st, int op, double t, cudaStream_t s) {
  state_kernel<<<1, 1, 0, s>>>(st, op, t);
  return cudaGetLastError();
}

}  // namespace asedf
