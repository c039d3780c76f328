// Flux difference, SSP-RK3 stage combination, CFL wave-speed reduction and status
// kernels of the ASE-DF library (sm_103a, FP64).
//
//   L_ij = -(F_{i+1/2,j} - F_{i-1/2,j}) / dx - (G_{i,j+1/2} - G_{i,j-1/2}) / dy
// (Sec. 2.1, Eq. 2.3, with the Gauss-averaged face fluxes of the sweep kernels) and
//   W1 = W^n + dt L(W^n)
//   W2 = 3/4 W^n + 1/4 W1 + 1/4 dt L(W1)
//   W^{n+1} = 1/3 W^n + 2/3 W2 + 2/3 dt L(W2)          (Sec. 2.3, Eq. SSP-RK3).
//
// Positivity of a stage update (the paper's "transition to a first-order scheme for
// preserving positivity", done a posteriori): the combine kernel marks every cell whose
// new average is non-physical; each repair pass gives every face of a marked cell the
// first-order Lax-Friedrichs flux of the stage's cell averages (and sigma 1e30) and
// updates again every cell next to such a face; cells that turn non-physical in a pass
// are marked for the next one.  Passes with nothing to do return at once.  Last resort:
// a cell still non-physical after the passes keeps the stage's combination of W^n and
// W^(s) without the flux update (a convex combination of physical states); where
// rounding of a near-vacuum pressure still leaves p <= 0, E is raised so that
// p = 1e-13 of the kinetic energy density.  The cell is then not conservative in that
// stage, and ASE_DF_FLAG_FROZEN is raised.

#include <cuda_runtime.h>

#include "ase_df_adjoint.cuh"
#include "ase_df_combine_body.cuh"

namespace asedf {
namespace {

template <int DIM>
__global__ void __launch_bounds__(256) combine_kernel(const GridInfo g, const CombineArgs a) {
  const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  combine_range<DIM>(g, a, first, (size_t)g.nx * g.ny, stride, first == 0);
}

template <int DIM>
__global__ void __launch_bounds__(256) repair_kernel(const GridInfo g, const RepairArgs a) {
  const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  repair_range<DIM>(g, a, first, (size_t)g.nx * g.ny, stride);
}

template <int DIM>
__global__ void __launch_bounds__(256) freeze_kernel(const GridInfo g, const RepairArgs a) {
  const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  freeze_range<DIM>(g, a, first, (size_t)g.nx * g.ny, stride);
}

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

}  // namespace

cudaError_t launch_combine(int dim, const GridInfo& g, const CombineArgs& a, cudaStream_t s) {
  const size_t ncell = (size_t)g.nx * g.ny;
  if (dim == 1) combine_kernel<1><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  else combine_kernel<2><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_repair(int dim, const GridInfo& g, const RepairArgs& a, cudaStream_t s) {
  const size_t ncell = (size_t)g.nx * g.ny;
  if (dim == 1) repair_kernel<1><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  else repair_kernel<2><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_freeze(int dim, const GridInfo& g, const RepairArgs& a, cudaStream_t s) {
  const size_t ncell = (size_t)g.nx * g.ny;
  if (dim == 1) freeze_kernel<1><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  else freeze_kernel<2><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_max_speed(int dim, const GridInfo& g, const SpeedArgs& a, cudaStream_t s) {
  const size_t ncell = (size_t)g.nx * g.ny;
  if (dim == 1) max_speed_kernel<1><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  else max_speed_kernel<2><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
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
