// Flux difference, SSP-RK3 stage combination, CFL wave-speed reduction and status
// kernels of the ASE-DF library (sm_103a, FP64).
//
//   L_ij = -(F_{i+1/2,j} - F_{i-1/2,j}) / dx - (G_{i,j+1/2} - G_{i,j-1/2}) / dy
// (Sec. 2.1, Eq. 2.3, with the Gauss-averaged face fluxes of the sweep kernels) and
//   W1 = W^n + dt L(W^n)
//   W2 = 3/4 W^n + 1/4 W1 + 1/4 dt L(W1)
//   W^{n+1} = 1/3 W^n + 2/3 W2 + 2/3 dt L(W2)          (Sec. 2.3, Eq. SSP-RK3).

#include <cuda_runtime.h>

#include "ase_df_internal.cuh"

namespace asedf {
namespace {

__device__ __forceinline__ double load_dt(const CombineArgs& a) {
  return a.dt_fixed > 0.0 ? a.dt_fixed : a.st->dt;
}

template <int DIM>
__global__ void __launch_bounds__(256) combine_kernel(const GridInfo g, const CombineArgs a) {
  constexpr int C = (DIM == 1) ? 3 : 4;
  const int nx = g.nx, ny = g.ny;
  const size_t ncell = (size_t)nx * ny;
  double dt = 0.0;
  if (a.stage == 1) {
    if (a.dt_fixed > 0.0) {
      dt = a.dt_fixed;
    } else {
      const double smax = fmax(__longlong_as_double((long long)a.st->max_speed_bits), a.inflow_speed);
      dt = a.cfl / smax;
      if (a.t_end > 0.0) dt = fmax(0.0, fmin(dt, a.t_end - a.st->t));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.st->dt = dt;
      if (!(dt > 0.0) || !isfinite(dt)) {
        if (!(a.t_end > 0.0 && a.st->t >= a.t_end)) atomicOr(&a.st->flags, 0x4u);
      }
    }
  } else if (a.stage > 1) {
    dt = load_dt(a);
  }
  bool bad = false;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < ncell; n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % nx), j = (int)(n / nx);
    double rho_out = 1.0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t fx = ((size_t)c * ny + j) * (nx + 1) + i;
      double L = -(a.Fx[fx + 1] - a.Fx[fx]) * a.inv_dx;
      if (DIM == 2) {
        const size_t fy = ((size_t)c * (ny + 1) + j) * nx + i;
        L = fma(-(a.Fy[fy + nx] - a.Fy[fy]), a.inv_dy, L);
      }
      const size_t w = (size_t)c * ncell + n;
      double out;
      if (a.stage == 0) {
        out = L;
      } else if (a.stage == 1) {
        out = fma(dt, L, a.Ws[w]);
      } else if (a.stage == 2) {
        out = fma(0.25 * dt, L, fma(0.75, a.Wn[w], 0.25 * a.Ws[w]));
      } else {
        out = fma((2.0 / 3.0) * dt, L, fma(1.0 / 3.0, a.Wn[w], (2.0 / 3.0) * a.Ws[w]));
      }
      a.out[w] = out;
      if (c == 0) rho_out = out;
      if (!isfinite(out)) bad = true;
    }
    if (a.stage == 3 && !(rho_out > 0.0)) bad = true;
  }
  if (bad) atomicOr(&a.st->flags, 0x1u);
  if (a.stage == 3 && blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->t += dt;
    a.st->last_dt = dt;
    a.st->max_speed_bits = 0ull;  // ready for the next CFL reduction
  }
}

// max over cells of (|u|+c)/dx [+ (|v|+c)/dy]; non-physical cells raise the flag.
template <int DIM>
__global__ void __launch_bounds__(256) max_speed_kernel(const GridInfo g, const SpeedArgs a) {
  constexpr int C = (DIM == 1) ? 3 : 4;
  const size_t ncell = (size_t)g.nx * g.ny;
  double smax = 0.0;
  bool bad = false;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < ncell; n += (size_t)gridDim.x * blockDim.x) {
    const double rho = a.W[n];
    const double inv_rho = 1.0 / rho;
    const double u = a.W[ncell + n] * inv_rho;
    const double v = (C == 4) ? a.W[2 * ncell + n] * inv_rho : 0.0;
    const double E = a.W[(C - 1) * ncell + n];
    const double p = (g.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    if (!(rho > 0.0) || !(p > 0.0) || !isfinite(p) || !isfinite(u) || !isfinite(v)) {
      bad = true;
      continue;
    }
    const double c = sqrt(g.gamma * p * inv_rho);
    double s = (fabs(u) + c) * a.inv_dx;
    if (C == 4) s = fma(fabs(v) + c, a.inv_dy, s);
    smax = fmax(smax, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if ((threadIdx.x & 31) == 0 && smax > 0.0)
    atomicMax(&a.st->max_speed_bits, (unsigned long long)__double_as_longlong(smax));
  if (bad) atomicOr(&a.st->flags, 0x1u);
}

__global__ void state_kernel(DevState* st, int op, double t) {
  if (op == 0) {  // reset
    st->flags = 0u;
    st->t = t;
    st->dt = 0.0;
    st->last_dt = 0.0;
    st->max_speed_bits = 0ull;
  }
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

cudaError_t launch_max_speed(int dim, const GridInfo& g, const SpeedArgs& a, cudaStream_t s) {
  const size_t ncell = (size_t)g.nx * g.ny;
  if (dim == 1) max_speed_kernel<1><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  else max_speed_kernel<2><<<grid_for(ncell, 256), 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_state_kernel(DevState* st, int op, double t, cudaStream_t s) {
  state_kernel<<<1, 1, 0, s>>>(st, op, t);
  return cudaGetLastError();
}

}  // namespace asedf
