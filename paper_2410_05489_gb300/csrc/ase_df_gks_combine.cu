// Stage kernels of the gas-kinetic path: flux differences of the face fluxes and of their
// time derivatives, and the two-stage fourth-order update (Sec. 2.2, Eq. S2O4):
//   W*      = W^n + dt/2 L(W^n) + dt^2/8 L_t(W^n)
//   W^{n+1} = W^n + dt L(W^n) + dt^2/6 (L_t(W^n) + 2 L_t(W*)).
// The CFL step is fixed before the first face kernel (its flux integrals need dt).

#include <cuda_runtime.h>

#include "ase_df_combine_body.cuh"
#include "ase_df_gks.cuh"

namespace asedf {
namespace {

template <int DIM>
__global__ void __launch_bounds__(256) gks_combine_kernel(const GridInfo g, const GksCombineArgs a) {
  constexpr int C = (DIM == 1) ? 3 : 4;
  const int nx = g.nx, ny = g.ny;
  const size_t ncell = (size_t)nx * ny;
  const double dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.st->dt;
  bool bad = false;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < ncell; n += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % nx), j = (int)(n / nx);
    double q[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t fx = ((size_t)c * ny + j) * (nx + 1) + i;
      double L = -(a.Fx[fx + 1] - a.Fx[fx]) * a.inv_dx;
      double Lt = -(a.Fxt[fx + 1] - a.Fxt[fx]) * a.inv_dx;
      if (DIM == 2) {
        const size_t fy = ((size_t)c * (ny + 1) + j) * nx + i;
        L = flux_div(a.Fx[fx + 1] - a.Fx[fx], a.inv_dx, a.Fy[fy + nx] - a.Fy[fy], a.inv_dy);
        Lt = flux_div(a.Fxt[fx + 1] - a.Fxt[fx], a.inv_dx, a.Fyt[fy + nx] - a.Fyt[fy], a.inv_dy);
      }
      const size_t w = (size_t)c * ncell + n;
      if (a.stage == 0) {
        a.out[w] = L;
        a.Lt_out[w] = Lt;
        q[c] = L;
      } else if (a.stage == 1) {
        a.L0[w] = L;
        a.Lt0[w] = Lt;
        q[c] = a.Wn[w] + 0.5 * dt * L + 0.125 * dt * dt * Lt;
        a.out[w] = q[c];
      } else {
        q[c] = a.Wn[w] + dt * a.L0[w] + (1.0 / 6.0) * dt * dt * (a.Lt0[w] + 2.0 * Lt);
        a.out[w] = q[c];
      }
    }
    if (a.stage == 0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
        if (!isfinite(q[c])) bad = true;
    } else if (!physical_state<C>(q, g.gamma)) {
      bad = true;
    }
  }
  if (bad) atomicOr(&a.st->flags, 0x1u);
  if (a.stage == 2 && blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->t += dt;
    a.st->last_dt = dt;
    a.st->max_speed_bits = 0ull;
  }
}

__global__ void gks_dt_kernel(DevState* st, double dt_fixed, double cfl, double t_end, double inflow_speed) {
  double dt;
  if (dt_fixed > 0.0) {
    dt = dt_fixed;
  } else {
    const double smax = fmax(__longlong_as_double((long long)st->max_speed_bits), inflow_speed);
    dt = cfl / smax;
    if (t_end > 0.0) dt = fmax(0.0, fmin(dt, t_end - st->t));
  }
  st->dt = dt;
  if (!(dt > 0.0) || !isfinite(dt)) {
    if (!(t_end > 0.0 && st->t >= t_end)) atomicOr(&st->flags, 0x4u);
  }
}

int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_gks_combine(int dim, const GridInfo& g, const GksCombineArgs& a, cudaStream_t s) {
  const size_t ncell = (size_t)g.nx * g.ny;
  if (dim == 1) gks_combine_kernel<1><<<grid_for(ncell), 256, 0, s>>>(g, a);
  else gks_combine_kernel<2><<<grid_for(ncell), 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_gks_dt(DevState* st, double dt_fixed, double cfl, double t_end, double inflow_speed,
                          cudaStream_t s) {
  gks_dt_kernel<<<1, 1, 0, s>>>(st, dt_fixed, cfl, t_end, inflow_speed);
  return cudaGetLastError();
}

}  // namespace asedf
