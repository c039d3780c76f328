// Device bodies of the flux difference / SSP-RK3 combination, positivity repair and CFL
// wave-speed kernels (shared by the one-problem kernels in ase_df_combine.cu and the
// batched kernels in ase_df_batch.cu).  See ase_df_combine.cu for the method.
#pragma once

#include <cuda_runtime.h>

#include "ase_df_device.cuh"
#include "ase_df_internal.cuh"

namespace asedf {
namespace {


__device__ __forceinline__ double load_dt(const CombineArgs& a) {
  return a.dt_fixed > 0.0 ? a.dt_fixed : a.st->dt;
}

__device__ __forceinline__ double rk_stage(int stage, double dt, double wn, double ws, double L) {
  if (stage == 1) return fma(dt, L, ws);
  if (stage == 2) return fma(0.25 * dt, L, fma(0.75, wn, 0.25 * ws));
  return fma((2.0 / 3.0) * dt, L, fma(1.0 / 3.0, wn, (2.0 / 3.0) * ws));
}

// The flux difference -(dFx / dx + dFy / dy) as two rounded products and one add, so
// that it is symmetric in the two directions bit for bit (a transposed problem with
// dx = dy gives the transposed result).
__device__ __forceinline__ double flux_div(double dFx, double inv_dx, double dFy, double inv_dy) {
  return -__dadd_rn(__dmul_rn(dFx, inv_dx), __dmul_rn(dFy, inv_dy));
}

// rho > 0 and p > 0, all finite, tested on p rho / (gamma - 1) = E rho - |m|^2 / 2 (no
// division; gamma > 1, so the sign is that of p); the comparisons run on the bit patterns
// (pos_finite), which decide exactly as (rho > 0) && (x > 0) && isfinite(x) for
// x = E rho - |m|^2 / 2 (an infinite rho makes x non-finite).
template <int C>
__device__ __forceinline__ bool physical_state(const double* q, double /*gamma*/) {
  double mm = q[1] * q[1];
  if (C == 4) mm = fma(q[2], q[2], mm);
  return pos_finite(q[0]) && pos_finite(fma(q[C - 1], q[0], -0.5 * mm));
}

// isfinite on the bit pattern (exponent field not all ones)
__device__ __forceinline__ bool finite_bits(double x) {
  return (dbits(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// Cells n = first, first + stride, ... < last of one problem; `leader` is true for
// exactly one thread per problem and launch.
template <int DIM>
__device__ __forceinline__ void combine_range(const GridInfo& g, const CombineArgs& a, size_t first,
                                              size_t last, size_t stride, bool leader) {
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
    if (leader) {
      a.st->dt = dt;
      if (!(dt > 0.0) || !isfinite(dt)) {
        if (!(a.t_end > 0.0 && a.st->t >= a.t_end)) atomicOr(&a.st->flags, 0x4u);
      }
    }
  } else if (a.stage > 1) {
    dt = load_dt(a);
  }
  bool bad = false;
  unsigned int nmarked = 0;
  // The stage's weight of dt L (1, 1/4, 2/3 for SSP-RK3 stages 1, 2, 3; stage 0 gives L
  // itself) is folded into the inverse spacings, so that -(dFx kx + dFy ky) is that
  // weighted update, formed as one rounded product per direction and one add (symmetric in
  // x and y bit for bit when dx = dy).
  const double wdt = (a.stage == 0) ? 1.0 : (a.stage == 1) ? dt : (a.stage == 2) ? 0.25 * dt : (2.0 / 3.0) * dt;
  const double kx = wdt * a.inv_dx, ky = wdt * a.inv_dy;
  for (size_t n = first; n < last; n += stride) {
    const int i = (int)(n % nx), j = (int)(n / nx);
    double q[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t fx = ((size_t)c * ny + j) * (nx + 1) + i;
      double t = -(a.Fx[fx + 1] - a.Fx[fx]) * kx;
      if (DIM == 2) {
        const size_t fy = ((size_t)c * (ny + 1) + j) * nx + i;
        t = flux_div(a.Fx[fx + 1] - a.Fx[fx], kx, a.Fy[fy + nx] - a.Fy[fy], ky);
      }
      const size_t w = (size_t)c * ncell + n;
      if (a.stage == 0) q[c] = t;
      else if (a.stage == 1) q[c] = a.Ws[w] + t;
      else if (a.stage == 2) q[c] = fma(0.75, a.Wn[w], fma(0.25, a.Ws[w], t));
      else q[c] = fma(1.0 / 3.0, a.Wn[w], fma(2.0 / 3.0, a.Ws[w], t));
      a.out[w] = q[c];
      if (!finite_bits(q[c])) bad = true;
    }
    if (a.stage > 0) {
      const bool ok = physical_state<C>(q, g.gamma);
      a.mark[n] = ok ? 0 : 1;
      nmarked += ok ? 0u : 1u;
    }
  }
  if (a.stage == 0 && bad) atomicOr(&a.st->flags, 0x1u);
  if (nmarked) {
    atomicAdd(&a.st->cnt[0], nmarked);
    atomicAdd(&a.st->repaired_total, (unsigned long long)nmarked);
  }
  if (a.stage == 3 && leader) {
    a.st->t += dt;
    a.st->last_dt = dt;
    a.st->max_speed_bits = 0ull;  // ready for the next CFL reduction
  }
}

__device__ __forceinline__ int across(int k, int n, int bc_lo, int bc_hi) {
  if (k >= 0 && k < n) return k;
  return ((k < 0 ? bc_lo : bc_hi) == BC_PERIODIC) ? (k < 0 ? k + n : k - n) : -1;
}

// One repair pass: cells that are marked (passes 1..pass) or next to a marked cell are
// updated again with the first-order flux on every face next to a marked cell.
template <int DIM>
__device__ __forceinline__ void repair_range(const GridInfo& g, const RepairArgs& a, size_t first,
                                             size_t last, size_t stride) {
  constexpr int C = (DIM == 1) ? 3 : 4;
  // marks and counters of other threads' cells are read through L2 (ld.cg): in the
  // single-launch repair they were written by other CTAs during this kernel
  if (__ldcg(&a.st->cnt[a.pass - 1]) == 0u) return;  // no new marks in the previous pass
  const int nx = g.nx, ny = g.ny;
  const size_t ncell = (size_t)nx * ny;
  const double dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.st->dt;
  const double ts = stage_time(a.st, a.tfrac, dt);  // for time-dependent ghosts
  const unsigned int pass = (unsigned int)a.pass;
  auto marked = [&](int i, int j) {
    const unsigned int m = __ldcg(&a.mark[(size_t)j * nx + i]);
    return m >= 1u && m <= pass;
  };
  unsigned int nnew = 0, nbad = 0;
  for (size_t n = first; n < last; n += stride) {
    const int i = (int)(n % nx), j = (int)(n / nx);
    const bool self = marked(i, j);
    const int il = across(i - 1, nx, g.bc[0], g.bc[1]), ir = across(i + 1, nx, g.bc[0], g.bc[1]);
    const bool fL = self || (il >= 0 && marked(il, j));
    const bool fR = self || (ir >= 0 && marked(ir, j));
    bool fD = false, fU = false;
    if (DIM == 2) {
      const int jd = across(j - 1, ny, g.bc[2], g.bc[3]), ju = across(j + 1, ny, g.bc[2], g.bc[3]);
      fD = self || (jd >= 0 && marked(i, jd));
      fU = self || (ju >= 0 && marked(i, ju));
    }
    if (!(fL || fR || fD || fU)) continue;
    double F[2][2][C];  // [dir][lower / upper face][component]
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int f = i + side;
      if (side == 0 ? fL : fR) {
        double cl[C], cr[C], F2[C], sg;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          cl[c] = fetch_w(g, a.Ws, c, f - 1, j, ts);
          cr[c] = fetch_w(g, a.Ws, c, f, j, ts);
        }
        lf_point<C, 1, 2>(cl, cr, cl, cr, 1, g.gm1, g.gg1, F2, sg);
#pragma unroll
        for (int c = 0; c < C; ++c) F[0][side][c] = 0.5 * F2[c];
        a.sx_out[(size_t)j * (nx + 1) + f] = kSigmaBig;
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) F[0][side][c] = a.Fx[((size_t)c * ny + j) * (nx + 1) + f];
      }
      if (DIM == 2) {
        const int fy = j + side;
        if (side == 0 ? fD : fU) {
          double cl[C], cr[C], F2[C], sg;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            cl[c] = fetch_w(g, a.Ws, c, i, fy - 1, ts);
            cr[c] = fetch_w(g, a.Ws, c, i, fy, ts);
          }
          lf_point<C, 2, 1>(cl, cr, cl, cr, 1, g.gm1, g.gg1, F2, sg);
#pragma unroll
          for (int c = 0; c < C; ++c) F[1][side][c] = 0.5 * F2[c];
          a.sy_out[(size_t)fy * nx + i] = kSigmaBig;
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) F[1][side][c] = a.Fy[((size_t)c * (ny + 1) + fy) * nx + i];
        }
      }
    }
    double q[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      double L = -(F[0][1][c] - F[0][0][c]) * a.inv_dx;
      if (DIM == 2) L = flux_div(F[0][1][c] - F[0][0][c], a.inv_dx, F[1][1][c] - F[1][0][c], a.inv_dy);
      const size_t w = (size_t)c * ncell + n;
      q[c] = rk_stage(a.stage, dt, a.Wn[w], a.Ws[w], L);
      a.out[w] = q[c];
    }
    if (!physical_state<C>(q, g.gamma)) {
      ++nbad;
      if (a.mark[n] == 0) {
        a.mark[n] = (unsigned char)(pass + 1);
        ++nnew;
      }
    }
  }
  if (nnew) {
    atomicAdd(&a.st->cnt[pass], nnew);
    atomicAdd(&a.st->repaired_total, (unsigned long long)nnew);
  }
  if (nbad) atomicAdd(&a.st->rbad[pass], nbad);
}

// Last resort after the repair passes (see the file comment).
template <int DIM>
__device__ __forceinline__ void freeze_range(const GridInfo& g, const RepairArgs& a, size_t first,
                                             size_t last, size_t stride) {
  constexpr int C = (DIM == 1) ? 3 : 4;
  if (__ldcg(&a.st->cnt[0]) == 0u) return;  // the stage update was physical everywhere
  const size_t ncell = (size_t)g.nx * g.ny;
  const double dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.st->dt;
  unsigned int nfrozen = 0;
  bool still_bad = false;
  for (size_t n = first; n < last; n += stride) {
    double q[C];
#pragma unroll
    for (int c = 0; c < C; ++c) q[c] = a.out[(size_t)c * ncell + n];
    if (physical_state<C>(q, g.gamma)) continue;
#pragma unroll
    for (int c = 0; c < C; ++c) q[c] = rk_stage(a.stage, dt, a.Wn[(size_t)c * ncell + n], a.Ws[(size_t)c * ncell + n], 0.0);
    if (!physical_state<C>(q, g.gamma) && q[0] > 0.0 && isfinite(q[C - 1])) {
      // a pressure at the rounding level of E (near vacuum): floor it at 1e-13 of the
      // kinetic energy density by adjusting E
      double mm = q[1] * q[1];
      if (C == 4) mm = fma(q[2], q[2], mm);
      const double ke = 0.5 * mm / q[0];
      q[C - 1] = ke + 1e-13 * fmax(ke, fabs(q[C - 1])) / (g.gamma - 1.0);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) a.out[(size_t)c * ncell + n] = q[c];
    ++nfrozen;
    if (!physical_state<C>(q, g.gamma)) still_bad = true;
  }
  if (nfrozen) {
    atomicAdd(&a.st->frozen_total, (unsigned long long)nfrozen);
    atomicOr(&a.st->flags, 0x8u);
  }
  if (still_bad) atomicOr(&a.st->flags, 0x1u);
}

// max over cells of (|u|+c)/dx [+ (|v|+c)/dy]; non-physical cells raise the flag.
template <int DIM>
__device__ __forceinline__ void max_speed_range(const GridInfo& g, const SpeedArgs& a, size_t first,
                                                size_t last, size_t stride) {
  constexpr int C = (DIM == 1) ? 3 : 4;
  const size_t ncell = (size_t)g.nx * g.ny;
  double smax = 0.0;
  bool bad = false;
  for (size_t n = first; n < last; n += stride) {
    double q[C];
#pragma unroll
    for (int c = 0; c < C; ++c) q[c] = a.W[(size_t)c * ncell + n];
    if (!physical_state<C>(q, g.gamma)) {
      bad = true;
      continue;
    }
    const double rho = q[0];
    const double inv_rho = 1.0 / rho;
    const double u = q[1] * inv_rho;
    const double v = (C == 4) ? q[2] * inv_rho : 0.0;
    const double p = (g.gamma - 1.0) * (q[C - 1] - 0.5 * rho * (u * u + v * v));
    const double c = sqrt(fmax(g.gamma * p * inv_rho, 0.0));
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

}  // namespace
}  // namespace asedf
