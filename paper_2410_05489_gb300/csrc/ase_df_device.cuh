// Device helpers shared by the sweep kernel and the combine / repair kernels: ghost-cell
// index maps (periodic wrap, zero-gradient clamp, mirror at a reflecting wall, x-lo inflow
// band) and the local Lax-Friedrichs flux with the discontinuity strength of one Gauss
// point.
#pragma once

#include <cuda_runtime.h>

#include "ase_df_internal.cuh"

namespace asedf {
namespace {

constexpr double kSigmaBig = 1e30;  // sigma of a Gauss point that took first-order states

// ---------------------------------------------------------------------------------
// FP64-pipe economy.  This part issues FP64 at 2 lanes per cycle per SM and the face
// kernel is bound by that pipe, so comparisons whose outcome the bit patterns fix run
// as integer operations, and the reciprocal and reciprocal square root of the flux
// start from an FP32 approximation (XU pipe) refined by one FP64 step of order three.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// x > 0 and finite: sign bit clear, not +0, exponent field not all ones (so false for
// NaN, +-0, negative values and +inf), as (x > 0 && isfinite(x)).
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = dbits(x);
  return b > 0 && b < 0x7ff0000000000000LL;
}

// a < t for a threshold t > 0: non-negative values (and +NaN) order like their bit
// patterns, and negative values (and -0) have the sign bit set and compare below.
// Equals (a < t) except for a NaN with the sign bit set.
__device__ __forceinline__ bool lt_pos(double a, double t) { return dbits(a) < dbits(t); }

// max of two non-negative values, by bit pattern
__device__ __forceinline__ double max_nonneg(double a, double b) { return dbits(a) < dbits(b) ? b : a; }

// 1/x for x > 0 with biased exponent in [3, 2044] (otherwise the division).  Seed: the
// FP32 reciprocal approximation of the leading 23 mantissa bits (x scaled into [1, 2)),
// relative error below 2^-22.  Then one step of the third-order Newton-Raphson
// (Householder) iteration for 1/x: with e = 1 - x y0, 1/x = y0 / (1 - e) =
// y0 (1 + e + e^2 + ...), so y1 = y0 + y0 (e + e^2), error O(e^3) < 2^-64 before the
// final rounding.
__device__ __forceinline__ double rcp_pos(double x) {
  const long long b = dbits(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (b <= 0 || ex < 3 || ex > 2044) return 1.0 / x;
  const unsigned fb = 0x3f800000u | (unsigned)((b >> 29) & 0x7fffff);
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__uint_as_float(fb)));
  // r ~ 1/m in [1/2, 1]; 1/x = r 2^(1023 - ex)
  const unsigned rb = __float_as_uint(r);
  const long long er = (long long)((rb >> 23) & 0xffu) - 127 + 1023 + (1023 - ex);
  const double y0 = __longlong_as_double((er << 52) | ((long long)(rb & 0x7fffffu) << 29));
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// 1/sqrt(x) for x > 0 normal and finite (otherwise rsqrt()).  Seed: the FP32 rsqrt
// approximation of x scaled by an even power of two into [1, 4).  Then one third-order
// step: with r = 1 - x y0^2, 1/sqrt(x) = y0 (1 - r)^(-1/2) = y0 (1 + r/2 + 3 r^2 / 8 + ...),
// so y1 = y0 + y0 r (1/2 + 3 r / 8), error O(r^3) < 2^-62 before rounding.
__device__ __forceinline__ double rsqrt_pos(double x) {
  const long long b = dbits(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (b <= 0 || ex < 1 || ex > 2046) return rsqrt(x);
  const int e = ex - 1023;   // x = 1.f 2^e
  const int par = e & 1;     // e = 2k + par
  const int k = (e - par) >> 1;
  const unsigned fb = ((unsigned)(127 + par) << 23) | (unsigned)((b >> 29) & 0x7fffff);
  float sf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(sf) : "f"(__uint_as_float(fb)));
  // sf ~ 1/sqrt(m) in [1/2, 1]; 1/sqrt(x) = sf 2^-k
  const unsigned sb = __float_as_uint(sf);
  const long long es = (long long)((sb >> 23) & 0xffu) - 127 + 1023 - k;
  const double y0 = __longlong_as_double((es << 52) | ((long long)(sb & 0x7fffffu) << 29));
  const double h = x * y0;
  const double r = fma(-h, y0, 1.0);
  return fma(y0 * r, fma(r, 0.375, 0.5), y0);
}

// cell index 0..n-1 of a (ghost) cell; a reflecting wall mirrors about its face (the
// ghost layers reach at most k+1 <= n cells deep, which the context validates); the wall
// part of a BC_WALL_AFTER boundary mirrors too (its fixed part is handled by the callers)
__device__ __forceinline__ int wrap_or_clamp(int i, int n, int bc_lo, int bc_hi) {
  if (i < 0) {
    if (bc_lo == BC_PERIODIC) { int m = i % n; return m < 0 ? m + n : m; }
    if (bc_lo == BC_REFLECT || bc_lo == BC_WALL_AFTER) return -1 - i;
    return 0;
  }
  if (i >= n) {
    if (bc_hi == BC_PERIODIC) return i % n;
    if (bc_hi == BC_REFLECT) return 2 * n - 1 - i;
    return n - 1;
  }
  return i;
}

// face index 0..n along a direction with n cells
__device__ __forceinline__ int face_map(int f, int n, int bc_lo, int bc_hi) {
  if (f >= 0 && f <= n) return f;
  if (f < 0) {
    if (bc_lo == BC_PERIODIC) { int m = f % n; return m < 0 ? m + n : m; }
    if (bc_lo == BC_REFLECT || bc_lo == BC_WALL_AFTER) return -f;
    return 0;
  }
  if (bc_hi == BC_PERIODIC) return f % n;
  if (bc_hi == BC_REFLECT) return 2 * n - f;
  return n;
}

// Time of a stage: st->t + tfrac dt (exactly st->t for tfrac = 0)
__device__ __forceinline__ double stage_time(const DevState* st, double tfrac, double dt) {
  return tfrac == 0.0 ? st->t : __dadd_rn(st->t, __dmul_rn(tfrac, dt));
}

// Component c of (ghost) cell (i, j) at time ts (the time-dependent BC_MOVING_SHOCK ghosts).
__device__ __forceinline__ double fetch_w(const GridInfo& g, const double* __restrict__ W, int c,
                                          int i, int j, double ts) {
  if (i < 0 && g.bc[0] == BC_INFLOW_BAND && j >= g.band_j0 && j <= g.band_j1) return g.inflow_cons[c];
  if (j < 0 && g.bc[2] == BC_WALL_AFTER && i < g.wall_i0) return g.inflow_cons[c];
  if (j >= g.ny && g.bc[3] == BC_MOVING_SHOCK) {
    // ghost centre against the shock position, each rounded once
    const double xc = __dadd_rn(g.x0, __dmul_rn((double)i + 0.5, g.dx));
    const double xs = __dadd_rn(g.shock_x0, __dmul_rn(g.shock_speed, ts));
    return xc < xs ? g.inflow_cons[c] : g.state_b_cons[c];
  }
  const int ii = wrap_or_clamp(i, g.nx, g.bc[0], g.bc[1]);
  const int jj = wrap_or_clamp(j, g.ny, g.bc[2], g.bc[3]);
  const double v = __ldg(W + ((size_t)c * g.ny + jj) * g.nx + ii);
  // a reflecting wall flips the momentum normal to it (x-walls: c = 1; y-walls, 2D: c = 2)
  const bool fx = (c == 1) && ((i < 0 && g.bc[0] == BC_REFLECT) || (i >= g.nx && g.bc[1] == BC_REFLECT));
  const bool fy = (c == 2) && ((j < 0 && (g.bc[2] == BC_REFLECT || g.bc[2] == BC_WALL_AFTER)) ||
                               (j >= g.ny && g.bc[3] == BC_REFLECT));
  return (fx || fy) ? -v : v;
}

// sigma of x-face f (index before the boundary map) on (ghost) row j; below a
// BC_WALL_AFTER boundary the rows of x-faces whose right-hand column is before the wall
// clamp (fixed ghosts), the others mirror
__device__ __forceinline__ double sigma_x_at(const GridInfo& g, const double* __restrict__ s, int f, int j) {
  const int jj = (j < 0 && g.bc[2] == BC_WALL_AFTER && f < g.wall_i0) ? 0 : wrap_or_clamp(j, g.ny, g.bc[2], g.bc[3]);
  return __ldg(s + (size_t)jj * (g.nx + 1) + face_map(f, g.nx, g.bc[0], g.bc[1]));
}

// sigma of y-face f (index before the boundary map) of (ghost) column i; the fixed part of
// a BC_WALL_AFTER boundary clamps, its wall part mirrors
__device__ __forceinline__ double sigma_y_at(const GridInfo& g, const double* __restrict__ s, int f, int i) {
  const int ff = (f < 0 && g.bc[2] == BC_WALL_AFTER && i < g.wall_i0) ? 0 : face_map(f, g.ny, g.bc[2], g.bc[3]);
  return __ldg(s + (size_t)ff * g.nx + wrap_or_clamp(i, g.nx, g.bc[0], g.bc[1]));
}

// Local Lax-Friedrichs flux (Sec. 2.3) and discontinuity strength sigma (Sec. 3.1) of
// one Gauss point; qa / qb are the left / right states in (x, y) momentum order and
// NI / TI select the normal and tangential momentum.  A state is physical when rho > 0
// and p > 0 (both finite); otherwise the point takes the cell averages ca / cb
// (component c at ca[c * cs], read only in that case), returns true and sets
// sigma = 1e30.  gm1 = gamma - 1 and gg1 = gamma (gamma - 1) come from the caller.
//
// The FP64 pipe bounds the face kernels, so the point is arranged for few FP64
// instructions (58 in 2D on the physical path, its Gauss-weighted accumulation included):
//   - one reciprocal gives 1/rho of both sides: 1/rho_l = rho_r / (rho_l rho_r);
//   - the pressure is kept as p' = p / (gamma - 1) = E - (m_n u_n + m_t u_t) / 2, so that
//     (gamma - 1) multiplies only the sums that need it;
//   - c^2 = gamma p / rho = gg1 p' / rho and 1/c from a seeded reciprocal square root;
//     c = c^2 / c;
//   - 1/p' = gg1 (1/rho) (1/c)^2 gives the pressure term of sigma without a reciprocal;
//   - the flux sum F_l + F_r - lambda (q_r - q_l) is formed per component as
//     q_l (u_l + lambda) + q_r (u_r - lambda) + pressure terms, and accumulated into the
//     caller's Gauss sum in the same FMAs.
// The point adds w (2F) to Fs (w: the Gauss weight with the 1/2 of the L-F formula folded
// in; gw = (gamma - 1) w), with w folded into the speeds u +- lambda so that each component
// takes two FMAs on top of its pressure term.
// Primitives of the two states of a Gauss point (face frame: NI normal, TI tangential
// momentum): 1/rho, u_n, u_t and p' = p / (gamma - 1) of each side, from one reciprocal.
struct LfPrims {
  double irL, irR, unL, unR, utL, utR, pL, pR;
};

template <int C, int NI, int TI>
__device__ __forceinline__ LfPrims lf_primitives(const double* a, const double* b) {
  LfPrims s;
  const double irr = rcp_pos(a[0] * b[0]);
  s.irL = b[0] * irr;
  s.irR = a[0] * irr;
  s.unL = a[NI] * s.irL;
  s.unR = b[NI] * s.irR;
  double kL = a[NI] * s.unL, kR = b[NI] * s.unR;  // |m|^2 / rho
  s.utL = s.utR = 0.0;
  if (C == 4) {
    s.utL = a[TI] * s.irL;
    s.utR = b[TI] * s.irR;
    kL = fma(a[TI], s.utL, kL);
    kR = fma(b[TI], s.utR, kR);
  }
  s.pL = fma(-0.5, kL, a[C - 1]);
  s.pR = fma(-0.5, kR, b[C - 1]);
  return s;
}

// Both states physical: rho > 0 and p > 0, all finite (on the bit patterns).
__device__ __forceinline__ bool lf_physical(double rhoL, double rhoR, const LfPrims& s) {
  return pos_finite(rhoL) && pos_finite(rhoR) && pos_finite(s.pL) && pos_finite(s.pR);
}

template <int C, int NI, int TI>
__device__ __forceinline__ bool lf_point_acc(const double* qa, const double* qb, const double* ca,
                                             const double* cb, int cs, double gm1, double gg1, double w,
                                             double gw, double* Fs, double& sigma) {
  double a[C], b[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    a[c] = qa[c];
    b[c] = qb[c];
  }
  LfPrims s = lf_primitives<C, NI, TI>(a, b);
  const bool ok = lf_physical(a[0], b[0], s);
  if (!ok) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      a[c] = ca[c * cs];
      b[c] = cb[c * cs];
    }
    s = lf_primitives<C, NI, TI>(a, b);
  }
  const double irL = s.irL, irR = s.irR, unL = s.unL, unR = s.unR, utL = s.utL, utR = s.utR;
  const double pL = s.pL, pR = s.pR;
  const double c2L = (gg1 * pL) * irL, c2R = (gg1 * pR) * irR;
  const double icL = rsqrt_pos(c2L), icR = rsqrt_pos(c2R);
  // lambda = max(|u_n| + c) with c = c^2 / c
  const double lam = max_nonneg(fma(c2L, icL, fabs(unL)), fma(c2R, icR, fabs(unR)));
  const double alL = w * (unL + lam), alR = w * (unR - lam);
  Fs[0] = fma(a[0], alL, fma(b[0], alR, Fs[0]));
  Fs[NI] = fma(a[NI], alL, fma(b[NI], alR, fma(gw, pL + pR, Fs[NI])));
  if (C == 4) Fs[TI] = fma(a[TI], alL, fma(b[TI], alR, Fs[TI]));
  Fs[C - 1] = fma(a[C - 1], alL, fma(b[C - 1], alR, fma(gw, fma(unL, pL, unR * pR), Fs[C - 1])));
  if (ok) {
    // sigma = |dp| (1/p_l + 1/p_r) + (dMa_n)^2 + (dMa_t)^2, Ma = u / c
    const double dmn = fma(unL, icL, -unR * icR);
    double s = dmn * dmn;
    if (C == 4) {
      const double dmt = fma(utL, icL, -utR * icR);
      s = fma(dmt, dmt, s);
    }
    const double tL = irL * icL, tR = irR * icR;
    const double ip = fma(tL, icL, tR * icR);  // (1/p'_l + 1/p'_r) / gg1
    sigma = fma(gg1 * fabs(pL - pR), ip, s);
  } else {
    sigma = kSigmaBig;
  }
  return !ok;
}

// The flux of one point as 2F = F_l + F_r - lambda (q_r - q_l), and sigma (lf_point_acc with
// weight 1).
template <int C, int NI, int TI>
__device__ __forceinline__ bool lf_point(const double* qa, const double* qb, const double* ca,
                                         const double* cb, int cs, double gm1, double gg1, double* F2,
                                         double& sigma) {
#pragma unroll
  for (int c = 0; c < C; ++c) F2[c] = 0.0;
  return lf_point_acc<C, NI, TI>(qa, qb, ca, cb, cs, gm1, gg1, 1.0, gm1, F2, sigma);
}

}  // namespace
}  // namespace asedf
