// Hand-written adjoint (vector-Jacobian product) of the ASE-DF residual of one sweep
// direction, sm_103a, FP64.  Compiled once per scheme order (ASE_DF_ORDER).
//
// The forward residual of one direction is, per face f of line b,
//   Q_s(line l)   = normal reconstruction of the cell of side s on line l (Sec. 3)
//   q_s,g         = tangential reconstruction of Q_s at Gauss point g (Sec. 2.1)
//   F_f           = sum_g (eta_g / 2) LF2(q_L,g, q_R,g)    (Sec. 2.3)
//   sigma_f       = (1/G) sum_g sigma(q_L,g, q_R,g)          (Sec. 3.1)
//   L(i)          = -(F_{i+1} - F_i) / dx   (+ the other direction)
// The adjoint runs it backwards in deterministic kernels (every output element is
// written by one thread; no atomics):
//   K1 face kernel: recomputes the tile like the forward sweep, forms
//      Fbar_f = (Lbar(f) - Lbar(f-1)) / dx, back-propagates through the Gauss sum, the
//      Lax-Friedrichs flux (|.| and max taken piecewise, on the branch of the forward
//      value), sigma_out and the tangential reconstruction of each side.  It writes, per
//      face, side and tangential offset t, the adjoint of Q_s(line b+t) (Tbar); the
//      adjoint of the two cell averages where a Gauss point took the first-order states
//      (Cbar); and the sigma_in adjoints of the tangential branch (Stb).
//   K2 normal kernel: per reconstructing cell (a, l) gathers the adjoints of its plus
//      face value (face a+1) and minus face value (face a) from Tbar and back-propagates
//      through the normal reconstruction: the adjoint of each stencil cell (Nbar) and
//      the sigma_in adjoints of the normal branch (Snb).
//   K3 gather: per cell, sums the Nbar and Cbar entries of every stencil position that
//      the boundary maps onto it (periodic wrap, zero-gradient clamp; inflow ghost cells
//      are constants) into Wbar.
//   K4 / K5 gathers: per sigma_in entry (normal / tangential faces), sum Snb / Stb over
//      the stencil positions that read it.
// Branch decisions (Algorithm 1) are recomputed from the same sigma_in and held fixed;
// at a kink of |x| or max whose argument is within a relative 2^-40 of it, the
// symmetric subgradient is taken (kKink below).
// Within a branch the reconstruction is differentiated as defined: constant weights on
// the linear branches; on the WENOZ-AO(5,3) branch the WENO-Z weights (beta, tau_Z, |.|
// piecewise) and the DF factors alpha = sigma_thres / A of Eq. (3.2), whose derivative
// -alpha^2 / sigma_thres carries the adjoint to the face strengths summed in A.

#include <algorithm>
#include <cuda_runtime.h>

#include "ase_df_adjoint.cuh"
#include "ase_df_sweep_body.cuh"

#ifndef ASE_DF_ORDER
#error "ASE_DF_ORDER must be defined"
#endif

namespace asedf {
namespace {

// Kinks: |x| and max(a, b) have no derivative at x = 0 and a = b.  Where the argument is
// within a relative 2^-40 of the kink its side is decided by rounding (it differs
// between two correct evaluations, and between the two sides of a central difference),
// so the adjoint takes the symmetric subgradient there: 0 for |x|, one half to each
// operand of max.
constexpr double kKink = 9.094947017729282e-13;  // 2^-40

// d|x|/dx with that rule; scale > 0 is the size x is compared with
__device__ __forceinline__ double dabs(double x, double scale) {
  if (fabs(x) <= kKink * scale) return 0.0;
  return (x < 0.0) ? -1.0 : 1.0;
}

// Scratch layouts of one direction: face f (0..n) of line b (0..m-1), and reconstructing
// cell a (-1..n) of line l (-KT..m-1+KT).  The index runs fastest along the direction in
// which the state arrays are contiguous (along the sweep for x-faces, along the lines for
// y-faces), so that the threads of a warp, which the kernels also order that way, touch
// consecutive addresses.
template <int DIR>
__device__ __forceinline__ size_t adj_face(int f, int b, int n, int m) {
  return (DIR == 0) ? (size_t)b * (n + 1) + f : (size_t)f * m + b;
}
template <int DIR>
__device__ __forceinline__ size_t adj_item(int a, int l, int n, int m, int KT) {
  return (DIR == 0) ? (size_t)(l + KT) * (n + 2) + (a + 1) : (size_t)(a + 1) * (m + 2 * KT) + (l + KT);
}

// ---------------------------------------------------------------------------------
// reconstruction VJPs.  Stencil values v[t*vs] (t = -K..K); vbc points at the adjoint
// of W_0 in a unit-stride array; ab[0..2] accumulate the adjoints of alpha of S3_{-1},
// S3_0, S3_1 and ab[3] that of alpha of S5 (or of S3_0 for the DF-damped order 3).
// ---------------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void lin_vjp(const double* w, double pb, double* vbc) {
  constexpr int H = (M - 1) / 2;
#pragma unroll
  for (int t = -H; t <= H; ++t) vbc[t] = fma(w[4 + t], pb, vbc[t]);
}

// WENOZ-AO(5,3) with DF damping (Sec. 3.2); pb[q] is the adjoint of the value at point
// p0+q.
template <int NP>
__device__ void weno_vjp(const double* v, int vs, const Branch& br, const Tables& T, int p0, const double* pb,
                         double* vbc, double* ab) {
  double c1[3], c2[3], beta[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double* vk = v + (k - 2) * vs;
    c1[k] = T.cq[k][0][0] * vk[0] + T.cq[k][0][1] * vk[vs] + T.cq[k][0][2] * vk[2 * vs];
    c2[k] = T.cq[k][1][0] * vk[0] + T.cq[k][1][1] * vk[vs] + T.cq[k][1][2] * vk[2 * vs];
    beta[k] = c1[k] * (c1[k] - 2.0 * c2[k]) + (16.0 / 3.0) * c2[k] * c2[k];
  }
  const double s02 = dabs(beta[0] - beta[2], beta[0] + beta[2]);
  const double b5 = (beta[0] + 4.0 * beta[1] + beta[2]) * (1.0 / 6.0) + fabs(beta[0] - beta[2]);
  double sk[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) sk[k] = dabs(b5 - beta[k], b5 + beta[k]);
  const double tau = (fabs(b5 - beta[0]) + fabs(b5 - beta[1]) + fabs(b5 - beta[2])) * (1.0 / 3.0);
  const double e5 = b5 + T.eps;
  const double w5 = T.d5 * (1.0 + tau * tau / (e5 * e5));
  double e[3], w3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    e[k] = beta[k] + T.eps;
    w3[k] = T.d3[k] * (1.0 + tau * tau / (e[k] * e[k]));
  }
  const double inv = 1.0 / (w5 + w3[0] + w3[1] + w3[2]);
  const double g5 = w5 * inv / T.d5;
  double g3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) g3[k] = w3[k] * inv - g5 * T.d3[k];
  const double W0 = v[0];
  // P = g5 P5 + sum_k g3_k P3_k,  P5 = W0 + a5 (L5 - W0),  P3_k = W0 + a3_k (u_k - W0)
  double gb5 = 0.0, gb3[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int p = p0 + q;
    const double L5 = lin_eval<5>(v, vs, T.lin[1][p]);
    gb5 = fma(pb[q], fma(br.a5, L5 - W0, W0), gb5);
    const double pb5 = pb[q] * g5;
    ab[3] = fma(pb5, L5 - W0, ab[3]);
    lin_vjp<5>(T.lin[1][p], br.a5 * pb5, vbc);
    vbc[0] = fma(1.0 - br.a5, pb5, vbc[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double* vk = v + (k - 2) * vs;
      const double u = T.sub[k][p][0] * vk[0] + T.sub[k][p][1] * vk[vs] + T.sub[k][p][2] * vk[2 * vs];
      gb3[k] = fma(pb[q], fma(br.a3[k], u - W0, W0), gb3[k]);
      const double pb3 = pb[q] * g3[k];
      ab[k] = fma(pb3, u - W0, ab[k]);
      const double a = br.a3[k] * pb3;
      vbc[k - 2] = fma(T.sub[k][p][0], a, vbc[k - 2]);
      vbc[k - 1] = fma(T.sub[k][p][1], a, vbc[k - 1]);
      vbc[k] = fma(T.sub[k][p][2], a, vbc[k]);
      vbc[0] = fma(1.0 - br.a3[k], pb3, vbc[0]);
    }
  }
  // g3_k = w3_k inv - g5 d3_k,  g5 = w5 inv / d5,  inv = 1 / (w5 + sum w3)
  double wb3[3], invb = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    wb3[k] = gb3[k] * inv;
    invb = fma(gb3[k], w3[k], invb);
    gb5 -= gb3[k] * T.d3[k];
  }
  double wb5 = gb5 * inv / T.d5;
  invb += gb5 * w5 / T.d5;
  const double Sb = -invb * inv * inv;
  wb5 += Sb;
#pragma unroll
  for (int k = 0; k < 3; ++k) wb3[k] += Sb;
  // w = d (1 + tau^2 / (beta + eps)^2)
  double taub = wb5 * T.d5 * 2.0 * tau / (e5 * e5);
  double b5b = -wb5 * T.d5 * 2.0 * tau * tau / (e5 * e5 * e5);
  double betab[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    taub += wb3[k] * T.d3[k] * 2.0 * tau / (e[k] * e[k]);
    betab[k] = -wb3[k] * T.d3[k] * 2.0 * tau * tau / (e[k] * e[k] * e[k]);
  }
  // tau = (|b5 - beta_0| + |b5 - beta_1| + |b5 - beta_2|) / 3
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    b5b += taub * sk[k] * (1.0 / 3.0);
    betab[k] -= taub * sk[k] * (1.0 / 3.0);
  }
  // b5 = (beta_0 + 4 beta_1 + beta_2) / 6 + |beta_0 - beta_2|
  betab[0] += b5b * (1.0 / 6.0 + s02);
  betab[1] += b5b * (4.0 / 6.0);
  betab[2] += b5b * (1.0 / 6.0 - s02);
  // beta = c1^2 - 2 c1 c2 + (16/3) c2^2
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double c1b = betab[k] * (2.0 * c1[k] - 2.0 * c2[k]);
    const double c2b = betab[k] * (-2.0 * c1[k] + (32.0 / 3.0) * c2[k]);
#pragma unroll
    for (int j = 0; j < 3; ++j) vbc[k - 2 + j] += T.cq[k][0][j] * c1b + T.cq[k][1][j] * c2b;
  }
}

// VJP of recon_eval<R, NP> (points p0 .. p0+NP-1).
template <int R, int NP>
__device__ __forceinline__ void recon_vjp(const double* v, int vs, const Branch& br, const Tables& T, int p0,
                                          const double* pb, double* vbc, double* ab) {
  if (br.m == R) {
#pragma unroll
    for (int q = 0; q < NP; ++q) lin_vjp<R>(T.lin[(R - 3) / 2][p0 + q], pb[q], vbc);
    return;
  }
  if (R == 3) {  // DF-damped order 3: W0 + a (lin3 - W0)
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const double l3 = lin_eval<3>(v, vs, T.lin[0][p0 + q]);
      ab[3] = fma(pb[q], l3 - v[0], ab[3]);
      lin_vjp<3>(T.lin[0][p0 + q], br.a5 * pb[q], vbc);
      vbc[0] = fma(1.0 - br.a5, pb[q], vbc[0]);
    }
    return;
  }
  if (R >= 9 && br.m == 7) {
#pragma unroll
    for (int q = 0; q < NP; ++q) lin_vjp<(R >= 7 ? 7 : 3)>(T.lin[2][p0 + q], pb[q], vbc);
    return;
  }
  if (R >= 7 && br.m == 5) {
#pragma unroll
    for (int q = 0; q < NP; ++q) lin_vjp<5>(T.lin[1][p0 + q], pb[q], vbc);
    return;
  }
  if (R >= 5) weno_vjp<NP>(v, vs, br, T, p0, pb, vbc, ab);
}

// Adjoints of the four face strengths sigma_{-3/2}, sigma_{-1/2}, sigma_{1/2}, sigma_{3/2}
// of a stencil (sb[0..3]) from the alpha adjoints ab.  alpha = thres / A where
// A >= thres (Eq. 3.2), so d alpha / d A = -alpha^2 / thres; alpha = 1 elsewhere.
template <int R>
__device__ __forceinline__ void sigma_vjp(const Branch& br, const double* ab, double thres, double* sb) {
  sb[0] = sb[1] = sb[2] = sb[3] = 0.0;
  if (R == 3) {
    if (br.m == -3) {
      const double Ab = -ab[3] * br.a5 * br.a5 / thres;  // A = sigma_{-1/2} + sigma_{1/2}
      sb[1] = Ab;
      sb[2] = Ab;
    }
    return;
  }
  if (br.m != 0) return;
  const double A5b = -ab[3] * br.a5 * br.a5 / thres;
  double A3b[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) A3b[k] = (br.a3[k] < 1.0) ? -ab[k] * br.a3[k] * br.a3[k] / thres : 0.0;
  // A3_{-1} = s_{-3/2} + s_{-1/2}, A3_0 = s_{-1/2} + s_{1/2}, A3_1 = s_{1/2} + s_{3/2}, A5 = all four
  sb[0] = A3b[0] + A5b;
  sb[1] = A3b[0] + A3b[1] + A5b;
  sb[2] = A3b[1] + A3b[2] + A5b;
  sb[3] = A3b[2] + A5b;
}

// ---------------------------------------------------------------------------------
// Lax-Friedrichs point VJP (the derivative of lf_point_acc)
// ---------------------------------------------------------------------------------
// The forward point, in the primitives of lf_primitives (p' = p / (gamma - 1)):
//   2F_c  = a_c (u_L + lambda) + b_c (u_R - lambda) + P_c,
//           P = (0, (gamma-1)(p'_L + p'_R), 0, (gamma-1)(u_L p'_L + u_R p'_R)) (face frame)
//   lambda = max(|u_L| + c_L, |u_R| + c_R),  c^2 = gamma (gamma-1) p' / rho,  ic = 1 / c
//   sigma = (u_L ic_L - u_R ic_R)^2 + (w_L ic_L - w_R ic_R)^2
//           + gamma (gamma-1) |p'_L - p'_R| (ic_L^2 / rho_L + ic_R^2 / rho_R)
// and p' = E - (m_n u + m_t w) / 2, u = m_n / rho, w = m_t / rho.  Given F2b (adjoint of 2F)
// and sb (adjoint of sigma, used only on a physical point: a first-order point has the
// constant sigma 1e30), sets ab / bb to the adjoints of the states a / b.  |x| and max take
// the symmetric subgradient near their kinks (reading G23, kKink).
// s = lf_primitives(a, b).
template <int C, int NI, int TI>
__device__ __forceinline__ void lf_point_vjp(const double* a, const double* b, const LfPrims& s, double gm1,
                                             double gg1, const double* F2b, double sb, bool physical, double* ab,
                                             double* bb) {
  const double c2L = (gg1 * s.pL) * s.irL, c2R = (gg1 * s.pR) * s.irR;
  const double icL = rsqrt_pos(c2L), icR = rsqrt_pos(c2R);
  const double cL = c2L * icL, cR = c2R * icR;
  const double sL = fabs(s.unL) + cL, sR = fabs(s.unR) + cR;
  const double lam = fmax(sL, sR);
  // direct terms of 2F and the adjoints of u, p', lambda
  double uLb = 0.0, uRb = 0.0, lamb = 0.0;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    ab[c] = F2b[c] * (s.unL + lam);
    bb[c] = F2b[c] * (s.unR - lam);
    uLb = fma(F2b[c], a[c], uLb);
    uRb = fma(F2b[c], b[c], uRb);
    lamb = fma(F2b[c], a[c] - b[c], lamb);
  }
  uLb = fma(F2b[C - 1] * gm1, s.pL, uLb);
  uRb = fma(F2b[C - 1] * gm1, s.pR, uRb);
  double pLb = gm1 * fma(F2b[C - 1], s.unL, F2b[NI]);
  double pRb = gm1 * fma(F2b[C - 1], s.unR, F2b[NI]);
  // lambda = max(s_L, s_R), s = |u| + c
  double tL = (sL < sR) ? 0.0 : 1.0;
  if (fabs(sL - sR) <= kKink * (sL + sR)) tL = 0.5;
  const double sLb = tL * lamb, sRb = (1.0 - tL) * lamb;
  uLb = fma(sLb, dabs(s.unL, cL), uLb);
  uRb = fma(sRb, dabs(s.unR, cR), uRb);
  double cLb = sLb, cRb = sRb, icLb = 0.0, icRb = 0.0, irLb = 0.0, irRb = 0.0, wLb = 0.0, wRb = 0.0;
  if (physical && sb != 0.0) {
    const double dmn = fma(s.unL, icL, -s.unR * icR);
    const double gn = 2.0 * sb * dmn;
    uLb = fma(gn, icL, uLb);
    uRb = fma(-gn, icR, uRb);
    icLb = fma(gn, s.unL, icLb);
    icRb = fma(-gn, s.unR, icRb);
    if (C == 4) {
      const double dmt = fma(s.utL, icL, -s.utR * icR);
      const double gt = 2.0 * sb * dmt;
      wLb = gt * icL;
      wRb = -gt * icR;
      icLb = fma(gt, s.utL, icLb);
      icRb = fma(-gt, s.utR, icRb);
    }
    const double dp = s.pL - s.pR;
    const double S = fma(s.irL * icL, icL, s.irR * icR * icR);
    const double gp = sb * gg1 * dabs(dp, s.pL + s.pR) * S;
    pLb += gp;
    pRb -= gp;
    const double Sb = sb * gg1 * fabs(dp);
    irLb = Sb * icL * icL;
    irRb = Sb * icR * icR;
    icLb = fma(2.0 * Sb * s.irL, icL, icLb);
    icRb = fma(2.0 * Sb * s.irR, icR, icRb);
  }
  // c = sqrt(c^2), ic = 1 / sqrt(c^2): dc/dc^2 = ic / 2, d ic / dc^2 = -ic^3 / 2;
  // c^2 = gamma (gamma-1) p' / rho
  const double c2Lb = 0.5 * icL * fma(-icLb, icL * icL, cLb);
  const double c2Rb = 0.5 * icR * fma(-icRb, icR * icR, cRb);
  pLb = fma(c2Lb * gg1, s.irL, pLb);
  pRb = fma(c2Rb * gg1, s.irR, pRb);
  irLb = fma(c2Lb * gg1, s.pL, irLb);
  irRb = fma(c2Rb * gg1, s.pR, irRb);
  // p' = E - (m_n u + m_t w) / 2
  ab[C - 1] += pLb;
  bb[C - 1] += pRb;
  ab[NI] = fma(-0.5 * pLb, s.unL, ab[NI]);
  bb[NI] = fma(-0.5 * pRb, s.unR, bb[NI]);
  uLb = fma(-0.5 * pLb, a[NI], uLb);
  uRb = fma(-0.5 * pRb, b[NI], uRb);
  if (C == 4) {
    ab[TI] = fma(-0.5 * pLb, s.utL, ab[TI]);
    bb[TI] = fma(-0.5 * pRb, s.utR, bb[TI]);
    wLb = fma(-0.5 * pLb, a[TI], wLb);
    wRb = fma(-0.5 * pRb, b[TI], wRb);
    ab[TI] = fma(wLb, s.irL, ab[TI]);
    bb[TI] = fma(wRb, s.irR, bb[TI]);
    irLb = fma(wLb, a[TI], irLb);
    irRb = fma(wRb, b[TI], irRb);
  }
  // u = m_n / rho, 1/rho
  ab[NI] = fma(uLb, s.irL, ab[NI]);
  bb[NI] = fma(uRb, s.irR, bb[NI]);
  irLb = fma(uLb, a[NI], irLb);
  irRb = fma(uRb, b[NI], irRb);
  ab[0] = fma(-irLb * s.irL, s.irL, ab[0]);
  bb[0] = fma(-irRb * s.irR, s.irR, bb[0]);
}

// ---------------------------------------------------------------------------------
// boundary preimages
// ---------------------------------------------------------------------------------
// Cells x in [xlo, xhi] that the ghost map (periodic wrap / clamp) sends to cell i.
__device__ __forceinline__ int cell_preimages(int i, int n, int bl, int bh, int xlo, int xhi, int* xs) {
  constexpr int cap = 16;
  int cnt = 0;
  if (i >= xlo && i <= xhi) xs[cnt++] = i;
  if (bl == BC_PERIODIC) {
    for (int x = i - n; x >= xlo && cnt < cap; x -= n) xs[cnt++] = x;
  } else if (i == 0) {
    for (int x = -1; x >= xlo && cnt < cap; --x) xs[cnt++] = x;
  }
  if (bh == BC_PERIODIC) {
    for (int x = i + n; x <= xhi && cnt < cap; x += n) xs[cnt++] = x;
  } else if (i == n - 1) {
    for (int x = n; x <= xhi && cnt < cap; ++x) xs[cnt++] = x;
  }
  return cnt;
}

// Faces f in [flo, fhi] that face_map sends to face e (0 <= e <= n).
__device__ __forceinline__ int face_preimages(int e, int n, int bl, int bh, int flo, int fhi, int* fs) {
  constexpr int cap = 16;
  int cnt = 0;
  if (e >= flo && e <= fhi) fs[cnt++] = e;
  if (bl == BC_PERIODIC) {
    if (e < n)
      for (int f = e - n; f >= flo && cnt < cap; f -= n) fs[cnt++] = f;
  } else if (e == 0) {
    for (int f = -1; f >= flo && cnt < cap; --f) fs[cnt++] = f;
  }
  if (bh == BC_PERIODIC) {
    if (e < n)
      for (int f = e + n; f <= fhi && cnt < cap; f += n)
        if (f > n) fs[cnt++] = f;
  } else if (e == n) {
    for (int f = n + 1; f <= fhi && cnt < cap; ++f) fs[cnt++] = f;
  }
  return cnt;
}

// ---------------------------------------------------------------------------------
// K1: face kernel
// ---------------------------------------------------------------------------------
// 2D: 8 faces x 16 lines per CTA of 128 threads, one face per thread; four CTAs per SM up to
// order 7 (128 registers, a few hundred bytes of spills: measured 9 % faster than three CTAs
// at 168 registers), three at order 9 (its 64 KB of shared memory per CTA allows no more);
// 1D: 256 faces per CTA of 256 threads.  Phase A (per face) recomputes the two states at
// each Gauss point and writes their adjoints to shared memory; phase B (per face and side)
// takes them back through the tangential reconstruction.
template <int R, int DIM>
struct AdjShape {
  static constexpr int TN = (DIM == 2) ? 8 : 256;
  static constexpr int TT = (DIM == 2) ? 16 : 1;
  static constexpr int NT = TN * TT;
  static constexpr int MINB = (DIM == 2) ? (R <= 7 ? 4 : 3) : 1;
};

template <int R, int DIM>
using AdjTile = Tile<R, DIM, AdjShape<R, DIM>::TT, AdjShape<R, DIM>::TN>;

template <int R, int DIM>
constexpr size_t adj_smem_doubles() {
  using TL = AdjTile<R, DIM>;
  return TL::smem_doubles + (size_t)AdjShape<R, DIM>::NT * 2 * TL::G * TL::C;
}

template <int R, int DIM, int DIR>
__global__ void __launch_bounds__(AdjShape<R, DIM>::NT, AdjShape<R, DIM>::MINB)
adj_face_kernel(const GridInfo g, const SweepArgs args, const AdjArgs aa, const __grid_constant__ Tables T) {
  using TL = AdjTile<R, DIM>;
  constexpr int K = TL::K, C = TL::C, KT = TL::KT, G = TL::G;
  constexpr int TN = TL::TN, TT = TL::TT, NT = AdjShape<R, DIM>::NT;
  constexpr int NA = TL::NA, NB = TL::NB, NQ = TL::NQ, NSN = TL::NSN, NST = TL::NST;
  constexpr int NI = (DIR == 0) ? 1 : 2;
  constexpr int TI = (DIR == 0) ? 2 : 1;
  constexpr int NTAP = 2 * KT + 1;

  extern __shared__ double smem[];
  double* sW = smem;
  double* sQP = sW + C * NB * NA;
  double* sQM = sQP + C * NB * NQ;
  double* sSn = sQM + C * NB * NQ;
  double* sSt = sSn + NB * NSN;
  // adjoints of the Gauss-point states, [side][G][C][face of the tile] (conflict-free: the
  // threads of a warp take consecutive faces)
  double* sStb = smem + TL::smem_doubles;

  const int n = (DIR == 0) ? g.nx : g.ny;
  const int mlin = (DIR == 0) ? g.ny : g.nx;
  const int a0 = blockIdx.x * TN, b0 = blockIdx.y * TT;
  const int tid = threadIdx.x;
  const int bcn_lo = (DIR == 0) ? g.bc[0] : g.bc[2], bcn_hi = (DIR == 0) ? g.bc[1] : g.bc[3];
  const int bct_lo = (DIR == 0) ? g.bc[2] : g.bc[0], bct_hi = (DIR == 0) ? g.bc[3] : g.bc[1];

  // ---- stage the tile as the forward sweep does ----
  for (int idx = tid; idx < C * NB * NA; idx += NT) {
    int c, bb, ai;
    if (DIR == 0) { ai = idx % NA; bb = (idx / NA) % NB; c = idx / (NA * NB); }
    else { bb = idx % NB; ai = (idx / NB) % NA; c = idx / (NA * NB); }
    const int a = a0 - 1 - K + ai, b = b0 - KT + bb;
    const int i = (DIR == 0) ? a : b, j = (DIR == 0) ? b : a;
    sW[(c * NB + bb) * NA + ai] = fetch_w(g, args.W, c, i, j, 0.0);
  }
  // sigma staging: consecutive threads take consecutive entries of the global arrays
  for (int idx = tid; idx < NB * NSN; idx += NT) {
    int fa, bb;
    if (DIR == 0) { fa = idx % NSN; bb = idx / NSN; }
    else { bb = idx % NB; fa = idx / NB; }
    const int f = face_map(a0 - K + fa, n, bcn_lo, bcn_hi);
    const int b = wrap_or_clamp(b0 - KT + bb, mlin, bct_lo, bct_hi);
    sSn[bb * NSN + fa] = (DIR == 0) ? args.s_norm[(size_t)b * (g.nx + 1) + f] : args.s_norm[(size_t)f * g.nx + b];
  }
  if (DIM == 2) {
    for (int idx = tid; idx < NQ * (NST - 1); idx += NT) {
      int qa, fb;
      if (DIR == 0) { qa = idx % NQ; fb = idx / NQ; }
      else { fb = idx % (NST - 1); qa = idx / (NST - 1); }
      const int a = wrap_or_clamp(a0 - 1 + qa, n, bcn_lo, bcn_hi);
      const int f = face_map(b0 - K + 1 + fb, mlin, bct_lo, bct_hi);
      sSt[qa * NST + fb] = (DIR == 0) ? args.s_tan[(size_t)f * g.nx + a] : args.s_tan[(size_t)a * (g.nx + 1) + f];
    }
  }
  __syncthreads();
  for (int it = tid; it < NQ * NB; it += NT) {
    const int qa = it % NQ, bb = it / NQ;
    const Branch br = select_branch<R>(sSn + bb * NSN + qa, g.thres);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const double* v = sW + (c * NB + bb) * NA + qa + K;
      double out[2];
      recon_eval<R, 2>(v, 1, br, T, 0, out);
      sQP[(c * NB + bb) * NQ + qa] = out[0];
      sQM[(c * NB + bb) * NQ + qa] = out[1];
    }
  }
  __syncthreads();

  const size_t nfaces = (size_t)(n + 1) * mlin;
  const double fscale = aa.lscale * aa.inv_h;
  auto face_of = [&](int it, int& fa, int& tb) {
    if (DIR == 0) { fa = it % TN; tb = it / TN; }
    else { tb = it % TT; fa = it / TT; }
  };

  // ---- phase A (per face): the Gauss-point flux VJPs ----
  {
    const int it = tid;  // NT = TN * TT: one face per thread
    int fa, tb;
    face_of(it, fa, tb);
    const int f = a0 + fa, b = b0 + tb;
    if (f <= n && b < mlin) {
      const size_t face = adj_face<DIR>(f, b, n, mlin);
      // F_f enters L of cell f with +1/h and L of cell f-1 with -1/h
      double Fb[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        double lb = 0.0;
        if (aa.Lbar) {
          if (f < n)
            lb += (DIR == 0) ? aa.Lbar[((size_t)c * g.ny + b) * g.nx + f] : aa.Lbar[((size_t)c * g.ny + f) * g.nx + b];
          if (f >= 1)
            lb -= (DIR == 0) ? aa.Lbar[((size_t)c * g.ny + b) * g.nx + f - 1]
                             : aa.Lbar[((size_t)c * g.ny + f - 1) * g.nx + b];
        }
        Fb[c] = lb * fscale;
      }
      double sbar = 0.0;
      if (aa.sbar_out)
        sbar = ((DIR == 0) ? aa.sbar_out[(size_t)b * (g.nx + 1) + f] : aa.sbar_out[(size_t)f * g.nx + b]) * (1.0 / G);
      // adjoints of the two cell averages (first-order points), accumulated in place
#pragma unroll
      for (int c = 0; c < 2 * C; ++c) aa.Cbar[(size_t)c * nfaces + face] = 0.0;
#pragma unroll 1
      for (int q = 0; q < G; ++q) {
        double st[2][C];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int qa = fa + side;
          const double* Q = side == 0 ? sQP : sQM;
          if (DIM == 2) {
            const Branch bt = select_branch<R>(sSt + qa * NST + tb, g.thres);
#pragma unroll
            for (int c = 0; c < C; ++c) {
              double out[1];
              recon_eval<R, 1>(Q + (c * NB + tb + K) * NQ + qa, NQ, bt, T, 2 + q, out);
              st[side][c] = out[0];
            }
          } else {
#pragma unroll
            for (int c = 0; c < C; ++c) st[side][c] = Q[c * NQ + qa];
          }
        }
        double F2b[C];
        const double hw = T.hgw[q];
#pragma unroll
        for (int c = 0; c < C; ++c) F2b[c] = hw * Fb[c];
        const LfPrims pr = lf_primitives<C, NI, TI>(st[0], st[1]);
        double* out0 = sStb + (size_t)(q * C) * NT + it;        // side 0, point q, component 0
        double* out1 = sStb + (size_t)((G + q) * C) * NT + it;  // side 1
        double ab[C], bb[C];
        if (lf_physical(st[0][0], st[1][0], pr)) {
          lf_point_vjp<C, NI, TI>(st[0], st[1], pr, g.gm1, g.gg1, F2b, sbar, true, ab, bb);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            out0[c * NT] = ab[c];
            out1[c * NT] = bb[c];
          }
        } else {
          // the point took the cell averages either side of the face
          double ca[C], cb[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            ca[c] = sW[(c * NB + tb + KT) * NA + fa + K];
            cb[c] = sW[(c * NB + tb + KT) * NA + fa + K + 1];
            out0[c * NT] = out1[c * NT] = 0.0;
          }
          lf_point_vjp<C, NI, TI>(ca, cb, lf_primitives<C, NI, TI>(ca, cb), g.gm1, g.gg1, F2b, sbar, false, ab,
                                  bb);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            aa.Cbar[(size_t)c * nfaces + face] += ab[c];
            aa.Cbar[(size_t)(C + c) * nfaces + face] += bb[c];
          }
        }
      }
    }
  }
  __syncthreads();

  // ---- phase B (per face and side): the tangential reconstruction VJP ----
  for (int item = tid; item < 2 * NT; item += NT) {
    const int side = item / NT, it = item - side * NT;  // a warp: consecutive faces of one side
    int fa, tb;
    face_of(it, fa, tb);
    const int f = a0 + fa, b = b0 + tb;
    if (f > n || b >= mlin) continue;
    const size_t face = adj_face<DIR>(f, b, n, mlin);
    const int qa = fa + side;
    const double* Q = side == 0 ? sQP : sQM;
    const double* pin = sStb + (size_t)(side * G * C) * NT + it;  // [G][C] at stride NT
    Branch bt;
    if (DIM == 2) bt = select_branch<R>(sSt + qa * NST + tb, g.thres);
    double ab[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < C; ++c) {
      double vb[NTAP];
#pragma unroll
      for (int t = 0; t < NTAP; ++t) vb[t] = 0.0;
      if (DIM == 2) {
        double pb[G];
#pragma unroll
        for (int q = 0; q < G; ++q) pb[q] = pin[(size_t)(q * C + c) * NT];
        recon_vjp<R, G>(Q + (c * NB + tb + K) * NQ + qa, NQ, bt, T, 2, pb, vb + KT, ab);
      } else {
        vb[0] = pin[(size_t)c * NT];
      }
#pragma unroll
      for (int t = 0; t < NTAP; ++t) aa.Tbar[((size_t)((side * NTAP + t) * C + c)) * nfaces + face] = vb[t];
    }
    if (DIM == 2) {
      double sb[4];
      sigma_vjp<R>(bt, ab, g.thres, sb);
#pragma unroll
      for (int q = 0; q < 4; ++q) aa.Stb[(size_t)(side * 4 + q) * nfaces + face] = sb[q];
    }
  }
}

// ---------------------------------------------------------------------------------
// K2: normal VJP per reconstructing cell (a in [-1, n], line l in [-KT, m+KT))
// ---------------------------------------------------------------------------------
// 128 threads and three CTAs per SM: the WENO branch's VJP needs ~170 registers.
template <int R, int DIM, int DIR>
__global__ void __launch_bounds__(128, 3) adj_normal_kernel(const GridInfo g, const SweepArgs args, const AdjArgs aa,
                                                         const __grid_constant__ Tables T) {
  constexpr int K = (R - 1) / 2, C = (DIM == 1) ? 3 : 4, KT = (DIM == 2) ? K : 0;
  constexpr int NTAP = 2 * KT + 1, NS = 2 * K + 1;
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int mlin = (DIR == 0) ? g.ny : g.nx;
  const int bcn_lo = (DIR == 0) ? g.bc[0] : g.bc[2], bcn_hi = (DIR == 0) ? g.bc[1] : g.bc[3];
  const int bct_lo = (DIR == 0) ? g.bc[2] : g.bc[0], bct_hi = (DIR == 0) ? g.bc[3] : g.bc[1];
  const size_t nfaces = (size_t)(n + 1) * mlin;
  const int na = n + 2, nl = mlin + 2 * KT;
  const size_t nitems = (size_t)na * nl;
  // one thread per (component, reconstructing cell); consecutive threads take consecutive
  // items of one component (the item index is adj_item<DIR>(a, l))
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < C * nitems;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / nitems);
    const size_t it = idx - (size_t)c * nitems;
    const int a = (DIR == 0) ? (int)(it % na) - 1 : (int)(it / nl) - 1;
    const int l = (DIR == 0) ? (int)(it / na) - KT : (int)(it % nl) - KT;
    // adjoints of the plus (xi = 0) and minus (xi = -1) values of cell (a, l): the
    // plus value is the left state of face a+1, the minus value the right state of face
    // a, each read by the tangential stencils of the face lines b = l - t
    double QPb = 0.0, QMb = 0.0;
    bool any = false;
#pragma unroll
    for (int t = -KT; t <= KT; ++t) {
      const int b = l - t;
      if (b < 0 || b >= mlin) continue;
      if (a + 1 <= n) {
        QPb += aa.Tbar[((size_t)((0 * NTAP + t + KT) * C + c)) * nfaces + adj_face<DIR>(a + 1, b, n, mlin)];
        any = true;
      }
      if (a >= 0) {
        QMb += aa.Tbar[((size_t)((1 * NTAP + t + KT) * C + c)) * nfaces + adj_face<DIR>(a, b, n, mlin)];
        any = true;
      }
    }
    double* out = aa.Nbar + (size_t)c * nitems + it;  // [m][c][item]
    double* sout = aa.Snb + (size_t)c * nitems + it;  // [q][c][item]: this component's share
    if (!any) {
#pragma unroll
      for (int m = 0; m < NS; ++m) out[(size_t)m * C * nitems] = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) sout[(size_t)q * C * nitems] = 0.0;
      continue;
    }
    // branch of cell (a, l) from the normal faces of its (mapped) line
    double s[2 * K];
    const int lm = wrap_or_clamp(l, mlin, bct_lo, bct_hi);
#pragma unroll
    for (int q = 0; q < 2 * K; ++q) {
      const int f = face_map(a - K + 1 + q, n, bcn_lo, bcn_hi);
      s[q] = (DIR == 0) ? args.s_norm[(size_t)lm * (g.nx + 1) + f] : args.s_norm[(size_t)f * g.nx + lm];
    }
    const Branch br = select_branch<R>(s, g.thres);
    double ab[4] = {0.0, 0.0, 0.0, 0.0};
    double v[NS], vb[NS];
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      const int x = a - K + m;
      v[m] = (DIR == 0) ? fetch_w(g, args.W, c, x, l, 0.0) : fetch_w(g, args.W, c, l, x, 0.0);
      vb[m] = 0.0;
    }
    const double pb[2] = {QPb, QMb};
    recon_vjp<R, 2>(v + K, 1, br, T, 0, pb, vb + K, ab);
#pragma unroll
    for (int m = 0; m < NS; ++m) out[(size_t)m * C * nitems] = vb[m];
    // the sigma_in adjoints are linear in ab: each component writes its share, the gather sums
    double sb[4];
    sigma_vjp<R>(br, ab, g.thres, sb);
#pragma unroll
    for (int q = 0; q < 4; ++q) sout[(size_t)q * C * nitems] = sb[q];
  }
}

// ---------------------------------------------------------------------------------
// K3: gather into Wbar (per interior cell)
// ---------------------------------------------------------------------------------
// This direction's adjoint of W component c of one interior cell: the Nbar and Cbar
// entries of every stencil position that the boundary maps onto it (a fixed order).
template <int R, int DIM, int DIR>
__device__ __forceinline__ double gather_w_sum(const GridInfo& g, const AdjArgs& aa, int c, size_t cell) {
  constexpr int K = (R - 1) / 2, C = (DIM == 1) ? 3 : 4, KT = (DIM == 2) ? K : 0;
  constexpr int NS = 2 * K + 1;
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int mlin = (DIR == 0) ? g.ny : g.nx;
  const int bcn_lo = (DIR == 0) ? g.bc[0] : g.bc[2], bcn_hi = (DIR == 0) ? g.bc[1] : g.bc[3];
  const int bct_lo = (DIR == 0) ? g.bc[2] : g.bc[0], bct_hi = (DIR == 0) ? g.bc[3] : g.bc[1];
  const size_t nfaces = (size_t)(n + 1) * mlin;
  const size_t nitems = (size_t)(n + 2) * (mlin + 2 * KT);
  const int ci = (int)(cell % g.nx), cj = (int)(cell / g.nx);
  const int i = (DIR == 0) ? ci : cj;  // along the sweep
  const int j = (DIR == 0) ? cj : ci;  // line
  int xs[16], ls[16];
  const int nxs = cell_preimages(i, n, bcn_lo, bcn_hi, -K - 1, n + K, xs);
  int nls = 1;
  ls[0] = j;
  if (DIM == 2) nls = cell_preimages(j, mlin, bct_lo, bct_hi, -KT, mlin + KT - 1, ls);
  double acc = 0.0;
  for (int il = 0; il < nls; ++il) {
    const int l = ls[il];
    for (int ix = 0; ix < nxs; ++ix) {
      const int x = xs[ix];
      // inflow ghost cells hold the constant inflow state
      const int gi = (DIR == 0) ? x : l, gj = (DIR == 0) ? l : x;
      if (gi < 0 && g.bc[0] == BC_INFLOW_BAND && gj >= g.band_j0 && gj <= g.band_j1) continue;
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        const int a = x - (m - K);
        if (a < -1 || a > n) continue;
        acc += aa.Nbar[((size_t)(m * C + c)) * nitems + adj_item<DIR>(a, l, n, mlin, KT)];
      }
      // first-order states: face x+1 has this cell on its left, face x on its right
      if (l >= 0 && l < mlin) {
        if (x + 1 >= 0 && x + 1 <= n) acc += aa.Cbar[(size_t)c * nfaces + adj_face<DIR>(x + 1, l, n, mlin)];
        if (x >= 0 && x <= n) acc += aa.Cbar[(size_t)(C + c) * nfaces + adj_face<DIR>(x, l, n, mlin)];
      }
    }
  }
  return acc;
}

template <int R, int DIM, int DIR>
__global__ void __launch_bounds__(256) adj_gather_w_kernel(const GridInfo g, const AdjArgs aa) {
  constexpr int C = (DIM == 1) ? 3 : 4;
  const size_t ncell = (size_t)g.nx * g.ny;
  // one thread per (component, cell): consecutive threads take consecutive cells
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < C * ncell;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / ncell);
    aa.Wbar[idx] += gather_w_sum<R, DIM, DIR>(g, aa, c, idx - (size_t)c * ncell);
  }
}

// ---------------------------------------------------------------------------------
// K4: gather of the normal-face sigma_in adjoints (per entry of this direction's
// normal sigma array)
// ---------------------------------------------------------------------------------
// Entry idx of the normal sigma array: sx[j][e] (x-sweep) or sy[e][j] (y-sweep), row-major.
template <int R, int DIM, int DIR>
__device__ __forceinline__ double gather_sn_sum(const GridInfo& g, const AdjArgs& aa, size_t idx) {
  constexpr int K = (R - 1) / 2, KT = (DIM == 2) ? K : 0, C = (DIM == 1) ? 3 : 4;
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int mlin = (DIR == 0) ? g.ny : g.nx;
  const int bcn_lo = (DIR == 0) ? g.bc[0] : g.bc[2], bcn_hi = (DIR == 0) ? g.bc[1] : g.bc[3];
  const int bct_lo = (DIR == 0) ? g.bc[2] : g.bc[0], bct_hi = (DIR == 0) ? g.bc[3] : g.bc[1];
  const size_t nitems = (size_t)(n + 2) * (mlin + 2 * KT);
  int e, j;
  if (DIR == 0) { e = (int)(idx % (g.nx + 1)); j = (int)(idx / (g.nx + 1)); }  // sx[j][e]
  else { j = (int)(idx % g.nx); e = (int)(idx / g.nx); }                       // sy[e][j]
  int fs[16], ls[16];
  const int nfs = face_preimages(e, n, bcn_lo, bcn_hi, -2, n + 2, fs);
  int nls = 1;
  ls[0] = j;
  if (DIM == 2) nls = cell_preimages(j, mlin, bct_lo, bct_hi, -KT, mlin + KT - 1, ls);
  double acc = 0.0;
#pragma unroll 1
  for (int il = 0; il < nls; ++il) {
#pragma unroll 1
    for (int k = 0; k < nfs; ++k) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = fs[k] + 1 - q;  // the cell whose stencil face q (face a-1+q) is f
        if (a < -1 || a > n) continue;
        const size_t item = adj_item<DIR>(a, ls[il], n, mlin, KT);
#pragma unroll
        for (int c = 0; c < C; ++c) acc += aa.Snb[(size_t)(q * C + c) * nitems + item];
      }
    }
  }
  return acc;
}

template <int R, int DIM, int DIR>
__global__ void __launch_bounds__(256) adj_gather_sn_kernel(const GridInfo g, const AdjArgs aa) {
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int mlin = (DIR == 0) ? g.ny : g.nx;
  const size_t nent = (size_t)(n + 1) * mlin;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nent;
       idx += (size_t)gridDim.x * blockDim.x)
    aa.sbar_norm[idx] += gather_sn_sum<R, DIM, DIR>(g, aa, idx);
}

// ---------------------------------------------------------------------------------
// K5: gather of the tangential-face sigma_in adjoints (2D)
// ---------------------------------------------------------------------------------
// Entry idx of the tangential sigma array: sy[te][i] (x-sweep) or sx[i][te] (y-sweep).
template <int R, int DIR>
__device__ __forceinline__ double gather_st_sum(const GridInfo& g, const AdjArgs& aa, size_t idx) {
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int mlin = (DIR == 0) ? g.ny : g.nx;
  const int bcn_lo = (DIR == 0) ? g.bc[0] : g.bc[2], bcn_hi = (DIR == 0) ? g.bc[1] : g.bc[3];
  const int bct_lo = (DIR == 0) ? g.bc[2] : g.bc[0], bct_hi = (DIR == 0) ? g.bc[3] : g.bc[1];
  const size_t nfaces = (size_t)(n + 1) * mlin;
  int te, i;
  if (DIR == 0) { i = (int)(idx % g.nx); te = (int)(idx / g.nx); }            // sy[te][i]
  else { te = (int)(idx % (g.nx + 1)); i = (int)(idx / (g.nx + 1)); }         // sx[i][te]
  int xs[16], tfs[16];
  const int nxs = cell_preimages(i, n, bcn_lo, bcn_hi, -1, n, xs);
  const int ntf = face_preimages(te, mlin, bct_lo, bct_hi, -1, mlin + 1, tfs);
  double acc = 0.0;
  for (int side = 0; side < 2; ++side) {
    for (int ix = 0; ix < nxs; ++ix) {
      const int f = xs[ix] + 1 - side;  // the face whose side-`side` column is x
      if (f < 0 || f > n) continue;
      for (int k = 0; k < ntf; ++k) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int b = tfs[k] + 1 - q;
          if (b < 0 || b >= mlin) continue;
          acc += aa.Stb[(size_t)(side * 4 + q) * nfaces + adj_face<DIR>(f, b, n, mlin)];
        }
      }
    }
  }
  return acc;
}

template <int R, int DIR>
__global__ void __launch_bounds__(256) adj_gather_st_kernel(const GridInfo g, const AdjArgs aa) {
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int mlin = (DIR == 0) ? g.ny : g.nx;
  const size_t nent = (size_t)(mlin + 1) * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nent;
       idx += (size_t)gridDim.x * blockDim.x)
    aa.sbar_tan[idx] += gather_st_sum<R, DIR>(g, aa, idx);
}

// ---------------------------------------------------------------------------------
// K3-K5 of both directions in one launch (2D)
// ---------------------------------------------------------------------------------
// The three outputs are disjoint: Wbar, sigma_x's adjoint (the x-direction's normal faces and
// the y-direction's tangential ones) and sigma_y's.  Each element is one thread's, and it adds
// the x-direction's sum before the y-direction's, the order of the per-direction launches,
// so the results are theirs bit for bit.
template <int R>
__global__ void __launch_bounds__(256) adj_gather_both_kernel(const GridInfo g, const AdjArgs ax, const AdjArgs ay) {
  constexpr int C = 4;
  const size_t ncell = (size_t)g.nx * g.ny;
  const size_t nw = C * ncell;
  const size_t nsx = ax.sbar_norm ? (size_t)(g.nx + 1) * g.ny : 0;
  const size_t nsy = ay.sbar_norm ? (size_t)(g.ny + 1) * g.nx : 0;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nw + nsx + nsy;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (idx < nw) {
      const int c = (int)(idx / ncell);
      const size_t cell = idx - (size_t)c * ncell;
      double w = ax.Wbar[idx];
      w += gather_w_sum<R, 2, 0>(g, ax, c, cell);
      w += gather_w_sum<R, 2, 1>(g, ay, c, cell);
      ax.Wbar[idx] = w;
    } else if (idx < nw + nsx) {
      const size_t k = idx - nw;
      double s = ax.sbar_norm[k];
      s += gather_sn_sum<R, 2, 0>(g, ax, k);
      s += gather_st_sum<R, 1>(g, ay, k);
      ax.sbar_norm[k] = s;
    } else {
      const size_t k = idx - nw - nsx;
      double s = ay.sbar_norm[k];
      s += gather_st_sum<R, 0>(g, ax, k);
      s += gather_sn_sum<R, 2, 1>(g, ay, k);
      ay.sbar_norm[k] = s;
    }
  }
}

inline int grid_for(size_t n, int threads = 256) {
  return (int)std::max<size_t>(1, std::min<size_t>((n + threads - 1) / threads, 152 * 16));
}

// Phase 1 (K1, K2) writes only this direction's scratch; phase 2 (K3 - K5) adds into the
// outputs shared with the other direction.  Phase 1 of the two directions may run
// concurrently when their scratch is separate; phase 2 runs in a fixed order.
template <int R, int DIM, int DIR>
cudaError_t adj_launch(int phase, const GridInfo& g, const SweepArgs& a, const AdjArgs& aa, const Tables& t,
                       cudaStream_t s) {
  using TL = AdjTile<R, DIM>;
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int m = (DIR == 0) ? g.ny : g.nx;
  cudaError_t e = cudaSuccess;
  if (phase & 1) {
    const size_t smem = adj_smem_doubles<R, DIM>() * sizeof(double);
    auto k1 = adj_face_kernel<R, DIM, DIR>;
    static std::atomic<unsigned long long> attr_done{0ull};
    e = ensure_smem_limit(k1, smem, attr_done);
    if (e != cudaSuccess) return e;
    dim3 grid((n + 1 + TL::TN - 1) / TL::TN, (m + TL::TT - 1) / TL::TT);
    k1<<<grid, AdjShape<R, DIM>::NT, smem, s>>>(g, a, aa, t);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t nitems = (size_t)(n + 2) * (m + 2 * TL::KT);
    adj_normal_kernel<R, DIM, DIR><<<grid_for((size_t)TL::C * nitems, 128), 128, 0, s>>>(g, a, aa, t);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (!(phase & 2)) return cudaSuccess;
  adj_gather_w_kernel<R, DIM, DIR><<<grid_for((size_t)TL::C * g.nx * g.ny), 256, 0, s>>>(g, aa);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (aa.sbar_norm) {
    adj_gather_sn_kernel<R, DIM, DIR><<<grid_for((size_t)(n + 1) * m), 256, 0, s>>>(g, aa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (DIM == 2 && aa.sbar_tan) {
    adj_gather_st_kernel<R, DIR><<<grid_for((size_t)(m + 1) * n), 256, 0, s>>>(g, aa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int R>
cudaError_t adj_gather_both_launch(const GridInfo& g, const AdjArgs& ax, const AdjArgs& ay, cudaStream_t s) {
  const size_t n = (size_t)4 * g.nx * g.ny + (ax.sbar_norm ? (size_t)(g.nx + 1) * g.ny : 0) +
                   (ay.sbar_norm ? (size_t)(g.ny + 1) * g.nx : 0);
  adj_gather_both_kernel<R><<<grid_for(n), 256, 0, s>>>(g, ax, ay);
  return cudaGetLastError();
}

}  // namespace

#define ASE_DF_CAT2(a, b) a##b
#define ASE_DF_CAT(a, b) ASE_DF_CAT2(a, b)

cudaError_t ASE_DF_CAT(launch_adjoint_r, ASE_DF_ORDER)(int dim, int dir, int phase, const GridInfo& g,
                                                       const SweepArgs& a, const AdjArgs& aa, const Tables& t,
                                                       cudaStream_t s) {
  constexpr int R = ASE_DF_ORDER;
  if (dim == 1) return adj_launch<R, 1, 0>(phase, g, a, aa, t, s);
  if (dir == 0) return adj_launch<R, 2, 0>(phase, g, a, aa, t, s);
  return adj_launch<R, 2, 1>(phase, g, a, aa, t, s);
}

cudaError_t ASE_DF_CAT(launch_adjoint_gathers_2d_r, ASE_DF_ORDER)(const GridInfo& g, const AdjArgs& ax,
                                                                   const AdjArgs& ay, cudaStream_t s) {
  return adj_gather_both_launch<ASE_DF_ORDER>(g, ax, ay, s);
}

}  // namespace asedf
