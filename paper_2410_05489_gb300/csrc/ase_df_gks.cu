// Gas-kinetic face kernel of the ASE-DF scheme (Sec. 2.2 with Appendix A), one sweep
// direction, sm_103a, FP64.  Compiled once per scheme order (ASE_DF_ORDER).
//
// Per face the tile is staged like the Lax-Friedrichs sweep; phase 1 reconstructs every
// cell of the band at both of its faces, value and normal derivative (Sec. 3 polynomials
// and their derivatives); phase 2 reconstructs, per face side, the G Gauss-point values
// and tangential derivatives from the face line-averages, and the Gauss-point normal
// derivatives from the line-averages of the normal derivative (the same tangential
// procedure applied to them), then evaluates the gas-kinetic flux at each Gauss point:
//   Maxwellians g_l, g_r of the two states and their moments (erfc half-line moments),
//   slopes a from <psi psi^T> a = W_x / rho (closed form of Appendix A), the
//   kinetic-weighted equilibrium state g_c and its slopes, A_c from the compatibility
//   condition, and the time integrals of the distribution function of Eq. (GKS flux)
//   with the physical collision time 0 over [0, dt] and [0, dt/2]:
//     F(d) = c1 T0 + c2 (T1 - T4) + c3 T2 + c4 T3,
//     c1 = d - tn (1 - e), c2 = tn^2 (1 - e) - tn d e, c3 = d^2 / 2, c4 = tn (1 - e),
//     e = exp(-d / tn), tn = C1 dt + C2 |p_l - p_r| / (p_l + p_r) dt (C1, C2 of the problem);
//   T0 = rho_c <u psi>_c, T1 = rho_c <u (a_x^c u + a_y^c v) psi>_c, T2 = rho_c <u A^c psi>_c,
//   T3 = rho_l <u psi>_{l,u>0} + rho_r <u psi>_{r,u<0}, T4 = the same with (a_x u + a_y v).
//   F = (4 F(dt/2) - F(dt)) / dt and F_t = 4 (F(dt) - 2 F(dt/2)) / dt^2 (Sec. 2.2).
// A Gauss point where either side's state is non-physical takes the two cell averages
// with zero derivatives and sigma 1e30, as the Lax-Friedrichs path does.

#include <cuda_runtime.h>

#include "ase_df_gks.cuh"
#include "ase_df_sweep_body.cuh"

#ifndef ASE_DF_ORDER
#error "ASE_DF_ORDER must be defined"
#endif

namespace asedf {
namespace {

// ---------------------------------------------------------------------------------
// value and d/dxi of the chosen polynomial (Algorithm 1) at NP points p0..
// ---------------------------------------------------------------------------------
template <int NP>
__device__ void weno_eval_d(const double* v, int vs, const Branch& br, const Tables& T, const DTables& D, int p0,
                            double* out, double* dout) {
  double beta[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double* vk = v + (k - 2) * vs;
    const double c1 = T.cq[k][0][0] * vk[0] + T.cq[k][0][1] * vk[vs] + T.cq[k][0][2] * vk[2 * vs];
    const double c2 = T.cq[k][1][0] * vk[0] + T.cq[k][1][1] * vk[vs] + T.cq[k][1][2] * vk[2 * vs];
    beta[k] = c1 * (c1 - 2.0 * c2) + (16.0 / 3.0) * c2 * c2;
  }
  const double b5 = (beta[0] + 4.0 * beta[1] + beta[2]) * (1.0 / 6.0) + fabs(beta[0] - beta[2]);
  const double tau = (fabs(b5 - beta[0]) + fabs(b5 - beta[1]) + fabs(b5 - beta[2])) * (1.0 / 3.0);
  const double tau2 = tau * tau;
  const double e5 = b5 + T.eps;
  const double w5 = T.d5 * (1.0 + tau2 / (e5 * e5));
  double w3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double e = beta[k] + T.eps;
    w3[k] = T.d3[k] * (1.0 + tau2 / (e * e));
  }
  const double inv = 1.0 / (w5 + w3[0] + w3[1] + w3[2]);
  const double g5 = (w5 * inv) / T.d5;
  double g3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) g3[k] = w3[k] * inv - g5 * T.d3[k];
  const double W0 = v[0];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int p = p0 + q;
    double P = g5 * fma(br.a5, lin_eval<5>(v, vs, T.lin[1][p]) - W0, W0);
    double dP = g5 * br.a5 * lin_eval<5>(v, vs, D.dlin[1][p]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double* vk = v + (k - 2) * vs;
      const double u = T.sub[k][p][0] * vk[0] + T.sub[k][p][1] * vk[vs] + T.sub[k][p][2] * vk[2 * vs];
      const double du = D.dsub[k][p][0] * vk[0] + D.dsub[k][p][1] * vk[vs] + D.dsub[k][p][2] * vk[2 * vs];
      P = fma(g3[k], fma(br.a3[k], u - W0, W0), P);
      dP = fma(g3[k] * br.a3[k], du, dP);
    }
    out[q] = P;
    dout[q] = dP;
  }
}

template <int R, int NP>
__device__ __forceinline__ void recon_eval_d(const double* v, int vs, const Branch& br, const Tables& T,
                                             const DTables& D, int p0, double* out, double* dout) {
  if (br.m == R) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      out[q] = lin_eval<R>(v, vs, T.lin[(R - 3) / 2][p0 + q]);
      dout[q] = lin_eval<R>(v, vs, D.dlin[(R - 3) / 2][p0 + q]);
    }
    return;
  }
  if (R == 3) {  // DF-damped order 3: W0 + a (lin3 - W0)
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      out[q] = fma(br.a5, lin_eval<3>(v, vs, T.lin[0][p0 + q]) - v[0], v[0]);
      dout[q] = br.a5 * lin_eval<3>(v, vs, D.dlin[0][p0 + q]);
    }
    return;
  }
  if (R >= 9 && br.m == 7) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      out[q] = lin_eval<(R >= 7 ? 7 : 3)>(v, vs, T.lin[2][p0 + q]);
      dout[q] = lin_eval<(R >= 7 ? 7 : 3)>(v, vs, D.dlin[2][p0 + q]);
    }
    return;
  }
  if (R >= 7 && br.m == 5) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      out[q] = lin_eval<5>(v, vs, T.lin[1][p0 + q]);
      dout[q] = lin_eval<5>(v, vs, D.dlin[1][p0 + q]);
    }
    return;
  }
  if (R >= 5) weno_eval_d<NP>(v, vs, br, T, D, p0, out, dout);
}

// ---------------------------------------------------------------------------------
// Maxwellian moments (Appendix A)
// ---------------------------------------------------------------------------------
// FP64 division and square root take 6-9 FMA issue slots on this part, so the moments
// work from the reciprocal density and h = p / rho = 1 / (2 lambda), each one seeded
// reciprocal (rcp_pos), and every later division becomes a multiplication.
struct Maxw {
  double rho, ir, U, V, lam, h;  // ir = 1 / rho, h = 1 / (2 lambda)
  double mu[7], mv[6], mx[3];    // <u^n> (n <= 6), <v^n> (n <= 5), <xi^0>, <xi^2>, <xi^4>
  double dx4;                    // <xi^4> - <xi^2>^2 = 2 K h^2
};

template <int DIM>
__device__ __forceinline__ void maxw_init(const double* W, double gamma, double K, Maxw& m) {
  m.rho = W[0];
  const double ir = rcp_pos(W[0]);
  m.ir = ir;
  m.U = W[1] * ir;
  m.V = (DIM == 2) ? W[2] * ir : 0.0;
  const double p = (gamma - 1.0) * (W[DIM + 1] - 0.5 * m.rho * (m.U * m.U + m.V * m.V));
  const double h = p * ir;  // 1 / (2 lambda)
  m.h = h;
  m.lam = 0.5 * rcp_pos(h);
  m.mu[0] = 1.0;
  m.mu[1] = m.U;
#pragma unroll
  for (int n = 0; n < 5; ++n) m.mu[n + 2] = fma(m.U, m.mu[n + 1], (n + 1) * h * m.mu[n]);
  m.mv[0] = 1.0;
  m.mv[1] = m.V;
#pragma unroll
  for (int n = 0; n < 4; ++n) m.mv[n + 2] = (DIM == 2) ? fma(m.V, m.mv[n + 1], (n + 1) * h * m.mv[n]) : 0.0;
  m.mx[0] = 1.0;
  m.mx[1] = K * h;
  m.mx[2] = (K + 2.0) * h * m.mx[1];
  m.dx4 = 2.0 * K * h * h;
}

// <u^n> over u > 0 (pos) or u < 0, n <= 6
__device__ __forceinline__ void half_moments(const Maxw& m, bool pos, double* mh) {
  const double isl = rsqrt_pos(m.lam);  // 1 / sqrt(lambda)
  const double sl = m.lam * isl;
  // exp(-lambda U^2) / (2 sqrt(pi lambda)), 1 / (2 sqrt(pi)) = 0.28209479177387814
  const double e = 0.28209479177387814 * exp(-m.lam * m.U * m.U) * isl;
  mh[0] = 0.5 * erfc(pos ? -sl * m.U : sl * m.U);
  mh[1] = fma(m.U, mh[0], pos ? e : -e);
  const double h = m.h;
#pragma unroll
  for (int n = 0; n < 5; ++n) mh[n + 2] = fma(m.U, mh[n + 1], (n + 1) * h * mh[n]);
}

// <u^s v^t psi_i> and <u^s v^t psi_i psi_j> with psi = (1, u, v, (u^2+v^2+xi^2)/2) in 2D,
// (1, u, (u^2+xi^2)/2) in 1D; mu are the u moments (full or half line).
template <int DIM>
__device__ __forceinline__ double mom1(int i, int s, int t, const double* mu, const Maxw& m) {
  auto M = [&](int a, int b, int l) { return mu[a] * m.mv[b] * m.mx[l]; };
  if (DIM == 2) {
    if (i == 0) return M(s, t, 0);
    if (i == 1) return M(s + 1, t, 0);
    if (i == 2) return M(s, t + 1, 0);
    return 0.5 * (M(s + 2, t, 0) + M(s, t + 2, 0) + M(s, t, 1));
  }
  if (i == 0) return M(s, 0, 0);
  if (i == 1) return M(s + 1, 0, 0);
  return 0.5 * (M(s + 2, 0, 0) + M(s, 0, 1));
}

// out_i = rho sum_j a_j <u^s v^t psi_j psi_i> = rho <u^s v^t psi_i P> with the polynomial
// P = psi . a = a0 + a1 u + a2 v + (a3 / 2)(u^2 + v^2 + xi^2) (2D; 1D without v).  The
// u, v and xi moments factor, so with a0' = a0 + (a3 / 2) <xi^2>,
//   A(n) = a0' <u^n> + a1 <u^(n+1)> + (a3 / 2) <u^(n+2)>,  B(n) = a2 <v^(n+1)> + (a3 / 2) <v^(n+2)>,
//   Phi(i, j) = <u^(s+i) v^(t+j) P> = <v^(t+j)> A(s+i) + <u^(s+i)> B(t+j),
//   <u^s v^t xi^2 P> = <xi^2> Phi(0, 0) + (a3 / 2) (<xi^4> - <xi^2>^2) <u^s> <v^t>,
// and out = rho (Phi(0,0), Phi(1,0), Phi(0,1), (Phi(2,0) + Phi(0,2) + <u^s v^t xi^2 P>) / 2).
template <int DIM>
__device__ __forceinline__ void slope_moments(const double* a, int s, int t, const double* mu, const Maxw& m,
                                              double* out) {
  if (DIM == 2) {
    const double a3h = 0.5 * a[3];
    const double a0p = fma(a3h, m.mx[1], a[0]);
    double A[3], B[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      A[k] = fma(a3h, mu[s + k + 2], fma(a[1], mu[s + k + 1], a0p * mu[s + k]));
      B[k] = fma(a3h, m.mv[t + k + 2], a[2] * m.mv[t + k + 1]);
    }
    const double P00 = fma(m.mv[t], A[0], mu[s] * B[0]);
    const double P10 = fma(m.mv[t], A[1], mu[s + 1] * B[0]);
    const double P01 = fma(m.mv[t + 1], A[0], mu[s] * B[1]);
    const double P20 = fma(m.mv[t], A[2], mu[s + 2] * B[0]);
    const double P02 = fma(m.mv[t + 2], A[0], mu[s] * B[2]);
    const double Px = fma(m.mx[1], P00, a3h * m.dx4 * (mu[s] * m.mv[t]));
    out[0] = m.rho * P00;
    out[1] = m.rho * P10;
    out[2] = m.rho * P01;
    out[3] = 0.5 * m.rho * (P20 + P02 + Px);
  } else {
    const double a2h = 0.5 * a[2];
    const double a0p = fma(a2h, m.mx[1], a[0]);
    double A[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) A[k] = fma(a2h, mu[s + k + 2], fma(a[1], mu[s + k + 1], a0p * mu[s + k]));
    const double Px = fma(m.mx[1], A[0], a2h * m.dx4 * mu[s]);
    out[0] = m.rho * A[0];
    out[1] = m.rho * A[1];
    out[2] = 0.5 * m.rho * (A[2] + Px);
  }
}

// a with <psi psi^T> a = b (Appendix A closed form; b = W_x / rho).  D = K + DIM, i4D = 4 / D.
template <int DIM>
__device__ __forceinline__ void solve_slope(const Maxw& m, double D, double i4D, const double* b, double* a) {
  const double l = m.lam, U = m.U, V = m.V;
  if (DIM == 2) {
    const double q = U * U + V * V + D * m.h;
    const double R4 = 2.0 * b[3] - q * b[0], R3 = b[2] - V * b[0], R2 = b[1] - U * b[0];
    a[3] = i4D * l * l * (R4 - 2.0 * U * R2 - 2.0 * V * R3);
    a[2] = 2.0 * l * R3 - V * a[3];
    a[1] = 2.0 * l * R2 - U * a[3];
    a[0] = b[0] - U * a[1] - V * a[2] - 0.5 * a[3] * q;
  } else {
    const double q = U * U + D * m.h;
    const double R3 = 2.0 * b[2] - q * b[0], R2 = b[1] - U * b[0];
    a[2] = i4D * l * l * (R3 - 2.0 * U * R2);
    a[1] = 2.0 * l * R2 - U * a[2];
    a[0] = b[0] - U * a[1] - 0.5 * a[2] * q;
  }
}

template <int DIM>
__device__ void gks_point(const double* Wl, const double* Wlx, const double* Wly, const double* Wr,
                          const double* Wrx, const double* Wry, double gamma, double K, double i4D,
                          double dt, double idt, double C1, double C2, double* F, double* Ft) {
  constexpr int n = DIM + 2;
  if (!(dt > 0.0)) {  // a step of length 0 (t_end reached): no transport
#pragma unroll
    for (int i = 0; i < n; ++i) F[i] = Ft[i] = 0.0;
    return;
  }
  const double D = K + DIM;
  Maxw gl, gr;
  maxw_init<DIM>(Wl, gamma, K, gl);
  maxw_init<DIM>(Wr, gamma, K, gr);
  double b[4], alx[4], aly[4], arx[4], ary[4];
#pragma unroll
  for (int i = 0; i < n; ++i) b[i] = Wlx[i] * gl.ir;
  solve_slope<DIM>(gl, D, i4D, b, alx);
#pragma unroll
  for (int i = 0; i < n; ++i) b[i] = Wrx[i] * gr.ir;
  solve_slope<DIM>(gr, D, i4D, b, arx);
  if (DIM == 2) {
#pragma unroll
    for (int i = 0; i < n; ++i) b[i] = Wly[i] * gl.ir;
    solve_slope<DIM>(gl, D, i4D, b, aly);
#pragma unroll
    for (int i = 0; i < n; ++i) b[i] = Wry[i] * gr.ir;
    solve_slope<DIM>(gr, D, i4D, b, ary);
  }
  double mlp[7], mrn[7];
  half_moments(gl, true, mlp);
  half_moments(gr, false, mrn);
  // kinetic-weighted equilibrium state and its derivatives
  double Wc[4], Wcx[4], Wcy[4], t1[4], t2[4];
#pragma unroll
  for (int i = 0; i < n; ++i) Wc[i] = gl.rho * mom1<DIM>(i, 0, 0, mlp, gl) + gr.rho * mom1<DIM>(i, 0, 0, mrn, gr);
  slope_moments<DIM>(alx, 0, 0, mlp, gl, t1);
  slope_moments<DIM>(arx, 0, 0, mrn, gr, t2);
#pragma unroll
  for (int i = 0; i < n; ++i) Wcx[i] = t1[i] + t2[i];
  if (DIM == 2) {
    slope_moments<DIM>(aly, 0, 0, mlp, gl, t1);
    slope_moments<DIM>(ary, 0, 0, mrn, gr, t2);
#pragma unroll
    for (int i = 0; i < n; ++i) Wcy[i] = t1[i] + t2[i];
  }
  Maxw gc;
  maxw_init<DIM>(Wc, gamma, K, gc);
  double acx[4], acy[4] = {0.0, 0.0, 0.0, 0.0}, Ac[4];
#pragma unroll
  for (int i = 0; i < n; ++i) b[i] = Wcx[i] * gc.ir;
  solve_slope<DIM>(gc, D, i4D, b, acx);
  if (DIM == 2) {
#pragma unroll
    for (int i = 0; i < n; ++i) b[i] = Wcy[i] * gc.ir;
    solve_slope<DIM>(gc, D, i4D, b, acy);
  }
  // compatibility: <psi psi^T> A = -(<u a_x psi> + <v a_y psi>)
  slope_moments<DIM>(acx, 1, 0, gc.mu, gc, t1);
  if (DIM == 2) slope_moments<DIM>(acy, 0, 1, gc.mu, gc, t2);
#pragma unroll
  for (int i = 0; i < n; ++i) b[i] = -(t1[i] + (DIM == 2 ? t2[i] : 0.0)) * gc.ir;
  solve_slope<DIM>(gc, D, i4D, b, Ac);
  // flux vectors
  double T0[4], T1[4], T2[4], T3[4], T4[4];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    T0[i] = gc.rho * mom1<DIM>(i, 1, 0, gc.mu, gc);
    T3[i] = gl.rho * mom1<DIM>(i, 1, 0, mlp, gl) + gr.rho * mom1<DIM>(i, 1, 0, mrn, gr);
  }
  slope_moments<DIM>(acx, 2, 0, gc.mu, gc, T1);
  slope_moments<DIM>(Ac, 1, 0, gc.mu, gc, T2);
  slope_moments<DIM>(alx, 2, 0, mlp, gl, t1);
  slope_moments<DIM>(arx, 2, 0, mrn, gr, t2);
#pragma unroll
  for (int i = 0; i < n; ++i) T4[i] = t1[i] + t2[i];
  if (DIM == 2) {
    slope_moments<DIM>(acy, 1, 1, gc.mu, gc, t1);
#pragma unroll
    for (int i = 0; i < n; ++i) T1[i] += t1[i];
    slope_moments<DIM>(aly, 1, 1, mlp, gl, t1);
    slope_moments<DIM>(ary, 1, 1, mrn, gr, t2);
#pragma unroll
    for (int i = 0; i < n; ++i) T4[i] += t1[i] + t2[i];
  }
  // numerical collision time and the time integrals over [0, dt] and [0, dt/2]
  const double pl = gl.rho * gl.h, pr = gr.rho * gr.h;
  const double taun = C1 * dt + C2 * (fabs(pl - pr) * rcp_pos(pl + pr)) * dt;
  // exp(-dt / tau_n) = exp(-dt / (2 tau_n))^2
  const double eh = exp(-0.5 * dt * rcp_pos(taun));
  double Fd[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double d = (h == 0) ? dt : 0.5 * dt;
    const double e = (h == 0) ? eh * eh : eh;
    const double c1 = d - taun * (1.0 - e);
    const double c2 = taun * taun * (1.0 - e) - taun * d * e;
    const double c3 = 0.5 * d * d;
    const double c4 = taun * (1.0 - e);
#pragma unroll
    for (int i = 0; i < n; ++i) Fd[h][i] = c1 * T0[i] + c2 * (T1[i] - T4[i]) + c3 * T2[i] + c4 * T3[i];
  }
#pragma unroll
  for (int i = 0; i < n; ++i) {
    F[i] = (4.0 * Fd[1][i] - Fd[0][i]) * idt;
    Ft[i] = 4.0 * (Fd[0][i] - 2.0 * Fd[1][i]) * idt * idt;
  }
}

// sigma of one Gauss point (Sec. 3.1) for physical states in the face frame:
// |dp| (1/p_a + 1/p_b) + (dMa_n)^2 + (dMa_t)^2, with seeded reciprocals of rho and p and
// seeded reciprocal square roots of c^2 (no FP64 division or square root)
template <int C, int NI, int TI>
__device__ __forceinline__ double sigma_point(const double* qa, const double* qb, double gamma) {
  const double ia = rcp_pos(qa[0]), ib = rcp_pos(qb[0]);
  const double ua = qa[NI] * ia, ub = qb[NI] * ib;
  const double wa = (C == 4) ? qa[TI] * ia : 0.0, wb = (C == 4) ? qb[TI] * ib : 0.0;
  const double pa = (gamma - 1.0) * (qa[C - 1] - 0.5 * qa[0] * (ua * ua + wa * wa));
  const double pb = (gamma - 1.0) * (qb[C - 1] - 0.5 * qb[0] * (ub * ub + wb * wb));
  const double ica = rsqrt_pos(gamma * pa * ia), icb = rsqrt_pos(gamma * pb * ib);  // 1 / c
  const double dp = fabs(pa - pb);
  const double dmn = ua * ica - ub * icb;
  double s = fma(dp, rcp_pos(pa) + rcp_pos(pb), dmn * dmn);
  if (C == 4) {
    const double dmt = wa * ica - wb * icb;
    s = fma(dmt, dmt, s);
  }
  return s;
}

template <int C>
__device__ __forceinline__ bool gks_physical(const double* q, double gamma) {
  double mm = q[1] * q[1];
  if (C == 4) mm = fma(q[2], q[2], mm);
  const double pr = (gamma - 1.0) * fma(q[C - 1], q[0], -0.5 * mm);
  return pos_finite(q[0]) && pos_finite(pr);
}

// ---------------------------------------------------------------------------------
// the face kernel
// ---------------------------------------------------------------------------------
// One (face, Gauss point) per thread.  The gas-kinetic flux needs ~200 registers, so in 2D
// a CTA of 128 threads with a tile of TN x TT faces, TN TT G ~ 128, runs two to an SM: while
// one CTA waits at a barrier or reconstructs its band, the other keeps the FP64 pipe busy,
// and the tiles are small enough that the last wave of a 100^2 grid is a small part of it.
// 1D: 256 faces per CTA of 256 threads.
template <int R, int DIM>
struct GksShape {
  static constexpr int G = (DIM == 2) ? (R == 3 ? 1 : (R - 1) / 2) : 1;
  static constexpr int NT = (DIM == 2) ? 128 : 256;
  static constexpr int MINB = (DIM == 2) ? 2 : 1;
  static constexpr int TN = (DIM == 2) ? (G == 1 ? 8 : 4) : 256;
  static constexpr int TT = (DIM == 2) ? NT / (TN * G) : 1;  // r9: 8, r7: 10, r5: 16, r3: 16
};

template <int R, int DIM>
using GksTileShape = Tile<R, DIM, GksShape<R, DIM>::TT, GksShape<R, DIM>::TN>;

template <int R, int DIM>
struct GksTile {
  using TL = GksTileShape<R, DIM>;
  // + normal derivatives at both faces, + per-point flux, flux derivative and sigma
  static constexpr size_t smem_doubles = TL::smem_doubles + 2 * (size_t)TL::C * TL::NB * TL::NQ +
                                         (size_t)TL::TN * TL::TT * TL::G * (2 * TL::C + 1);
};

template <int R, int DIM, int DIR>
__global__ void __launch_bounds__(GksShape<R, DIM>::NT, GksShape<R, DIM>::MINB)
gks_sweep_kernel(const GridInfo g, const GksSweepArgs args, const __grid_constant__ Tables T,
                 const __grid_constant__ DTables D) {
  using TL = GksTileShape<R, DIM>;
  constexpr int K = TL::K, C = TL::C, KT = TL::KT, G = TL::G;
  constexpr int TN = TL::TN, TT = TL::TT, NT = GksShape<R, DIM>::NT;
  constexpr int NA = TL::NA, NB = TL::NB, NQ = TL::NQ, NSN = TL::NSN, NST = TL::NST;
  constexpr int NI = (DIR == 0) ? 1 : 2;
  constexpr int TI = (DIR == 0) ? 2 : 1;

  extern __shared__ double smem[];
  double* sW = smem;                 // [C][NB][NA]
  double* sQP = sW + C * NB * NA;    // values at xi = 0 / -1
  double* sQM = sQP + C * NB * NQ;
  double* sSn = sQM + C * NB * NQ;
  double* sSt = sSn + NB * NSN;
  double* sDP = sSt + (DIM == 2 ? NQ * NST : 0);  // normal derivatives (physical) at xi = 0 / -1
  double* sDM = sDP + C * NB * NQ;
  double* sR = sDM + C * NB * NQ;                 // [TN TT][G][2C + 1]: F, F_t, sigma per point

  const int n = (DIR == 0) ? g.nx : g.ny;
  const int mlin = (DIR == 0) ? g.ny : g.nx;
  const int a0 = blockIdx.x * TN, b0 = blockIdx.y * TT;
  const int tid = threadIdx.x;
  const double dt = args.dt_fixed > 0.0 ? args.dt_fixed : args.st->dt;
  const double ts = stage_time(args.st, args.tfrac, dt);  // for time-dependent ghosts
  const double idt = 1.0 / dt;
  // internal degrees of freedom K (Sec. 2.2) and 4 / (K + DIM) of the slope solves
  const double Kdof = (DIM == 2) ? (4.0 - 2.0 * g.gamma) / (g.gamma - 1.0) : (3.0 - g.gamma) / (g.gamma - 1.0);
  const double i4D = 4.0 / (Kdof + DIM);

  for (int idx = tid; idx < C * NB * NA; idx += NT) {
    int c, bb, ai;
    if (DIR == 0) { ai = idx % NA; bb = (idx / NA) % NB; c = idx / (NA * NB); }
    else { bb = idx % NB; ai = (idx / NB) % NA; c = idx / (NA * NB); }
    const int a = a0 - 1 - K + ai, b = b0 - KT + bb;
    const int i = (DIR == 0) ? a : b, j = (DIR == 0) ? b : a;
    sW[(c * NB + bb) * NA + ai] = fetch_w(g, args.W, c, i, j, ts);
  }
  for (int idx = tid; idx < NB * NSN; idx += NT) {
    const int fa = idx % NSN, bb = idx / NSN;
    sSn[bb * NSN + fa] = (DIR == 0) ? sigma_x_at(g, args.s_norm, a0 - K + fa, b0 - KT + bb)
                                    : sigma_y_at(g, args.s_norm, a0 - K + fa, b0 - KT + bb);
  }
  if (DIM == 2) {
    for (int idx = tid; idx < NQ * (NST - 1); idx += NT) {
      const int qa = idx % NQ, fb = idx / NQ;
      sSt[qa * NST + fb] = (DIR == 0) ? sigma_y_at(g, args.s_tan, b0 - K + 1 + fb, a0 - 1 + qa)
                                      : sigma_x_at(g, args.s_tan, b0 - K + 1 + fb, a0 - 1 + qa);
    }
  }
  __syncthreads();
  // phase 1: value and normal derivative of every cell of the band at both faces
  for (int it = tid; it < NQ * NB; it += NT) {
    const int qa = it % NQ, bb = it / NQ;
    const Branch br = select_branch<R>(sSn + bb * NSN + qa, g.thres);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const double* v = sW + (c * NB + bb) * NA + qa + K;
      double out[2], dout[2];
      recon_eval_d<R, 2>(v, 1, br, T, D, 0, out, dout);
      sQP[(c * NB + bb) * NQ + qa] = out[0];
      sQM[(c * NB + bb) * NQ + qa] = out[1];
      sDP[(c * NB + bb) * NQ + qa] = dout[0] * args.inv_dn;
      sDM[(c * NB + bb) * NQ + qa] = dout[1] * args.inv_dn;
    }
  }
  __syncthreads();

  // phase 2: one (face, Gauss point) per thread; the G points of a face are neighbours
  constexpr int NF = TN * TT;
  for (int it = tid; it < NF * G; it += NT) {
    const int fi = it / G, q = it % G;
    int fa, tb;
    if (DIR == 0) { fa = fi % TN; tb = fi / TN; }
    else { tb = fi % TT; fa = fi / TT; }
    const int f = a0 + fa, b = b0 + tb;
    if (f > n || b >= mlin) continue;
    // each side's value, normal (x) and tangential (y) derivative at point q, face frame
    // (rho, m_n, m_t, E)
    double ql[C], qr[C], qlx[C], qrx[C], qly[C], qry[C];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int qa = fa + side;
      const double* Q = side == 0 ? sQP : sQM;
      const double* Dn = side == 0 ? sDP : sDM;
      double* v = side == 0 ? ql : qr;
      double* vx = side == 0 ? qlx : qrx;
      double* vy = side == 0 ? qly : qry;
      Branch bt;
      if (DIM == 2) bt = select_branch<R>(sSt + qa * NST + tb, g.thres);  // the side's column
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int src = (c == 1) ? NI : (c == 2 && C == 4) ? TI : c;
        if (DIM == 2) {
          double o, d, nd;
          recon_eval_d<R, 1>(Q + (src * NB + tb + K) * NQ + qa, NQ, bt, T, D, 2 + q, &o, &d);
          recon_eval<R, 1>(Dn + (src * NB + tb + K) * NQ + qa, NQ, bt, T, 2 + q, &nd);
          v[c] = o;
          vx[c] = nd;
          vy[c] = d * args.inv_dt;
        } else {
          v[c] = Q[src * NQ + qa];
          vx[c] = Dn[src * NQ + qa];
          vy[c] = 0.0;
        }
      }
    }
    double sg;
    if (!(gks_physical<C>(ql, g.gamma) && gks_physical<C>(qr, g.gamma))) {
      // first-order fallback: the two cell averages, no slopes
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int src = (c == 1) ? NI : (c == 2 && C == 4) ? TI : c;
        ql[c] = sW[(src * NB + tb + KT) * NA + fa + K];
        qr[c] = sW[(src * NB + tb + KT) * NA + fa + K + 1];
        qlx[c] = qrx[c] = qly[c] = qry[c] = 0.0;
      }
      sg = kSigmaBig;
      atomicOr(&const_cast<DevState*>(args.st)->flags, 0x2u);
    } else {
      sg = sigma_point<C, 1, 2>(ql, qr, g.gamma);
    }
    double Fq[C], Ftq[C];
    gks_point<DIM>(ql, qlx, qly, qr, qrx, qry, g.gamma, Kdof, i4D, dt, idt, args.c1, args.c2, Fq, Ftq);
    double* res = sR + (size_t)it * (2 * C + 1);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      res[c] = Fq[c];
      res[C + c] = Ftq[c];
    }
    res[2 * C] = sg;
  }
  __syncthreads();

  // Gauss sums per face, points in order
  for (int fi = tid; fi < NF; fi += NT) {
    int fa, tb;
    if (DIR == 0) { fa = fi % TN; tb = fi / TN; }
    else { tb = fi % TT; fa = fi / TT; }
    const int f = a0 + fa, b = b0 + tb;
    if (f > n || b >= mlin) continue;
    double Fs[C], Fts[C];
#pragma unroll
    for (int c = 0; c < C; ++c) Fs[c] = Fts[c] = 0.0;
    double ssum = 0.0;
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const double* res = sR + (size_t)(fi * G + q) * (2 * C + 1);
      const double w = (DIM == 2) ? T.gw[q] : 1.0;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int dst = (c == 1) ? NI : (c == 2 && C == 4) ? TI : c;
        Fs[dst] = fma(w, res[c], Fs[dst]);
        Fts[dst] = fma(w, res[C + c], Fts[dst]);
      }
      ssum += res[2 * C];
    }
    const double sface = (G == 1) ? ssum : ssum * (1.0 / G);
    if (DIR == 0) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        args.F[((size_t)c * g.ny + b) * (g.nx + 1) + f] = Fs[c];
        args.Ft[((size_t)c * g.ny + b) * (g.nx + 1) + f] = Fts[c];
      }
      args.s_out[(size_t)b * (g.nx + 1) + f] = sface;
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        args.F[((size_t)c * (g.ny + 1) + f) * g.nx + b] = Fs[c];
        args.Ft[((size_t)c * (g.ny + 1) + f) * g.nx + b] = Fts[c];
      }
      args.s_out[(size_t)f * g.nx + b] = sface;
    }
  }
}

template <int R, int DIM, int DIR>
cudaError_t gks_launch(const GridInfo& g, const GksSweepArgs& a, const Tables& t, const DTables& d,
                       cudaStream_t s) {
  using TL = GksTileShape<R, DIM>;
  const size_t smem = GksTile<R, DIM>::smem_doubles * sizeof(double);
  auto k = gks_sweep_kernel<R, DIM, DIR>;
  static std::atomic<unsigned long long> attr_done{0ull};
  {
    cudaError_t e = ensure_smem_limit(k, smem, attr_done);
    if (e != cudaSuccess) return e;
  }
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int m = (DIR == 0) ? g.ny : g.nx;
  dim3 grid((n + 1 + TL::TN - 1) / TL::TN, (m + TL::TT - 1) / TL::TT);
  k<<<grid, GksShape<R, DIM>::NT, smem, s>>>(g, a, t, d);
  return cudaGetLastError();
}

}  // namespace

#define ASE_DF_CAT2(a, b) a##b
#define ASE_DF_CAT(a, b) ASE_DF_CAT2(a, b)

cudaError_t ASE_DF_CAT(launch_gks_sweep_r, ASE_DF_ORDER)(int dim, int dir, const GridInfo& g, const GksSweepArgs& a,
                                                         const Tables& t, const DTables& d, cudaStream_t s) {
  constexpr int R = ASE_DF_ORDER;
  if (dim == 1) return gks_launch<R, 1, 0>(g, a, t, d, s);
  if (dir == 0) return gks_launch<R, 2, 0>(g, a, t, d, s);
  return gks_launch<R, 2, 1>(g, a, t, d, s);
}

}  // namespace asedf
