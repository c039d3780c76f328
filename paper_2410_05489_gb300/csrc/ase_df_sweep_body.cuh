// Device body of the fused ASE-DF face sweep (shared by the one-problem kernel and the
// batched persistent kernel).  See ase_df_sweep.cu for the algorithm.
#pragma once

#include <cuda_runtime.h>

#include "ase_df_device.cuh"
#include "ase_df_internal.cuh"

namespace asedf {
namespace {


// Branch of Algorithm 1 capped at order R, from the 2K face strengths of a cell's
// stencil, s[m+K-1] = sigma_{m-1/2} (m = -K+1..K).  Stencil sums use one fixed
// association, symmetric under mirroring: A3 = left + right,
// A5 = (s_-3/2 + s_-1/2) + (s_1/2 + s_3/2), A7 = A5 + (s_-5/2 + s_5/2),
// A9 = A7 + (s_-7/2 + s_7/2).  Smooth iff A < sigma_thres; else alpha = sigma_thres / A.
struct Branch {
  int m;          // R..5 odd: linear m-th order; 0: WENOZ-AO(5,3)+DF; 3: linear 3; -3: DF-damped 3
  double a3[3];   // alpha of S3_{-1}, S3_0, S3_1 (fallback)
  double a5;      // alpha of S5 (fallback) / of S3_0 (DF-damped order 3)
};

template <int R>
__device__ __forceinline__ Branch select_branch(const double* s, double thres) {
  constexpr int K = (R - 1) / 2;
  Branch b;
  b.m = R;
  b.a3[0] = b.a3[1] = b.a3[2] = 1.0;
  b.a5 = 1.0;
  // Smooth data without FP64 arithmetic: if every one of the 2K <= 8 strengths is at most
  // thres/16 (compared as unsigned bit patterns, so negative values and NaN fail), each
  // stencil sum is at most 8 thres/16 = thres/2 also after rounding (rounded addition is
  // monotone in its operands), so every sum is below thres and the branch is linear order R.
  {
    const long long tb = dbits(thres);
    const unsigned long long lim = ((tb >> 52) > 4) ? (unsigned long long)(tb - (4LL << 52)) : 0ull;
    unsigned long long mx = (unsigned long long)dbits(s[0]);
#pragma unroll
    for (int t = 1; t < 2 * K; ++t) mx = max(mx, (unsigned long long)dbits(s[t]));
    if (mx <= lim) return b;
  }
  const double sm12 = s[K - 1], sp12 = s[K];  // sigma_{-1/2}, sigma_{1/2}
  if (R == 3) {
    const double A = sm12 + sp12;
    if (lt_pos(A, thres)) { b.m = 3; } else { b.m = -3; b.a5 = thres / A; }
    return b;
  }
  const double sm32 = s[K - 2], sp32 = s[K + 1];
  const double A5 = (sm32 + sm12) + (sp12 + sp32);
  if (!lt_pos(A5, thres)) {
    b.m = 0;
    const double A3m = sm32 + sm12, A30 = sm12 + sp12, A3p = sp12 + sp32;
    b.a3[0] = lt_pos(A3m, thres) ? 1.0 : thres / A3m;
    b.a3[1] = lt_pos(A30, thres) ? 1.0 : thres / A30;
    b.a3[2] = lt_pos(A3p, thres) ? 1.0 : thres / A3p;
    b.a5 = thres / A5;
    return b;
  }
  b.m = 5;
  if (R >= 7) {
    const double A7 = A5 + (s[K - 3] + s[K + 2]);
    if (lt_pos(A7, thres)) {
      b.m = 7;
      if (R >= 9) {
        const double A9 = A7 + (s[K - 4] + s[K + 3]);
        if (lt_pos(A9, thres)) b.m = 9;
      }
    }
  }
  return b;
}

// Histogram slot of a branch (kBranchSlots order): linear 9, 7, 5 -> 0, 1, 2; the
// WENOZ-AO(5,3)+DF fallback -> 3; linear 3 -> 4; DF-damped 3 -> 5.
__device__ __forceinline__ int branch_slot(int m) {
  return m >= 5 ? (9 - m) / 2 : (m == 0 ? 3 : (m == 3 ? 4 : 5));
}

// Linear M-cell value at point p: v points at W_0, with W_t at v[t*vs].
template <int M>
__device__ __forceinline__ double lin_eval(const double* v, int vs, const double* w) {
  constexpr int H = (M - 1) / 2;
  double acc = w[4 - H] * v[-H * vs];
#pragma unroll
  for (int t = -H + 1; t <= H; ++t) acc = fma(w[4 + t], v[t * vs], acc);
  return acc;
}

// WENOZ-AO(5,3) with DF damping (Sec. 3.2) of one component, at NP points p0..p0+NP-1.
// v points at W_0 (stride vs).
template <int NP>
__device__ __forceinline__ void weno_eval(const double* v, int vs, const Branch& br,
                                          const Tables& T, int p0, double* out) {
  double beta[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double* vk = v + (k - 2) * vs;  // sub-stencil S3_{k-1}: offsets k-2 .. k
    const double c1 = T.cq[k][0][0] * vk[0] + T.cq[k][0][1] * vk[vs] + T.cq[k][0][2] * vk[2 * vs];
    const double c2 = T.cq[k][1][0] * vk[0] + T.cq[k][1][1] * vk[vs] + T.cq[k][1][2] * vk[2 * vs];
    // int_{-1}^{0} (p')^2 + (p'')^2 for p = c0 + c1 xi + c2 xi^2
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
    const double P5 = fma(br.a5, lin_eval<5>(v, vs, T.lin[1][p]) - W0, W0);
    double P = g5 * P5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double* vk = v + (k - 2) * vs;
      const double u = T.sub[k][p][0] * vk[0] + T.sub[k][p][1] * vk[vs] + T.sub[k][p][2] * vk[2 * vs];
      P = fma(g3[k], fma(br.a3[k], u - W0, W0), P);
    }
    out[q] = P;
  }
}

// Value of the chosen polynomial of one component at NP points p0.. (Algorithm 1).
template <int R, int NP>
__device__ __forceinline__ void recon_eval(const double* v, int vs, const Branch& br,
                                           const Tables& T, int p0, double* out) {
  if (br.m == R) {
#pragma unroll
    for (int q = 0; q < NP; ++q) out[q] = lin_eval<R>(v, vs, T.lin[(R - 3) / 2][p0 + q]);
    return;
  }
  if (R == 3) {  // DF-damped 3rd order
#pragma unroll
    for (int q = 0; q < NP; ++q) out[q] = fma(br.a5, lin_eval<3>(v, vs, T.lin[0][p0 + q]) - v[0], v[0]);
    return;
  }
  if (R >= 9 && br.m == 7) {
#pragma unroll
    for (int q = 0; q < NP; ++q) out[q] = lin_eval<(R >= 7 ? 7 : 3)>(v, vs, T.lin[2][p0 + q]);
    return;
  }
  if (R >= 7 && br.m == 5) {
#pragma unroll
    for (int q = 0; q < NP; ++q) out[q] = lin_eval<5>(v, vs, T.lin[1][p0 + q]);
    return;
  }
  if (R >= 5) weno_eval<NP>(v, vs, br, T, p0, out);
}

// Gauss-point values (tangential reconstruction, Sec. 2.1) of the order-R linear
// branch, using the reflection symmetry of the centred stencil: the points eta and
// -1 - eta share E = w_0 W_0 + sum e_t (W_t + W_-t) and differ in the sign of
// O = sum o_t (W_t - W_-t).  Used for G >= 3, where it saves FMAs over G dot products.
template <int R, int G>
__device__ __forceinline__ void lin_gauss_sym(const double* v, int vs, const Tables& T, double* out) {
  constexpr int K = (R - 1) / 2;
  double S[K + 1], D[K + 1];
#pragma unroll
  for (int t = 1; t <= K; ++t) {
    S[t] = v[t * vs] + v[-t * vs];
    D[t] = v[t * vs] - v[-t * vs];
  }
#pragma unroll
  for (int g = 0; g < (G + 1) / 2; ++g) {
    double E = T.se[g][0] * v[0];
#pragma unroll
    for (int t = 1; t <= K; ++t) E = fma(T.se[g][t], S[t], E);
    if (2 * g + 1 == G) {
      out[g] = E;  // middle point
    } else {
      double O = T.so[g][1] * D[1];
#pragma unroll
      for (int t = 2; t <= K; ++t) O = fma(T.so[g][t], D[t], O);
      out[g] = E + O;
      out[G - 1 - g] = E - O;
    }
  }
}

// Tangential reconstruction at the G Gauss points (points 2..G+1 of the tables).
template <int R, int G>
__device__ __forceinline__ void tang_eval(const double* v, int vs, const Branch& br, const Tables& T,
                                          double* out) {
  if (G >= 3 && br.m == R) {
    lin_gauss_sym<R, G>(v, vs, T, out);
    return;
  }
  recon_eval<R, G>(v, vs, br, T, 2, out);
}

// Tile of the face kernels: TN faces along the sweep on TT lines.  The Lax-Friedrichs sweep
// uses 8 x 64 in 2D (measured on GB300 against 16 x 32, 16 x 16, 32 x 16 and 8 x 32: 1.4 %
// faster than 16 x 32 at order 9, from the smaller share of halo lines); 255 faces in 1D (256
// reconstructing cells: phase 1 gives every one of the 256 threads one cell).
// A 1D sweep of fewer than one 255-face tile per SM takes tiles of 31 faces in CTAs of 32
// threads (Tile<R, 1, 1, 31, 32>): FP64 issues at 2 instructions per cycle per SM, so one
// CTA of 256 threads on a 200-cell problem runs its FP64 work on one SM, 16 us per sweep.
template <int R, int DIM, int TT_ = (DIM == 2) ? 64 : 1, int TN_ = (DIM == 2) ? 8 : 255, int NT_ = 256>
struct Tile {
  static constexpr int K = (R - 1) / 2;
  static constexpr int C = (DIM == 1) ? 3 : 4;
  static constexpr int KT = (DIM == 2) ? K : 0;
  static constexpr int G = (DIM == 2) ? (R == 3 ? 1 : K) : 1;
  static constexpr int TN = TN_;                     // faces along the sweep
  static constexpr int TT = TT_;                     // lines
  static constexpr int NT = NT_;                     // threads
  static constexpr int NA = TN + 1 + 2 * K;          // staged cells along the sweep
  static constexpr int NB = TT + 2 * KT;             // staged lines
  static constexpr int NQ = TN + 1;                  // cells reconstructed along the sweep
  static constexpr int NSN = TN + 2 * K;             // normal faces staged per line
  static constexpr int NST = TT + 2 * K;             // tangential faces staged per column
  // queue of deferred fallback items (defer_item) and its two counters, after the arrays
  static constexpr int QCAP = (NQ * NB > TN * TT) ? NQ * NB : TN * TT;
  static constexpr size_t queue_offset =
      (size_t)C * NB * NA + 2 * (size_t)C * NB * NQ + (size_t)NB * NSN + (DIM == 2 ? (size_t)NQ * NST : 0);
  static constexpr size_t smem_doubles = queue_offset + ((size_t)QCAP + 2 + 1) / 2;
};

// Deferral of the work items whose branch is the WENOZ-AO(5,3)+DF fallback.  Its arithmetic
// (smoothness indicators, nonlinear weights, four sub-polynomials) is several times that of
// a linear branch, so a warp holding one such item among linear ones would run the long path
// with most lanes idle.  A deferred item goes to a queue in shared memory, which every thread
// of the CTA works through after the linear items.  The lanes of a warp that defer reserve
// their slots together: one ballot, one shared-memory atomic by the first of them, and each
// lane's rank among them.  Returns whether this lane deferred its item.
__device__ __forceinline__ bool defer_item(bool defer, int item, int* queue, unsigned int* count) {
  const unsigned int active = __activemask();
  const unsigned int m = __ballot_sync(active, defer);
  if (m == 0u) return false;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned int base = 0u;
  if (lane == leader) base = atomicAdd(count, (unsigned int)__popc(m));
  base = __shfl_sync(active, base, leader);
  if (defer) queue[base + __popc(m & ((1u << lane) - 1u))] = item;
  return defer;
}

// One tile: faces a0 .. a0+TN-1 along the sweep on lines b0 .. b0+tt-1, 1 <= tt <= TT
// (threadIdx.x is the worker index); smem holds Tile<R, DIM, TT>::smem_doubles doubles,
// laid out for TT lines whatever tt is.
template <int R, int DIM, int DIR, int TT_ = (DIM == 2) ? 64 : 1, int TN_ = (DIM == 2) ? 8 : 255, int NT_ = 256>
__device__ __forceinline__ void sweep_tile(const GridInfo& g, const SweepArgs& args, const Tables& T, int a0,
                                           int b0, int tt, double* smem) {
  using TL = Tile<R, DIM, TT_, TN_, NT_>;
  constexpr int K = TL::K, C = TL::C, KT = TL::KT, G = TL::G;
  constexpr int TN = TL::TN, TT = TL::TT, NT = TL::NT;
  constexpr int NA = TL::NA, NB = TL::NB, NQ = TL::NQ, NSN = TL::NSN, NST = TL::NST;
  constexpr int NI = (DIR == 0) ? 1 : 2;  // normal momentum component
  constexpr int TI = (DIR == 0) ? 2 : 1;  // tangential momentum component

  double* sW = smem;                       // [C][NB][NA]
  double* sQP = sW + C * NB * NA;          // [C][NB][NQ] value at xi = 0
  double* sQM = sQP + C * NB * NQ;         // [C][NB][NQ] value at xi = -1
  double* sSn = sQM + C * NB * NQ;         // [NB][NSN]
  double* sSt = sSn + NB * NSN;            // [NQ][NST]

  const int n = (DIR == 0) ? g.nx : g.ny;       // cells along the sweep
  const int mlin = (DIR == 0) ? g.ny : g.nx;    // lines
  const int tid = threadIdx.x;
  const int nb = tt + 2 * KT;  // staged lines of this tile (<= NB)

  const double ts = stage_time(args.st, args.tfrac, args.st->dt);  // for time-dependent ghosts
  __shared__ unsigned int hist_s[kBranchSlots];
  const bool counting = args.hist != nullptr;
  if (counting && tid < kBranchSlots) hist_s[tid] = 0u;
  // queue of deferred fallback items: phase 1 (cells) and phase 2 (faces) share the slots
  int* s_queue = reinterpret_cast<int*>(smem + TL::queue_offset);
  unsigned int* s_qn = reinterpret_cast<unsigned int*>(s_queue + TL::QCAP);
  if (tid < 2) s_qn[tid] = 0u;
  // ---- stage cell averages: cells a0-1-K .. a0+TN-1+K, lines b0-KT .. b0+tt+KT-1 ----
  for (int idx = tid; idx < C * nb * NA; idx += NT) {
    int c, bb, aa;
    if (DIR == 0) { aa = idx % NA; bb = (idx / NA) % nb; c = idx / (NA * nb); }
    else { bb = idx % nb; aa = (idx / nb) % NA; c = idx / (NA * nb); }
    const int a = a0 - 1 - K + aa, b = b0 - KT + bb;
    const int i = (DIR == 0) ? a : b, j = (DIR == 0) ? b : a;
    sW[(c * NB + bb) * NA + aa] = fetch_w(g, args.W, c, i, j, ts);
  }
  // ---- normal face strengths: faces a0-K .. a0+TN-1+K of every staged line ----
  for (int idx = tid; idx < nb * NSN; idx += NT) {
    int fa, bb;
    if (DIR == 0) { fa = idx % NSN; bb = idx / NSN; }
    else { bb = idx % nb; fa = idx / nb; }
    sSn[bb * NSN + fa] = (DIR == 0) ? sigma_x_at(g, args.s_norm, a0 - K + fa, b0 - KT + bb)
                                    : sigma_y_at(g, args.s_norm, a0 - K + fa, b0 - KT + bb);
  }
  // ---- tangential face strengths of the reconstructing cells' columns ----
  if (DIM == 2) {
    const int nst = tt + 2 * K - 1;  // tangential faces b0-K+1 .. b0+tt+K-1
    for (int idx = tid; idx < NQ * nst; idx += NT) {
      int qa, fb;
      if (DIR == 0) { qa = idx % NQ; fb = idx / NQ; }
      else { fb = idx % nst; qa = idx / nst; }
      sSt[qa * NST + fb] = (DIR == 0) ? sigma_y_at(g, args.s_tan, b0 - K + 1 + fb, a0 - 1 + qa)
                                      : sigma_x_at(g, args.s_tan, b0 - K + 1 + fb, a0 - 1 + qa);
    }
  }
  __syncthreads();

  // ---- phase 1: normal reconstruction of cells a0-1 .. a0+TN-1 on all staged lines ----
  // Interior cells (qa = 1 .. NQ-2) serve a face on each side and are evaluated at both
  // xi = 0 and xi = -1; the two end cells serve one tile face each (qa = 0: its xi = 0
  // value, the left state of face a0; qa = NQ-1: its xi = -1 value), so they come last in
  // the work list and evaluate one point.
  // Fallback items are deferred (defer_item) and done in a second pass.
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int count = (pass == 0) ? NQ * nb : (int)s_qn[0];
    for (int k = tid; k < count; k += NT) {
      const int it = (pass == 0) ? k : s_queue[k];
      int qa, bb, pt;  // pt -1: an interior cell, both points; 0 / 1: an end cell, one point
      if (it < (NQ - 2) * nb) {
        if (DIR == 0) { qa = 1 + it % (NQ - 2); bb = it / (NQ - 2); }
        else { bb = it % nb; qa = 1 + it / nb; }
        pt = -1;
      } else {
        const int e = it - (NQ - 2) * nb;
        bb = e % nb;  // pt 0: cell qa = 0 at xi = 0; 1: qa = NQ-1 at xi = -1
        pt = e / nb;
        qa = pt * (NQ - 1);
      }
      const Branch br = select_branch<R>(sSn + bb * NSN + qa, g.thres);
      if (R >= 5 && pass == 0 && defer_item(br.m == 0, it, s_queue, &s_qn[0])) continue;
      if (pt < 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const double* v = sW + (c * NB + bb) * NA + qa + K;  // W_0 of this cell
          double out[2];
          recon_eval<R, 2>(v, 1, br, T, 0, out);
          sQP[(c * NB + bb) * NQ + qa] = out[0];
          sQM[(c * NB + bb) * NQ + qa] = out[1];
        }
      } else {
        double* dst = pt ? sQM : sQP;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const double* v = sW + (c * NB + bb) * NA + qa + K;
          double out[1];
          recon_eval<R, 1>(v, 1, br, T, pt, out);
          dst[(c * NB + bb) * NQ + qa] = out[0];
        }
      }
    }
    __syncthreads();  // pass 0: the queue is complete; last pass: phase 1 is done
    if (R < 5 || s_qn[0] == 0u) break;
  }

  // ---- phase 2: faces ----
  // Faces with a fallback tangential reconstruction on either side are deferred (2D).
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int count = (pass == 0) ? TN * tt : (int)s_qn[1];
    for (int k = tid; k < count; k += NT) {
      const int it = (pass == 0) ? k : s_queue[k];
      int fa, tb;
      if (DIR == 0) { fa = it % TN; tb = it / TN; }
      else { tb = it % tt; fa = it / tt; }
      const int f = a0 + fa, b = b0 + tb;
      if (f > n || b >= mlin) continue;
      Branch bt[2];
      if (DIM == 2) {
        bt[0] = select_branch<R>(sSt + fa * NST + tb, g.thres);  // the columns of the two states
        bt[1] = select_branch<R>(sSt + (fa + 1) * NST + tb, g.thres);
        if (R >= 5 && pass == 0 && defer_item(bt[0].m == 0 || bt[1].m == 0, it, s_queue, &s_qn[1])) continue;
      }
      double st[2][G][C];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int qa = fa + side;  // left state: cell f-1 (plus face); right: cell f (minus face)
        const double* Q = side == 0 ? sQP : sQM;
        if (counting) {  // the normal branch of this state's cell, as phase 1 chose it
          const Branch bn = select_branch<R>(sSn + (tb + KT) * NSN + qa, g.thres);
          atomicAdd(&hist_s[branch_slot(bn.m)], 1u);
        }
        if (DIM == 2) {
          if (counting) atomicAdd(&hist_s[branch_slot(bt[side].m)], 1u);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const double* v = Q + (c * NB + tb + K) * NQ + qa;
            double out[G];
            tang_eval<R, G>(v, NQ, bt[side], T, out);
#pragma unroll
            for (int q = 0; q < G; ++q) st[side][q][c] = out[q];
          }
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) st[side][0][c] = Q[c * NQ + qa];
        }
      }
      // cell averages either side of the face (read by a Gauss point only if it falls back)
      const double* ca = sW + (tb + KT) * NA + fa + K;
      const double* cb = ca + 1;
      double Fs[C];
#pragma unroll
      for (int c = 0; c < C; ++c) Fs[c] = 0.0;
      double ssum = 0.0;
      unsigned int nfb = 0u;
#pragma unroll
      for (int q = 0; q < G; ++q) {
        double sg;
        nfb += lf_point_acc<C, NI, TI>(st[0][q], st[1][q], ca, cb, NB * NA, g.gm1, g.gg1, T.hgw[q], g.gm1_hgw[q],
                                       Fs, sg) ? 1u : 0u;
        ssum += sg;
      }
      if (nfb) {
        atomicOr(&args.st->flags, 0x2u);
        if (counting) atomicAdd(&hist_s[kBranchSlots - 1], nfb);
      }
      const double sface = (G == 1) ? ssum : ssum * (1.0 / G);
      if (DIR == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) args.F[((size_t)c * g.ny + b) * (g.nx + 1) + f] = Fs[c];
        args.s_out[(size_t)b * (g.nx + 1) + f] = sface;
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) args.F[((size_t)c * (g.ny + 1) + f) * g.nx + b] = Fs[c];
        args.s_out[(size_t)f * g.nx + b] = sface;
      }
    }
    if (DIM == 1 || R < 5 || pass == 1) break;
    __syncthreads();  // the queue is complete
    if (s_qn[1] == 0u) break;
  }
  if (counting) {
    __syncthreads();
    if (tid < kBranchSlots && hist_s[tid]) atomicAdd(&args.hist[tid], (unsigned long long)hist_s[tid]);
  }
}

}  // namespace
}  // namespace asedf
