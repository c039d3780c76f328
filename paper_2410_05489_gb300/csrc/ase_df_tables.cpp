// Host-side construction of the reconstruction tables (exact rational arithmetic).
//
// A polynomial p(xi) of degree n-1 is fixed by its averages over the n cells
// [o-1, o] of a stencil (offsets o relative to the reconstructing cell [-1, 0]); this
// is the problem every coefficient table of Sec. 3.2-3.4 solves.  Here it is solved in
// the monomial basis: with the moment matrix M[i][q] = mean of xi^q over cell o_i,
// p's coefficients are c = M^{-1} W, so the value at a point xi is
// sum_i (sum_q xi^q M^{-1}[q][i]) W_i.  M^{-1} is computed exactly with 128-bit
// rationals; point weights at rational points are exact, at the irrational Gauss
// points they are summed in long double and rounded once.  Nothing here allocates
// (fixed-size arrays on the stack), so every entry point may call it.

#include <cmath>
#include <cstdint>
#include <cstring>

#include "ase_df_internal.cuh"

namespace asedf {
namespace {

typedef __int128 i128;

i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

struct Rat {
  i128 n, d;
};

Rat mk(i128 n, i128 d) {
  if (d < 0) { n = -n; d = -d; }
  i128 g = gcd128(n, d);
  if (g == 0) g = 1;
  return Rat{n / g, d / g};
}
Rat add(Rat a, Rat b) { return mk(a.n * b.d + b.n * a.d, a.d * b.d); }
Rat sub(Rat a, Rat b) { return mk(a.n * b.d - b.n * a.d, a.d * b.d); }
Rat mul(Rat a, Rat b) { return mk(a.n * b.n, a.d * b.d); }
Rat dvd(Rat a, Rat b) { return mk(a.n * b.d, a.d * b.n); }
long double to_ld(Rat a) { return (long double)a.n / (long double)a.d; }
double to_d(Rat a) { return (double)to_ld(a); }

i128 ipow(i128 b, int e) {
  i128 r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Inverse of the moment matrix of n <= 9 cells with the given offsets:
// inv.m[q][i] = coefficient of xi^q contributed by a unit average in cell i.  Fixed-size
// arrays only (no heap), so that the no-allocation residual can build its tables too.
struct Inverse {
  int n;
  Rat m[9][9];
};

bool moment_inverse(const int* offs, int n, Inverse* inv) {
  if (n < 1 || n > 9) return false;
  Rat A[9][18];
  for (int i = 0; i < n; ++i) {
    for (int q = 0; q < n; ++q) {
      i128 o = offs[i];
      A[i][q] = mk(ipow(o, q + 1) - ipow(o - 1, q + 1), q + 1);
    }
    for (int j = 0; j < n; ++j) A[i][n + j] = mk(i == j ? 1 : 0, 1);
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    while (piv < n && A[piv][col].n == 0) ++piv;
    if (piv == n) return false;  // singular (cannot happen for distinct offsets)
    for (int j = 0; j < 2 * n; ++j) {
      Rat t = A[piv][j];
      A[piv][j] = A[col][j];
      A[col][j] = t;
    }
    Rat pv = A[col][col];
    for (int j = 0; j < 2 * n; ++j) A[col][j] = dvd(A[col][j], pv);
    for (int r = 0; r < n; ++r) {
      if (r == col || A[r][col].n == 0) continue;
      Rat f = A[r][col];
      for (int j = 0; j < 2 * n; ++j) A[r][j] = sub(A[r][j], mul(f, A[col][j]));
    }
  }
  // A = [I | M^{-1}] with rows indexed by q (the unknown) after elimination
  inv->n = n;
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i) inv->m[q][i] = A[q][n + i];
  return true;
}

// Centred stencil of 2h+1 cells.
bool centred_inverse(int h, Inverse* inv) {
  int offs[9];
  for (int i = 0; i < 2 * h + 1; ++i) offs[i] = i - h;
  return moment_inverse(offs, 2 * h + 1, inv);
}

// Gauss-Legendre nodes/weights on [0, 1] by Newton iteration on P_G (three-term
// recurrence), in long double.
void gauss_legendre(int G, long double* t, long double* w) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < G; ++i) {
    long double x = cosl(pi * (i + 0.75L) / (G + 0.5L));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = x;
      for (int k = 2; k <= G; ++k) {
        long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (G == 1) { p1 = x; p0 = 1; }
      dp = G * (x * p1 - p0) / (x * x - 1);
      long double dx = p1 / dp;
      x -= dx;
      if (fabsl(dx) < 1e-30L) break;
    }
    // ascending order on [0, 1]
    t[G - 1 - i] = 0.5L * (x + 1);
    w[G - 1 - i] = 1.0L / ((1 - x * x) * dp * dp);  // weight on [-1,1] is 2/((1-x^2)P'^2); halved
  }
}

// Value weights of the polynomial of the given stencil at point xi (exact for rational
// xi given as a Rat, else long double).
void point_weights_rat(const Inverse& inv, Rat xi, double* w) {
  const int n = inv.n;
  for (int i = 0; i < n; ++i) {
    Rat s = mk(0, 1);
    Rat xp = mk(1, 1);
    for (int q = 0; q < n; ++q) {
      s = add(s, mul(xp, inv.m[q][i]));
      xp = mul(xp, xi);
    }
    w[i] = to_d(s);
  }
}

void point_weights_ld(const Inverse& inv, long double xi, double* w) {
  const int n = inv.n;
  for (int i = 0; i < n; ++i) {
    long double s = 0;
    for (int q = n - 1; q >= 0; --q) s = s * xi + to_ld(inv.m[q][i]);  // Horner
    w[i] = (double)s;
  }
}

// Derivative weights d/dxi of the polynomial at point xi: sum_q q xi^(q-1) inv[q][i].
void deriv_weights_rat(const Inverse& inv, Rat xi, double* w) {
  const int n = inv.n;
  for (int i = 0; i < n; ++i) {
    Rat s = mk(0, 1);
    Rat xp = mk(1, 1);
    for (int q = 1; q < n; ++q) {
      s = add(s, mul(mul(mk(q, 1), xp), inv.m[q][i]));
      xp = mul(xp, xi);
    }
    w[i] = to_d(s);
  }
}

void deriv_weights_ld(const Inverse& inv, long double xi, double* w) {
  const int n = inv.n;
  for (int i = 0; i < n; ++i) {
    long double s = 0;
    for (int q = n - 1; q >= 1; --q) s = s * xi + (long double)q * to_ld(inv.m[q][i]);  // Horner
    w[i] = (double)s;
  }
}

}  // namespace

bool build_dtables(int r, int ndim, DTables* D) {
  std::memset(D, 0, sizeof(DTables));
  const int G = (ndim == 2) ? (r == 3 ? 1 : (r - 1) / 2) : 1;
  long double gt[4], gwt[4];
  gauss_legendre(G, gt, gwt);
  const int npts = 2 + G;
  auto eval_all = [&](const Inverse& inv, int p, double* w) {
    if (p == 0) deriv_weights_rat(inv, mk(0, 1), w);
    else if (p == 1) deriv_weights_rat(inv, mk(-1, 1), w);
    else deriv_weights_ld(inv, gt[p - 2] - 1.0L, w);
  };
  Inverse inv;
  for (int b = 0; b < 4; ++b) {
    const int h = b + 1;
    if (!centred_inverse(h, &inv)) return false;
    for (int p = 0; p < npts; ++p) {
      double w[9];
      eval_all(inv, p, w);
      for (int i = 0; i < 2 * h + 1; ++i) D->dlin[b][p][4 - h + i] = w[i];
    }
  }
  for (int k = 0; k < 3; ++k) {
    const int offs[3] = {k - 2, k - 1, k};
    if (!moment_inverse(offs, 3, &inv)) return false;
    for (int p = 0; p < npts; ++p) eval_all(inv, p, D->dsub[k][p]);
  }
  return true;
}

bool build_tables(int r, int ndim, Tables* T) {
  std::memset(T, 0, sizeof(Tables));
  const int G = (ndim == 2) ? (r == 3 ? 1 : (r - 1) / 2) : 1;
  long double gt[4], gwt[4];
  gauss_legendre(G, gt, gwt);
  for (int g = 0; g < G; ++g) {
    T->gw[g] = (double)gwt[g];
    T->hgw[g] = (double)(0.5L * gwt[g]);
  }
  const int npts = 2 + G;

  auto eval_all = [&](const Inverse& inv, int p, double* w) {
    if (p == 0) point_weights_rat(inv, mk(0, 1), w);
    else if (p == 1) point_weights_rat(inv, mk(-1, 1), w);
    else point_weights_ld(inv, gt[p - 2] - 1.0L, w);
  };

  Inverse inv;
  // centred stencils of 3, 5, 7, 9 cells
  for (int b = 0; b < 4; ++b) {
    const int h = b + 1;
    if (!centred_inverse(h, &inv)) return false;
    for (int p = 0; p < npts; ++p) {
      double w[9];
      eval_all(inv, p, w);
      for (int i = 0; i < 2 * h + 1; ++i) T->lin[b][p][4 - h + i] = w[i];
    }
  }
  // symmetric / antisymmetric weights of the order-r linear branch at the Gauss points
  // (the reflection about the cell centre maps eta to -1 - eta and W_t to W_-t)
  {
    const int h = (r - 1) / 2;
    if (!centred_inverse(h, &inv)) return false;
    for (int g = 0; g < (G + 1) / 2 && g < 2; ++g) {
      long double w[9];
      const long double xi = gt[g] - 1.0L;
      for (int i = 0; i < 2 * h + 1; ++i) {
        long double sacc = 0;
        for (int q = 2 * h; q >= 0; --q) sacc = sacc * xi + to_ld(inv.m[q][i]);
        w[i] = sacc;
      }
      T->se[g][0] = (double)w[h];
      for (int t = 1; t <= h; ++t) {
        T->se[g][t] = (double)(0.5L * (w[h + t] + w[h - t]));
        T->so[g][t] = (double)(0.5L * (w[h + t] - w[h - t]));
      }
    }
  }
  // 3-cell sub-stencils S3_{-1}, S3_0, S3_1
  for (int k = 0; k < 3; ++k) {
    const int offs[3] = {k - 2, k - 1, k};
    if (!moment_inverse(offs, 3, &inv)) return false;
    for (int p = 0; p < npts; ++p) eval_all(inv, p, T->sub[k][p]);
    for (int q = 0; q < 2; ++q)
      for (int j = 0; j < 3; ++j) T->cq[k][q][j] = to_d(inv.m[q + 1][j]);
  }
  // Sec. 3.2: d5 = d_Hi, d3_{+-1} = (1-d_Hi)(1-d_Lo)/2, d3_0 = (1-d_Hi) d_Lo with
  // d_Hi = d_Lo = 0.85 (exact decimal values rounded once)
  T->d5 = to_d(mk(85, 100));
  T->d3[0] = to_d(mk(15 * 15, 100 * 100 * 2));
  T->d3[1] = to_d(mk(15 * 85, 100 * 100));
  T->d3[2] = T->d3[0];
  T->eps = 1e-6;
  return true;
}

}  // namespace asedf
