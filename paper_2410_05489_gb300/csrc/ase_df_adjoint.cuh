// Declarations of the adjoint (vector-Jacobian product) kernels of the ASE-DF residual.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "ase_df_internal.cuh"

namespace asedf {

// Arguments of the adjoint of one sweep direction.  "n" is the number of cells along
// the sweep and "m" the number of lines; K = (r-1)/2, KT = K in 2D and 0 in 1D.
struct AdjArgs {
  const double* Lbar;      // [C][ny][nx] adjoint of L (NULL: zero)
  double lscale;           // Lbar enters times this factor
  const double* sbar_out;  // adjoint of this direction's sigma_out, sigma layout (NULL: zero)
  // scratch (see adj_scratch_doubles)
  double* Tbar;            // [2][2KT+1][C][(n+1) m]: adjoint of the normal values per face, side, line offset
  double* Cbar;            // [2][C][(n+1) m]: adjoint of the two cell averages of a first-order face
  double* Stb;             // [2][4][(n+1) m]: sigma_in adjoints of the tangential branches (2D)
  double* Nbar;            // [2K+1][C][(n+2)(m+2KT)]: adjoint of each stencil cell of a normal reconstruction
  double* Snb;             // [4][C][(n+2)(m+2KT)]: sigma_in adjoints of the normal branches, per component
  // outputs (accumulated)
  double* Wbar;            // += [C][ny][nx]
  double* sbar_norm;       // += sigma_in adjoint of the faces normal to the sweep (NULL: not wanted)
  double* sbar_tan;        // += sigma_in adjoint of the faces along the sweep lines (2D; NULL: not wanted)
  double inv_h;            // 1/dx (x-sweep) or 1/dy (y-sweep)
};

// Scratch doubles one direction's adjoint needs (each direction has its own, so that the
// face and normal kernels of the two directions can run side by side).
inline size_t adj_scratch_doubles(int dim, int order, long long n, long long m) {
  const long long K = (order - 1) / 2, KT = (dim == 2) ? K : 0, C = (dim == 1) ? 3 : 4;
  const long long nf = (n + 1) * m, ni = (n + 2) * (m + 2 * KT);
  return (size_t)(2 * (2 * KT + 1) * C * nf + 2 * C * nf + (dim == 2 ? 8 * nf : 0) + (2 * K + 1) * C * ni + 4 * C * ni);
}

// phase: 1 = the face and normal kernels (this direction's scratch only), 2 = the gathers
// into the outputs (Wbar, sigma_in adjoints), 3 = both.
cudaError_t launch_adjoint_r3(int dim, int dir, int phase, const GridInfo& g, const SweepArgs& a,
                              const AdjArgs& aa, const Tables& t, cudaStream_t s);
cudaError_t launch_adjoint_r5(int dim, int dir, int phase, const GridInfo& g, const SweepArgs& a,
                              const AdjArgs& aa, const Tables& t, cudaStream_t s);
cudaError_t launch_adjoint_r7(int dim, int dir, int phase, const GridInfo& g, const SweepArgs& a,
                              const AdjArgs& aa, const Tables& t, cudaStream_t s);
cudaError_t launch_adjoint_r9(int dim, int dir, int phase, const GridInfo& g, const SweepArgs& a,
                              const AdjArgs& aa, const Tables& t, cudaStream_t s);

// 2D: the gathers (phase 2) of both directions in one launch, ax / ay the x- and
// y-direction's arguments (the same outputs; ax.sbar_norm == ay.sbar_tan and
// ay.sbar_norm == ax.sbar_tan).  The results equal phase 2 of x, then of y, bit for bit.
cudaError_t launch_adjoint_gathers_2d_r3(const GridInfo& g, const AdjArgs& ax, const AdjArgs& ay, cudaStream_t s);
cudaError_t launch_adjoint_gathers_2d_r5(const GridInfo& g, const AdjArgs& ax, const AdjArgs& ay, cudaStream_t s);
cudaError_t launch_adjoint_gathers_2d_r7(const GridInfo& g, const AdjArgs& ax, const AdjArgs& ay, cudaStream_t s);
cudaError_t launch_adjoint_gathers_2d_r9(const GridInfo& g, const AdjArgs& ax, const AdjArgs& ay, cudaStream_t s);

// out = a x + b y (y may be NULL, then out = a x); out may alias x or y.
cudaError_t launch_axpby(double* out, double a, const double* x, double b, const double* y, size_t n,
                         cudaStream_t s);

}  // namespace asedf
