// Fused face kernel of the ASE-DF residual for one sweep direction, sm_103a, FP64.
//
// One CTA owns a tile of TN faces along the sweep (normal) direction times TT lines.
// It stages the cell averages of the tile plus the stencil halo in shared memory (ghost
// cells resolved by the boundary index maps), then
//   phase 1: normal reconstruction (Sec. 3, Algorithm 1 with the DF factor of Eq. 3.2)
//            of every cell of the tile's band of lines, evaluated at both of its faces
//            (xi = 0 and xi = -1: one polynomial serves the left state of one face and
//            the right state of the next), into shared memory;
//   phase 2: per face, tangential reconstruction of those face line-averages at the
//            (r-1)/2 Gauss points (Sec. 2.1, Remark 2 of Sec. 3.1), the local
//            Lax-Friedrichs flux and the discontinuity strength per Gauss point
//            (Sec. 2.3, Sec. 3.1), the Gauss-weighted face flux and the face sigma.
// The face fluxes go to global memory; the flux difference and the RK combination are
// done by the combine kernel.
//
// This file is compiled once per scheme order (ASE_DF_ORDER = 3, 5, 7, 9).

#include <cuda_runtime.h>

#include "ase_df_sweep_body.cuh"

#ifndef ASE_DF_ORDER
#error "ASE_DF_ORDER must be defined"
#endif

namespace asedf {
namespace {

template <int R, int DIM, int DIR, int TT>
__global__ void __launch_bounds__(Tile<R, DIM, TT>::NT, 2)
sweep_kernel(const GridInfo g, const SweepArgs args, const __grid_constant__ Tables T) {
  extern __shared__ double smem[];
  if (DIR == 0 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x <= kRepairPasses) {
    args.st->cnt[threadIdx.x] = 0u;  // counters of the positivity repair of this stage
    args.st->rbad[threadIdx.x] = 0u;
  }
  sweep_tile<R, DIM, DIR, TT>(g, args, T, blockIdx.x * Tile<R, DIM, TT>::TN, blockIdx.y * Tile<R, DIM, TT>::TT,
                              smem);
}

template <int R, int DIM, int DIR, int TT>
cudaError_t launch_tt(const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s) {
  using TL = Tile<R, DIM, TT>;
  const size_t smem = TL::smem_doubles * sizeof(double);
  auto kern = sweep_kernel<R, DIM, DIR, TT>;
  static std::atomic<unsigned long long> attr_done{0ull};
  cudaError_t e = ensure_smem_limit(kern, smem, attr_done);
  if (e != cudaSuccess) return e;
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int m = (DIR == 0) ? g.ny : g.nx;
  dim3 grid((n + 1 + TL::TN - 1) / TL::TN, (m + TL::TT - 1) / TL::TT);
  kern<<<grid, TL::NT, smem, s>>>(g, a, t);
  return cudaGetLastError();
}

// Fraction of the CTA slots (two per SM) that a grid of `tiles` CTAs keeps busy over its waves.
double wave_fill(long long tiles, int slots) {
  const long long waves = (tiles + slots - 1) / slots;
  return waves > 0 ? (double)tiles / (double)(waves * slots) : 0.0;
}

// 2D: tiles of 8 x 64 faces (two per thread) where they fill the GPU's waves, else 8 x 32
// (one face per thread: twice the CTAs for small and medium grids; ~1 % more work per face
// from the larger share of halo lines, hence the margin).
template <int R, int DIM, int DIR>
cudaError_t launch(const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s) {
  if constexpr (DIM == 1) {
    return launch_tt<R, DIM, DIR, 1>(g, a, t, s);
  } else {
  const int slots = 2 * device_sm_count();
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int m = (DIR == 0) ? g.ny : g.nx;
  const long long cols = (n + 1 + 7) / 8;
  const double f64 = wave_fill(cols * ((m + 63) / 64), slots);
  const double f32 = wave_fill(cols * ((m + 31) / 32), slots);
  if (f32 > 1.02 * f64) return launch_tt<R, DIM, DIR, 32>(g, a, t, s);
  return launch_tt<R, DIM, DIR, 64>(g, a, t, s);
  }
}

}  // namespace

#define ASE_DF_CAT2(a, b) a##b
#define ASE_DF_CAT(a, b) ASE_DF_CAT2(a, b)

cudaError_t ASE_DF_CAT(launch_sweep_r, ASE_DF_ORDER)(int dim, int dir, const GridInfo& g, const SweepArgs& a,
                                                     const Tables& t, cudaStream_t s) {
  constexpr int R = ASE_DF_ORDER;
  if (dim == 1) return launch<R, 1, 0>(g, a, t, s);
  if (dir == 0) return launch<R, 2, 0>(g, a, t, s);
  return launch<R, 2, 1>(g, a, t, s);
}

}  // namespace asedf
