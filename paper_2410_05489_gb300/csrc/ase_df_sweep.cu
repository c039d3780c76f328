// Fused face kernel of the ASE-DF residual for one sweep direction, sm_103a, FP64.
//
// One CTA owns a tile of TN faces along the sweep (normal) direction times up to TT lines.
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
#include "ase_df_tileplan.h"

#ifndef ASE_DF_ORDER
#error "ASE_DF_ORDER must be defined"
#endif

namespace asedf {
namespace {

// PLAN = false: a uniform grid (x: tile column, y: blocks of TT lines, the last one ragged).
// TN, NT: faces along the sweep and threads of a tile (the Tile defaults, or the small 1D tile).
template <int R, int DIM, int DIR, int TT, bool PLAN, int TN = (DIM == 2) ? 8 : 255, int NT = 256>
__global__ void __launch_bounds__(NT, (NT == 256) ? 2 : 1)
sweep_kernel(const GridInfo g, const SweepArgs args, const __grid_constant__ Tables T, const TilePlan P) {
  extern __shared__ double smem[];
  if (DIR == 0 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x <= kRepairPasses) {
    args.st->cnt[threadIdx.x] = 0u;  // counters of the positivity repair of this stage
    args.st->rbad[threadIdx.x] = 0u;
  }
  if constexpr (PLAN) {
    int col, b0, tt;
    plan_tile(P, blockIdx.x, col, b0, tt);
    sweep_tile<R, DIM, DIR, TT, TN, NT>(g, args, T, col * TN, b0, tt, smem);
  } else {
    sweep_tile<R, DIM, DIR, TT, TN, NT>(g, args, T, blockIdx.x * TN, blockIdx.y * TT, TT, smem);
  }
}

template <int R, int DIM, int DIR, int TT, bool PLAN, int TN = (DIM == 2) ? 8 : 255, int NT = 256>
cudaError_t launch_grid(const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s, dim3 grid,
                        const TilePlan& p) {
  using TL = Tile<R, DIM, TT, TN, NT>;
  const size_t smem = TL::smem_doubles * sizeof(double);
  auto kern = sweep_kernel<R, DIM, DIR, TT, PLAN, TN, NT>;
  static std::atomic<unsigned long long> attr_done{0ull};
  cudaError_t e = ensure_smem_limit(kern, smem, attr_done);
  if (e != cudaSuccess) return e;
  kern<<<grid, NT, smem, s>>>(g, a, t, p);
  return cudaGetLastError();
}

// 2D: tiles of 8 faces x 64 lines.  While the tiles of a sweep fill at most eight waves of
// the GPU's CTA slots, a partly filled last wave costs part of a tile time, so the
// wave-filling plan is used (measured on GB300: +7 % on the 512^2 vortex, whose 520 tiles of 64
// lines become 608 of 51 - 57; +0.7 % on 1024^2, whose 2064 tiles become 2128 of 60 - 64); on
// larger grids the uniform grid is kept.
template <int R, int DIM, int DIR>
cudaError_t launch(const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s) {
  constexpr int TT = (DIM == 2) ? 64 : 1;
  const int n = (DIR == 0) ? g.nx : g.ny;
  const int m = (DIR == 0) ? g.ny : g.nx;
  const long long cols = (n + 1 + Tile<R, DIM, TT>::TN - 1) / Tile<R, DIM, TT>::TN;
  const TilePlan none{};
  if constexpr (DIM == 2) {
    const int slots = 2 * device_sm_count();
    const long long q = (m + TT - 1) / TT;
    if (use_tile_plan(cols, m, TT, slots)) {
      long long tiles;
      TilePlan p = make_tile_plan(cols, m, TT, slots, tiles);
      // the smallest grids: tiles of down to 8 lines while the two concurrent sweeps still fit
      // in one wave (64^2: 72 tiles per sweep instead of 36, measured +11 %; 128^2 would need two
      // waves and keeps 16)
      long long tiles8;
      const TilePlan p8 = make_tile_plan(cols, m, TT, slots, tiles8, 8);
      if (tiles8 > tiles && 2 * tiles8 <= slots) {
        p = p8;
        tiles = tiles8;
      }
      return launch_grid<R, DIM, DIR, TT, true>(g, a, t, s, dim3((unsigned)tiles), p);
    }
    if (cols > 0x7fffffffLL || q > 65535) return cudaErrorInvalidConfiguration;
    return launch_grid<R, DIM, DIR, TT, false>(g, a, t, s, dim3((unsigned)cols, (unsigned)q), none);
  } else {
    // fewer 255-face tiles than SMs: 31-face tiles in CTAs of 32 threads spread the FP64 work
    if (cols < device_sm_count()) {
      using TS = Tile<R, 1, 1, 31, 32>;
      const long long cs = (n + 1 + TS::TN - 1) / TS::TN;
      return launch_grid<R, DIM, DIR, TT, false, 31, 32>(g, a, t, s, dim3((unsigned)cs), none);
    }
    return launch_grid<R, DIM, DIR, TT, false>(g, a, t, s, dim3((unsigned)cols), none);
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
