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

#include <algorithm>

#include "ase_df_sweep_body.cuh"

#ifndef ASE_DF_ORDER
#error "ASE_DF_ORDER must be defined"
#endif

namespace asedf {
namespace {

// Tiles of a 2D sweep: the tile columns (TN faces along the sweep) split their lines into
// nb_lo blocks (columns 0 .. n1-1) or nb_lo + 1 blocks (the others), block k of nbk covering
// lines floor(k m / nbk) .. floor((k+1) m / nbk) - 1.  CTA x takes, in order, the n1 nb_lo
// tiles of the first columns (the larger tiles, so that the last wave is of the smaller
// ones), then the others; within each group consecutive CTAs are neighbours along the sweep.
// 1D: one line, one block per column.
struct TilePlan {
  int n1, n2;  // columns with nb_lo / nb_lo + 1 blocks
  int nb_lo;
  int m;       // lines
};

__device__ __forceinline__ void plan_tile(const TilePlan& p, int x, int& col, int& b0, int& tt) {
  const int g1 = p.n1 * p.nb_lo;
  int k, nbk;
  if (x < g1) {
    col = x % p.n1; k = x / p.n1; nbk = p.nb_lo;
  } else {
    x -= g1;
    col = p.n1 + x % p.n2; k = x / p.n2; nbk = p.nb_lo + 1;
  }
  b0 = (int)(((long long)k * p.m) / nbk);
  tt = (int)(((long long)(k + 1) * p.m) / nbk) - b0;
}

// PLAN = false: a uniform grid (x: tile column, y: blocks of TT lines, the last one ragged).
template <int R, int DIM, int DIR, int TT, bool PLAN>
__global__ void __launch_bounds__(Tile<R, DIM, TT>::NT, 2)
sweep_kernel(const GridInfo g, const SweepArgs args, const __grid_constant__ Tables T, const TilePlan P) {
  extern __shared__ double smem[];
  if (DIR == 0 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x <= kRepairPasses) {
    args.st->cnt[threadIdx.x] = 0u;  // counters of the positivity repair of this stage
    args.st->rbad[threadIdx.x] = 0u;
  }
  if constexpr (PLAN) {
    int col, b0, tt;
    plan_tile(P, blockIdx.x, col, b0, tt);
    sweep_tile<R, DIM, DIR, TT>(g, args, T, col * Tile<R, DIM, TT>::TN, b0, tt, smem);
  } else {
    sweep_tile<R, DIM, DIR, TT>(g, args, T, blockIdx.x * Tile<R, DIM, TT>::TN, blockIdx.y * TT, TT, smem);
  }
}

// Plan of the tiles of one 2D sweep on `slots` CTA slots (two per SM).  Tiles of up to TT
// lines need q = ceil(m / TT) blocks per column and w = ceil(cols q / slots) waves; the plan
// fills all w waves (w slots tiles, at most ceil(m / 16) blocks per column so that no tile
// is under ~16 lines), which shortens the tiles and with them the w waves.
TilePlan make_plan(long long cols, int m, int tt_max, int slots, long long& tiles) {
  const long long q = (m + tt_max - 1) / tt_max;
  const long long t0 = cols * q;
  const long long target = (t0 + slots - 1) / slots * slots;
  const long long nb_max = std::max(q, (long long)(m + 15) / 16);
  tiles = std::min(target, cols * nb_max);
  TilePlan p;
  p.nb_lo = (int)(tiles / cols);
  p.n2 = (int)(tiles % cols);
  p.n1 = (int)(cols - p.n2);
  p.m = m;
  return p;
}

template <int R, int DIM, int DIR, int TT, bool PLAN>
cudaError_t launch_grid(const GridInfo& g, const SweepArgs& a, const Tables& t, cudaStream_t s, dim3 grid,
                        const TilePlan& p) {
  using TL = Tile<R, DIM, TT>;
  const size_t smem = TL::smem_doubles * sizeof(double);
  auto kern = sweep_kernel<R, DIM, DIR, TT, PLAN>;
  static std::atomic<unsigned long long> attr_done{0ull};
  cudaError_t e = ensure_smem_limit(kern, smem, attr_done);
  if (e != cudaSuccess) return e;
  kern<<<grid, TL::NT, smem, s>>>(g, a, t, p);
  return cudaGetLastError();
}

// 2D: tiles of 8 faces x 64 lines.  While the tiles of a sweep fill at most three waves of
// the GPU's CTA slots, the CTAs run nearly in step and a partly filled last wave costs a
// whole tile time, so the wave-filling plan is used (measured on GB300: +7 % on the 512^2
// vortex, whose 520 tiles of 64 lines become 608 of 51 - 57); on larger grids the CTAs
// drift apart over the waves, the tail costs little and the uniform grid is kept.
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
    if (cols * q <= 3LL * slots) {
      long long tiles;
      const TilePlan p = make_plan(cols, m, TT, slots, tiles);
      return launch_grid<R, DIM, DIR, TT, true>(g, a, t, s, dim3((unsigned)tiles), p);
    }
    if (cols > 0x7fffffffLL || q > 65535) return cudaErrorInvalidConfiguration;
    return launch_grid<R, DIM, DIR, TT, false>(g, a, t, s, dim3((unsigned)cols, (unsigned)q), none);
  } else {
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
