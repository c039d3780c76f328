// Tile plan of a 2D face sweep: which faces and lines each CTA of the launch owns.
//
// A tile is TN faces along the sweep (one tile column) times up to tt_max lines.  While the
// tiles of tt_max lines fill at most eight waves of the GPU's CTA slots, a partly filled last
// wave still costs a measurable part of a tile time, and the plan fills every slot of those
// waves with shorter tiles (measured on GB300: +7 % on the 512^2 vortex at two waves, +0.7 %
// on 1024^2 at 6.8 waves).  Beyond that the uniform grid of tt_max-line tiles is kept.
//
// Plain C++ as well as CUDA, so that the host-side tests compile this very header.
#pragma once

#include <algorithm>

#ifdef __CUDACC__
#define ASE_DF_HOST_DEVICE __host__ __device__ __forceinline__
#else
#define ASE_DF_HOST_DEVICE inline
#endif

namespace asedf {

// The tile columns split their m lines into nb_lo blocks (columns 0 .. n1-1) or nb_lo + 1
// blocks (the n2 others), block k of nbk covering lines floor(k m / nbk) .. floor((k+1) m /
// nbk) - 1.  CTA x takes, in order, the n1 nb_lo tiles of the first columns (the larger
// tiles, so that the last wave is of the smaller ones), then the others; within each group
// consecutive CTAs are neighbours along the sweep.
struct TilePlan {
  int n1, n2;  // columns with nb_lo / nb_lo + 1 blocks
  int nb_lo;
  int m;       // lines
};

// Tile of CTA x (0 <= x < n1 nb_lo + n2 (nb_lo + 1)): its column and its lines b0 .. b0+tt-1.
ASE_DF_HOST_DEVICE void plan_tile(const TilePlan& p, int x, int& col, int& b0, int& tt) {
  const int g1 = p.n1 * p.nb_lo;
  int k, nbk;
  if (x < g1) {
    col = x % p.n1;
    k = x / p.n1;
    nbk = p.nb_lo;
  } else {
    x -= g1;
    col = p.n1 + x % p.n2;
    k = x / p.n2;
    nbk = p.nb_lo + 1;
  }
  b0 = (int)(((long long)k * p.m) / nbk);
  tt = (int)(((long long)(k + 1) * p.m) / nbk) - b0;
}

// Whether a sweep of `cols` tile columns over m lines takes the plan on `slots` CTA slots:
// its tiles of tt_max lines fill at most eight waves.
inline bool use_tile_plan(long long cols, int m, int tt_max, int slots) {
  const long long q = (m + tt_max - 1) / tt_max;
  return cols * q <= 8LL * slots;
}

// The plan: tiles of up to tt_max lines need q = ceil(m / tt_max) blocks per column and
// w = ceil(cols q / slots) waves; the plan fills all w waves with w slots tiles, at most
// max(q, ceil(m / min_lines)) blocks per column so that no tile is under ~min_lines lines.
// `tiles` is the CTA count of the launch.  Requires cols >= 1, m >= 1, tt_max >= 1,
// slots >= 1, min_lines >= 1.
inline TilePlan make_tile_plan(long long cols, int m, int tt_max, int slots, long long& tiles,
                               int min_lines = 16) {
  const long long q = (m + tt_max - 1) / tt_max;
  const long long t0 = cols * q;
  const long long target = (t0 + slots - 1) / slots * slots;
  const long long nb_max = std::max(q, (long long)(m + min_lines - 1) / min_lines);
  tiles = std::min(target, cols * nb_max);
  TilePlan p;
  p.nb_lo = (int)(tiles / cols);
  p.n2 = (int)(tiles % cols);
  p.n1 = (int)(cols - p.n2);
  p.m = m;
  return p;
}

}  // namespace asedf
