// Host-side check of the sweep's tile plan (csrc/ase_df_tileplan.h), compiled with g++ by
// tests/test_tile_plan.py.  Over grids of 1 .. 2048 faces and lines and 1 .. 528 CTA slots:
// every (tile column, line) is covered by exactly one tile, tiles have 1 .. 64 lines, the
// plan never has fewer tiles than the uniform grid, it fills whole waves unless the line floor
// (16, or 8 for the smallest grids) caps it, and its first group's tiles are on average at
// least as tall as the second's.
// Prints "ok <plans checked>" or the first failure.
#include <cstdio>
#include <vector>

#include "ase_df_tileplan.h"

using asedf::TilePlan;

static int fail(const char* what, long long n, int m, int slots) {
  std::printf("FAIL %s: faces %lld lines %d slots %d\n", what, n, m, slots);
  return 1;
}

int main() {
  const int faces_list[] = {2, 3, 4, 6, 8, 9, 10, 16, 17, 18, 32, 34, 64, 65, 66, 101, 128, 201, 256,
                            257, 258, 512, 513, 768, 1001, 1024, 1025, 1601, 2048};
  const int lines_list[] = {1, 2, 3, 5, 9, 15, 16, 17, 31, 63, 64, 65, 100, 129, 240, 256, 511, 800,
                            960, 1024, 1025, 2000};
  const int slots_list[] = {1, 2, 3, 148, 296, 304, 528};
  const int kTN = 8, kTT = 64;
  long long checked = 0;
  for (int floor_lines : {16, 8})
  for (int faces : faces_list) {
    for (int m : lines_list) {
      for (int slots : slots_list) {
        const long long cols = (faces + kTN - 1) / kTN;
        long long tiles = 0;
        const TilePlan p = asedf::make_tile_plan(cols, m, kTT, slots, tiles, floor_lines);
        const long long q = (m + kTT - 1) / kTT;
        const long long fl = (m + floor_lines - 1) / floor_lines;
        const long long nb_max = q > fl ? q : fl;
        if (tiles < cols * q) return fail("fewer tiles than the uniform grid", faces, m, slots);
        if (tiles % slots != 0 && tiles != cols * nb_max) return fail("waves not filled", faces, m, slots);
        if ((long long)p.n1 * p.nb_lo + (long long)p.n2 * (p.nb_lo + 1) != tiles)
          return fail("tile count", faces, m, slots);
        std::vector<int> cover((size_t)cols * m, 0);
        double sum1 = 0.0, sum2 = 0.0;
        long long cnt1 = 0, cnt2 = 0;
        const long long g1 = (long long)p.n1 * p.nb_lo;
        for (long long x = 0; x < tiles; ++x) {
          int col, b0, tt;
          asedf::plan_tile(p, (int)x, col, b0, tt);
          if (col < 0 || col >= cols) return fail("column out of range", faces, m, slots);
          if (tt < 1 || tt > kTT) return fail("tile height out of 1 .. 64", faces, m, slots);
          if (b0 < 0 || b0 + tt > m) return fail("lines out of range", faces, m, slots);
          for (int b = b0; b < b0 + tt; ++b) cover[(size_t)col * m + b] += 1;
          if (x < g1) { sum1 += tt; ++cnt1; } else { sum2 += tt; ++cnt2; }
        }
        for (int v : cover)
          if (v != 1) return fail("a (column, line) not covered exactly once", faces, m, slots);
        if (cnt1 > 0 && cnt2 > 0 && sum1 / cnt1 < sum2 / cnt2)
          return fail("smaller tiles first", faces, m, slots);
        ++checked;
      }
    }
  }
  // on 152 SMs: 512^2 and 1024^2 planned (2 and 7 waves), 2048^2 (27 waves) uniform
  if (!asedf::use_tile_plan((513 + 7) / 8, 512, kTT, 304)) return fail("512^2 not planned", 513, 512, 304);
  if (!asedf::use_tile_plan((1025 + 7) / 8, 1024, kTT, 304)) return fail("1024^2 not planned", 1025, 1024, 304);
  if (asedf::use_tile_plan((2049 + 7) / 8, 2048, kTT, 304)) return fail("2048^2 planned", 2049, 2048, 304);
  // the uniform-grid parity case of tests/test_gpu_parity.py: 12001 x 110, both directions
  if (asedf::use_tile_plan((12002 + 7) / 8, 110, kTT, 304)) return fail("12001 x 110 x-sweep planned", 12002, 110, 304);
  if (asedf::use_tile_plan((111 + 7) / 8, 12001, kTT, 304)) return fail("12001 x 110 y-sweep planned", 111, 12001, 304);
  long long tiles = 0;
  const TilePlan p = asedf::make_tile_plan((1025 + 7) / 8, 1024, kTT, 304, tiles);
  if (tiles != 2128 || p.nb_lo != 16 || p.n2 != 64) return fail("1024^2 plan", 1025, 1024, 304);
  std::printf("ok %lld\n", checked);
  return 0;
}
