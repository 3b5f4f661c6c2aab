// Host-side check of the plane-window scheduling (grid_win.cuh), with the
// kernels' own helpers:
//   1. part_range splits a window's slot range into contiguous parts that
//      cover it once, for every part count;
//   2. the chunks of a window run (chunk_at / chunk_after: chunk c takes
//      every nc-th slot from c, nc = ceil(L / C)) visit every slot of every
//      non-empty window exactly once, windows in order, at most C slots a
//      chunk, and the walk ends with the empty descriptor;
//   3. the degridding's clamped tap block (tap_corner) holds exactly the
//      footprint's cells inside the tile: for every start a0 in
//      [-(W - 1), T - 1] and W = 2..7, the taps i of the block at
//      corner + i with 0 <= i + corner - a0 < W are the columns of
//      [a0, a0 + W) inside [0, T), each once, and the block stays inside.
// Prints "ok" and exits 0, or the first failure and exits 1.
#include "grid_win.cuh"

#include <cstdio>
#include <random>
#include <vector>

using namespace pc;

int main() {
  std::mt19937 rng(12345);
  // 1. part ranges
  for (int trial = 0; trial < 2000; ++trial) {
    const int bs = (int)(rng() % 100000), len = (int)(rng() % 70000);
    const int parts = 1 + (int)(rng() % 40);
    int next = bs;
    for (int k = 0; k < parts; ++k) {
      const int2 r = gwin::part_range(bs, bs + len, k, parts);
      if (r.x != next || r.y < 0) {
        std::printf("part_range: part %d of %d of [%d, %d) starts at %d, expected %d\n", k, parts, bs, bs + len,
                    r.x, next);
        return 1;
      }
      next = r.x + r.y;
    }
    if (next != bs + len) {
      std::printf("part_range: parts of [%d, %d) end at %d\n", bs, bs + len, next);
      return 1;
    }
  }
  // 2. chunk walk over random window runs (some empty)
  for (int trial = 0; trial < 500; ++trial) {
    const int Pw = 1 + (int)(rng() % 20);
    std::vector<int2> wr(Pw);
    int pos = (int)(rng() % 1000);
    for (int j = 0; j < Pw; ++j) {
      const int L = (rng() % 4 == 0) ? 0 : (int)(rng() % 2000);
      wr[j] = make_int2(pos, L);
      pos += L + (int)(rng() % 5);
    }
    std::vector<int> seen(pos + 1, 0);
    int4 d = make_int4(-1, 0, 1, 0);
    for (int j = 0; j < Pw; ++j)
      if (wr[j].y > 0) {
        d = gwin::chunk_at(wr.data(), j, 0);
        break;
      }
    int last_j = -1, steps = 0;
    while (d.x >= 0) {
      if (d.x < last_j || d.w > gwin::C || d.w <= 0 || ++steps > 100000) {
        std::printf("chunk walk: bad descriptor {%d, %d, %d, %d}\n", d.x, d.y, d.z, d.w);
        return 1;
      }
      last_j = d.x;
      for (int i = 0; i < d.w; ++i) {
        const int sl = d.y + i * d.z;
        if (sl < wr[d.x].x || sl >= wr[d.x].x + wr[d.x].y) {
          std::printf("chunk walk: slot %d outside window %d\n", sl, d.x);
          return 1;
        }
        seen[sl] += 1;
      }
      d = gwin::chunk_after(wr.data(), Pw, d);
    }
    for (int j = 0; j < Pw; ++j)
      for (int sl = wr[j].x; sl < wr[j].x + wr[j].y; ++sl)
        if (seen[sl] != 1) {
          std::printf("chunk walk: slot %d of window %d visited %d times\n", sl, j, seen[sl]);
          return 1;
        }
  }
  // 3. the clamped tap block
  for (int W = 2; W <= 7; ++W)
    for (int a0 = -(W - 1); a0 <= gwin::T - 1; ++a0) {
      const int c = gwin::tap_corner(a0, W);
      if (c < 0 || c + W > gwin::T) {
        std::printf("tap_corner(%d, %d) = %d leaves the tile\n", a0, W, c);
        return 1;
      }
      std::vector<int> hit(gwin::T, 0);
      for (int i = 0; i < W; ++i) {
        const int own = i + c - a0;          // the footprint's tap index of block tap i
        if (own >= 0 && own < W) hit[c + i] += 1;
      }
      for (int a = 0; a < gwin::T; ++a) {
        const int want = (a >= a0 && a < a0 + W) ? 1 : 0;
        if (hit[a] != want) {
          std::printf("tap block of a0 = %d, W = %d: column %d taken %d times, expected %d\n", a0, W, a, hit[a],
                      want);
          return 1;
        }
      }
    }
  std::printf("ok\n");
  return 0;
}
