// Host-side check of the one-CTA FFT's shared-memory staging map
// (cfft::stage_mask / stage_pos in fft_cta.cuh), using the kernels' own lane
// mappings (cfft::freq, cfft::kept_freq): for G = 512 R, R = 4, 8, 16
//   1. stage_pos is a bijection of [0, G) that keeps every aligned group of R;
//   2. a lane's mask is the same for all its outputs (the kernels compute it
//      once per lane);
//   3. the stores of every warp instruction put the 16 lanes of each
//      half-warp on 16 different eight-byte bank pairs (no conflicts), for
//      the full-row staging (all 16 registers) and the kept outputs folded
//      into [0, G / 2);
//   4. runs of 16 consecutive frequencies read back from 16 different bank
//      pairs when they start on a multiple of 16.
// Prints "ok" and exits 0, or prints the first failure and exits 1.
#include "fft_cta.cuh"

#include <cstdio>
#include <set>
#include <vector>

using namespace pc;

template <int R>
static bool check() {
  constexpr int G = cfft::Cfg<R>::G;
  std::vector<int> seen(G, 0);
  for (int k = 0; k < G; ++k) {
    const int a = cfft::stage_pos<R, 8>(k), b = cfft::stage_pos<R, 7>(k);
    if (a < 0 || a >= G || a / R != k / R || b / R != k / R) {
      std::printf("R=%d: k=%d leaves its group\n", R, k);
      return false;
    }
    seen[a] += 1;
  }
  for (int k = 0; k < G; ++k)
    if (seen[k] != 1) {
      std::printf("R=%d: stage_pos is not a bijection at %d\n", R, k);
      return false;
    }
  auto fold = [](int k) { return k < G / 2 ? k : k - G / 2; };
  for (int k1 = 0; k1 < R; ++k1) {
    for (int half = 0; half < 2; ++half) {
      // full-row staging (degridding passes): every register kp
      for (int kp = 0; kp < cfft::L; ++kp) {
        std::set<int> banks;
        for (int lane = 16 * half; lane < 16 * half + 16; ++lane) {
          const int k = cfft::freq<R>(k1, lane, kp);
          const int m = cfft::stage_mask<R, 8>(cfft::freq<R>(k1, lane, 0));
          if (cfft::stage_mask<R, 8>(k) != m) {
            std::printf("R=%d: full-row mask varies over kp (lane %d)\n", R, lane);
            return false;
          }
          banks.insert((k ^ m) & 15);
        }
        if (banks.size() != 16) {
          std::printf("R=%d: full-row stores conflict (k1=%d kp=%d)\n", R, k1, kp);
          return false;
        }
      }
      // kept outputs folded into [0, G / 2) (certificate row pass)
      for (int c = 0; c < 8; ++c) {
        std::set<int> banks;
        for (int lane = 16 * half; lane < 16 * half + 16; ++lane) {
          const int k = fold(cfft::kept_freq<R>(k1, lane, c));
          const int m = cfft::stage_mask<R, 7>(fold(cfft::kept_freq<R>(k1, lane, 0)));
          if (cfft::stage_mask<R, 7>(k) != m) {
            std::printf("R=%d: kept mask varies over c (lane %d)\n", R, lane);
            return false;
          }
          banks.insert((k ^ m) & 15);
        }
        if (banks.size() != 16) {
          std::printf("R=%d: kept stores conflict (k1=%d c=%d)\n", R, k1, c);
          return false;
        }
      }
    }
  }
  for (int k0 = 0; k0 < G; k0 += 16) {
    std::set<int> a, b;
    for (int k = k0; k < k0 + 16; ++k) {
      a.insert(cfft::stage_pos<R, 8>(k) & 15);
      b.insert(cfft::stage_pos<R, 7>(k) & 15);
    }
    if (a.size() != 16 || b.size() != 16) {
      std::printf("R=%d: read-back run at %d conflicts\n", R, k0);
      return false;
    }
  }
  return true;
}

int main() {
  if (!check<4>() || !check<8>() || !check<16>()) return 1;
  std::printf("ok\n");
  return 0;
}
