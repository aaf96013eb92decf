// Host check of the window enumeration used by the contribution kernels
// (Eq. tDxx windows): window_split, window_outside_point, divmod_small.
// Prints "ok" and exits 0, or prints the first mismatch and exits 1.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2208_06097_gb300/csrc/sea_internal.cuh"

static unsigned long long rng_state = 0x9E3779B97F4A7C15ULL;
static int rnd(int lo, int hi) {  // uniform in [lo, hi]
  rng_state = rng_state * 6364136223846793005ULL + 1442695040888963407ULL;
  return lo + (int)((rng_state >> 33) % (unsigned long long)(hi - lo + 1));
}

int main() {
  // divmod_small: exhaustive in a for a set of divisors
  const int ds[] = {1, 2, 3, 5, 7, 13, 26, 96, 97, 255, 1000, 4097, 65535, 1 << 20, (1 << 23) - 1,
                    (1 << 23) + 1, (1 << 24) - 1};
  for (int d : ds)
    for (int a = 0; a < (1 << 24); a += (d < 64 ? 1 : 3)) {
      int r;
      const int q = sea::divmod_small(a, d, &r);
      if (q != a / d || r != a % d) {
        printf("divmod %d / %d: %d r %d\n", a, d, q, r);
        return 1;
      }
    }
  // window_split / window_outside_point against brute force
  for (int it = 0; it < 20000; ++it) {
    Entry e{};
    PairInfo P{};
    for (int a = 0; a < 3; ++a) {
      e.wl[a] = rnd(1, 12);
      e.ws[a] = rnd(-20, 20);
      P.ext[a] = rnd(1, 14);
      // pair box near, inside, around or away from the window
      P.lo[a] = e.ws[a] + rnd(-P.ext[a] - 3, e.wl[a] + 2);
    }
    const sea::WinSplit s = sea::window_split(e, P);
    const int wx = e.wl[0], wy = e.wl[1], wz = e.wl[2], nw = wx * wy * wz;
    std::vector<char> inside(nw), seen(nw, 0);
    int n_in = 0;
    for (int z = 0; z < wz; ++z)
      for (int y = 0; y < wy; ++y)
        for (int x = 0; x < wx; ++x) {
          const int lx = e.ws[0] + x - P.lo[0], ly = e.ws[1] + y - P.lo[1], lz = e.ws[2] + z - P.lo[2];
          const bool in = lx >= 0 && lx < P.ext[0] && ly >= 0 && ly < P.ext[1] && lz >= 0 && lz < P.ext[2];
          inside[(z * wy + y) * wx + x] = in;
          n_in += in;
          const bool in_split = x >= s.b0[0] && x < s.b1[0] && y >= s.b0[1] && y < s.b1[1] &&
                                z >= s.b0[2] && z < s.b1[2];
          if (in != in_split) {
            printf("split box disagrees at it %d\n", it);
            return 1;
          }
        }
    if (n_in != s.n_in || nw - n_in != s.n_out) {
      printf("counts at it %d: %d %d against %d %d\n", it, s.n_in, s.n_out, n_in, nw - n_in);
      return 1;
    }
    for (int u = 0; u < s.n_out; ++u) {
      int x, y, z;
      sea::window_outside_point(s, e.wl, u, &x, &y, &z);
      if (x < 0 || x >= wx || y < 0 || y >= wy || z < 0 || z >= wz) {
        printf("outside point %d out of the window at it %d\n", u, it);
        return 1;
      }
      const int t = (z * wy + y) * wx + x;
      if (inside[t] || seen[t]) {
        printf("outside point %d repeated or inside at it %d\n", u, it);
        return 1;
      }
      seen[t] = 1;
    }
  }
  printf("ok\n");
  return 0;
}
