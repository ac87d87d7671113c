// Host check of the x-face trace columns (csrc/xface_layout.h, the functions
// the trace, fused and stage kernels call): for meshes of n_x elements along
// x and nr rows, and lane groups of E, every face the trace kernel stores
// (x_pair_on_chip false) gets a column of its own on its side, below the row
// pitch (a multiple of 32 at least the element count), and every face the
// fused kernel reads from memory is found at the column its writer used.
// Prints "ok" or the first violation.
#include <cstdio>
#include <map>

#include "xface_layout.h"

using acmhd::x_col;
using acmhd::x_compact_mode;
using acmhd::x_pair_on_chip;

static int check(int nx, int nr, int E) {
  const int ne = nx * nr;
  const size_t stride = (size_t)((ne + 31) / 32 * 32);
  const int mode = x_compact_mode(nx, E);
  std::map<size_t, int> owner[2];
  for (int e = 0; e < ne; ++e) {
    const int ex = e % nx, row = e / nx;
    const int left = row * nx + (ex + nx - 1) % nx, right = row * nx + (ex + 1) % nx;
    for (int hi = 0; hi < 2; ++hi) {
      const bool stored = hi ? !x_pair_on_chip(e, right, E) : !x_pair_on_chip(left, e, E);
      if (!stored) continue;
      const size_t c = x_col(e, E, mode, hi != 0);
      if (c >= stride) {
        std::printf("nx=%d nr=%d E=%d: e=%d side %d column %zu >= pitch %zu\n", nx, nr, E, e,
                    hi, c, stride);
        return 1;
      }
      if (owner[hi].count(c)) {
        std::printf("nx=%d nr=%d E=%d: e=%d and e=%d share column %zu on side %d\n", nx, nr, E,
                    e, owner[hi][c], c, hi);
        return 1;
      }
      owner[hi][c] = e;
    }
  }
  for (int e = 0; e < ne; ++e) {
    const int ex = e % nx, row = e / nx;
    const int left = row * nx + (ex + nx - 1) % nx, right = row * nx + (ex + 1) % nx;
    if (!x_pair_on_chip(left, e, E)) {
      const size_t c = x_col(left, E, mode, true);
      if (!owner[1].count(c) || owner[1][c] != left) {
        std::printf("nx=%d nr=%d E=%d: e=%d reads its left neighbour's face at %zu\n", nx, nr,
                    E, e, c);
        return 1;
      }
    }
    if (!x_pair_on_chip(e, right, E)) {
      const size_t c = x_col(right, E, mode, false);
      if (!owner[0].count(c) || owner[0][c] != right) {
        std::printf("nx=%d nr=%d E=%d: e=%d reads its right neighbour's face at %zu\n", nx, nr,
                    E, e, c);
        return 1;
      }
    }
  }
  return 0;
}

int main() {
  const int Es[] = {4, 8, 16, 32};
  for (int E : Es)
    for (int nx = 1; nx <= 200; ++nx)
      for (int nr = 1; nr <= 5; ++nr)
        if (check(nx, nr, E)) return 1;
  std::printf("ok\n");
  return 0;
}
