// Where the trace buffer keeps the x-face traces (no CUDA types, so that a
// host test can compile it: tests/cpp/xface_layout_test.cpp).
//
// x-face exchange between lanes.  The fused kernel keeps E consecutive
// elements in E consecutive lanes, so the left x-neighbour of element e is
// the previous lane whenever both sit in the same group of E.  Its trace is
// then taken from that lane with a shuffle instead of from memory, and the
// trace kernel does not store it.  Both kernels decide with x_pair_on_chip.
//
// Column of a stored x-face trace (x_col).  Only elements whose x-neighbour
// on that side lies outside their lane group store the face: the group's
// first element (low face), its last (high face), and where a row of n_x
// elements starts or ends inside the group, that element.  Stored by group,
// the values that neighbouring CTAs read share sectors instead of each
// taking a sector of its own:
//  xcompact = 1 (n_x a multiple of E: rows are whole groups): column g;
//  xcompact = 2 (n_x > E otherwise: at most one row boundary inside a
//    group): columns 2g (the group's own end) and 2g + 1 (the row boundary);
//  xcompact = 0 (n_x < E): the element index, the layout of the y and z faces.
// hi: the high face (side 1) of element e, else the low face.
#pragma once

#include <cstddef>

#if defined(__CUDACC__)
#define ACMHD_HD __host__ __device__ __forceinline__
#else
#define ACMHD_HD inline
#endif

namespace acmhd {

ACMHD_HD bool x_pair_on_chip(int e_left, int e_right, int E) {
  return e_right == e_left + 1 && (e_right % E) != 0;
}

// the xcompact mode of a mesh with n_x elements along x and E per lane group
ACMHD_HD int x_compact_mode(int nx, int E) {
  return (E <= 0 || nx < E) ? 0 : (nx % E == 0 ? 1 : 2);
}

ACMHD_HD size_t x_col(int e, int E, int xcompact, bool hi) {
  if (xcompact == 0) return (size_t)e;
  if (xcompact == 1) return (size_t)(e / E);
  const int inside = hi ? ((e + 1) % E != 0) : (e % E != 0);
  return (size_t)(2 * (e / E) + inside);
}

}  // namespace acmhd

#undef ACMHD_HD
