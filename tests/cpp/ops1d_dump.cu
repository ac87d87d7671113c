// Host program: prints the library's FP64 1-D operator tables (build_ops1d)
// and degree projectors (degree_projector) for p = 1..6, DG and g2, as one
// JSON object, for tests/test_ops1d_host.py to compare with the oracle.  No
// CUDA call is made, so it runs without a GPU.
#include <cstdio>

#include "fr_internal.h"

using acmhd::kMaxM;
using acmhd::Ops1D;

static void vec(const double* v, int m) {
  std::printf("[");
  for (int i = 0; i < m; ++i) std::printf("%s%.17e", i ? "," : "", v[i]);
  std::printf("]");
}

static void mat(const double (*a)[kMaxM], int m) {
  std::printf("[");
  for (int i = 0; i < m; ++i) {
    std::printf("%s", i ? "," : "");
    vec(a[i], m);
  }
  std::printf("]");
}

int main() {
  std::printf("{");
  bool first = true;
  for (int corr = 0; corr < 2; ++corr) {
    for (int order = 1; order <= 6; ++order) {
      Ops1D o;
      if (!acmhd::build_ops1d(order, corr == 0 ? FR_CORR_DG : FR_CORR_G2, &o)) return 1;
      const int m = o.m;
      std::printf("%s\"%s%d\":{", first ? "" : ",", corr == 0 ? "dg" : "g2", order);
      first = false;
      std::printf("\"xi\":");
      vec(o.xi, m);
      std::printf(",\"w\":");
      vec(o.w, m);
      std::printf(",\"D\":");
      mat(o.D, m);
      std::printf(",\"lm\":");
      vec(o.lm, m);
      std::printf(",\"lp\":");
      vec(o.lp, m);
      std::printf(",\"dhl\":");
      vec(o.dhl, m);
      std::printf(",\"dhr\":");
      vec(o.dhr, m);
      std::printf(",\"Dt\":");
      mat(o.Dt, m);
      std::printf(",\"proj\":[");
      for (int q = 0; q <= order; ++q) {
        double P[kMaxM][kMaxM];
        acmhd::degree_projector(o, q, P);
        std::printf("%s", q ? "," : "");
        mat(P, m);
      }
      std::printf("]}");
    }
  }
  std::printf("}\n");
  return 0;
}
