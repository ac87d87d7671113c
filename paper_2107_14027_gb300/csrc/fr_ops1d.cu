// Host FP64 construction of the 1-D FR operators (Sec. 2.1, FR divergence
// equation; Table fr_adv, stage 3 grouping).
//
// Gauss-Legendre nodes by Newton's method on P_m, weights 2/((1-x^2) P_m'^2);
// Lagrange basis by the barycentric formula; correction functions from
// Legendre derivatives: the DG choice h_l = right Radau polynomial
// R_{R,m} = ((-1)^m / 2)(P_m - P_{m-1}) and Huynh's g2 choice
// h_l = ((m-1) R_{R,m} + m R_{R,m-1}) / (2m - 1); h_r(x) = h_l(-x).
#include <cmath>

#include "fr_internal.h"

namespace acmhd {
namespace {

// P_n(x) and P_n'(x)
void legendre_pd(int n, double x, double* p, double* dp) {
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    // derivative recurrence: P_k' = P_{k-2}' + (2k - 1) P_{k-1}
    double d2 = d0 + (2.0 * k - 1.0) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *p = p1;
  *dp = d1;
}

// derivative of the right Radau polynomial of degree k at x
double radau_right_d(int k, double x) {
  double pk, dpk, pk1, dpk1;
  legendre_pd(k, x, &pk, &dpk);
  legendre_pd(k - 1, x, &pk1, &dpk1);
  double s = (k % 2 == 0) ? 0.5 : -0.5;
  return s * (dpk - dpk1);
}

double corr_left_d(int correction, int m, double x) {
  if (correction == FR_CORR_DG) return radau_right_d(m, x);
  double ca = (m - 1.0) / (2.0 * m - 1.0), cb = m / (2.0 * m - 1.0);
  return ca * radau_right_d(m, x) + cb * radau_right_d(m - 1, x);
}

}  // namespace

void degree_projector(const Ops1D& o, int q, double (*P)[kMaxM]) {
  // P[i][k] = sum_{n <= q} phi_n(x_i) phi_n(x_k) w_k, phi_n = sqrt((2n+1)/2) P_n
  for (int i = 0; i < o.m; ++i)
    for (int k = 0; k < o.m; ++k) {
      double acc = 0.0;
      for (int n = 0; n <= q; ++n) {
        double pi, pk, d;
        legendre_pd(n, o.xi[i], &pi, &d);
        legendre_pd(n, o.xi[k], &pk, &d);
        acc += (2.0 * n + 1.0) / 2.0 * pi * pk * o.w[k];
      }
      P[i][k] = acc;
    }
}

bool build_ops1d(int order, int correction, Ops1D* o) {
  const int m = order + 1;
  if (m < 2 || m > kMaxM) return false;
  if (correction != FR_CORR_DG && correction != FR_CORR_G2) return false;
  o->m = m;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < m; ++i) {
    // i-th node counted from the right, then stored ascending
    double x = std::cos(pi * (i + 0.75) / (m + 0.5));
    for (int it = 0; it < 64; ++it) {
      double p, dp;
      legendre_pd(m, x, &p, &dp);
      double dx = p / dp;
      x -= dx;
      if (std::fabs(dx) <= 1e-17) break;
    }
    double p, dp;
    legendre_pd(m, x, &p, &dp);
    o->xi[m - 1 - i] = x;
    o->w[m - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  // barycentric weights
  double bw[kMaxM];
  for (int k = 0; k < m; ++k) {
    double prod = 1.0;
    for (int q = 0; q < m; ++q)
      if (q != k) prod *= (o->xi[k] - o->xi[q]);
    bw[k] = 1.0 / prod;
  }
  // derivative matrix D[i][k] = l_k'(xi_i)
  for (int i = 0; i < m; ++i) {
    double diag = 0.0;
    for (int k = 0; k < m; ++k) {
      if (k == i) continue;
      o->D[i][k] = (bw[k] / bw[i]) / (o->xi[i] - o->xi[k]);
      diag -= o->D[i][k];
    }
    o->D[i][i] = diag;
  }
  // end values l_k(-1), l_k(+1) (the ends are never nodes)
  for (int side = 0; side < 2; ++side) {
    double x = side ? 1.0 : -1.0;
    double den = 0.0, num[kMaxM];
    for (int k = 0; k < m; ++k) {
      num[k] = bw[k] / (x - o->xi[k]);
      den += num[k];
    }
    for (int k = 0; k < m; ++k) (side ? o->lp : o->lm)[k] = num[k] / den;
  }
  for (int i = 0; i < m; ++i) {
    o->dhl[i] = corr_left_d(correction, m, o->xi[i]);
    o->dhr[i] = -corr_left_d(correction, m, -o->xi[i]);
  }
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < m; ++k)
      o->Dt[i][k] = o->D[i][k] - o->dhl[i] * o->lm[k] - o->dhr[i] * o->lp[k];
  return true;
}

}  // namespace acmhd
