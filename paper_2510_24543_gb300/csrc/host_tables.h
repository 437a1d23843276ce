// Host-side constant tables shared by every engine and by the allocation-free
// entry point: FFT twiddles, the Gauss-Legendre rule of the LHY u-integral
// with its per-node constants (Eq. 1 LHY term, Sec. II branch potentials), and
// the per-instance threshold below which the FP64 kernels drop LHY terms.
// Everything is computed in long double and rounded once to field precision.
#pragma once
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "egpe.h"

namespace egpe {

// W_L^m = exp(-2 pi i m / L), m = 0..L-1.
template <class R> inline void twiddle_table(int L, C2<R>* out) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int m = 0; m < L; ++m) {
    const long double ang = 2.0L * pi * (long double)m / (long double)L;
    out[m] = cmk<C2<R>>((R)cosl(ang), (R)(-sinl(ang)));
  }
}

// Legendre polynomial P_Q(x) and its predecessor P_{Q-1}(x) by the three-term
// recurrence (P_0 = 1, P_1 = x).
inline void legendre_pq(int Q, long double x, long double& pq, long double& pq1) {
  long double p0 = 1.0L, p1 = x;
  for (int k = 2; k <= Q; ++k) {
    const long double p2 = ((2.0L * k - 1.0L) * x * p1 - (k - 1.0L) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  pq = p1;
  pq1 = p0;
}

// Q-point Gauss-Legendre rule mapped to [0,1]: the roots of P_Q by Newton
// iteration from the usual cosine guesses, weights 2/((1 - x^2) P_Q'(x)^2),
// both halved by the map from [-1,1].
inline void gauss_legendre01(int Q, std::vector<long double>& u, std::vector<long double>& w) {
  u.resize(Q);
  w.resize(Q);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < Q; ++i) {
    long double x = cosl(pi * (i + 0.75L) / (Q + 0.5L));
    long double pq, pq1, dp = 1.0L;
    for (int it = 0; it < 100; ++it) {
      legendre_pq(Q, x, pq, pq1);
      dp = Q * (x * pq - pq1) / (x * x - 1.0L);
      const long double dx = pq / dp;
      x -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    legendre_pq(Q, x, pq, pq1);
    dp = Q * (x * pq - pq1) / (x * x - 1.0L);
    u[i] = 0.5L * (1.0L + x);
    w[i] = 1.0L / ((1.0L - x * x) * dp * dp);
  }
}

// Node constants of the LHY u-integral for the couplings p (Q = p.lhy_nodes
// entries written to out), with the nodes whose det eta(u_q) > 0 first; returns
// their count.  W carries kappa eta_s^{-5/2} times the quadrature weight.
template <class R> inline int lhy_node_table(const egpe_params& p, LhyNode<R>* out) {
  const int Q = p.lhy_nodes;
  std::vector<long double> u, w;
  gauss_legendre01(Q, u, w);
  const long double c5 = (long double)p.lhy_kappa * powl((long double)p.lhy_eta_scale, -2.5L);
  std::vector<LhyNode<R>> pos, neg;
  for (int q = 0; q < Q; ++q) {
    const long double s = 3.0L * u[q] * u[q] - 1.0L;
    const long double e12 = p.g[0][1] + p.gdd[0][1] * s;
    const long double det = (p.g[0][0] + p.gdd[0][0] * s) * (p.g[1][1] + p.gdd[1][1] * s) - e12 * e12;
    LhyNode<R> nd;
    nd.w = (R)s;
    nd.W = (R)(c5 * w[q]);
    nd.Ww = (R)(c5 * w[q] * s);
    nd.e12sq = (R)(e12 * e12);
    nd.gq = (R)(det > 0.0L ? 2.0L * sqrtl(det) : 0.0L);
    nd.Www = (R)(c5 * w[q] * s * s);
    nd.pad0 = nd.pad1 = (R)0;
    (det > 0.0L ? pos : neg).push_back(nd);
  }
  const int Qm = (int)pos.size();
  std::copy(pos.begin(), pos.end(), out);
  std::copy(neg.begin(), neg.end(), out + Qm);
  return Qm;
}

// Density below which a point's LHY terms are dropped by the FP64 kernels.
// With eb = max over u of |eta11| + |eta22| + |eta12| every branch potential
// obeys V <= 2 eb n (n = n1 + n2), so F <= 2 c5 (2 eb n)^{5/2} and
// mu_LHY <= 15 c5 eb (2 eb n)^{3/2}; below the threshold these are under 1e-40
// and 1e-30.  eta is affine in w = 3u^2 - 1, so the maximum over u in [0,1]
// sits at w = -1 or w = 2.
inline double lhy_skip_threshold(const egpe_params& p) {
  double eb = 0.0;
  for (double w : {-1.0, 2.0})
    eb = std::max(eb, std::fabs(p.g[0][0] + p.gdd[0][0] * w) + std::fabs(p.g[1][1] + p.gdd[1][1] * w) +
                          std::fabs(p.g[0][1] + p.gdd[0][1] * w));
  const double c5a = std::fabs(p.lhy_kappa * std::pow(p.lhy_eta_scale, -2.5));
  double ns = 1e30;
  if (c5a > 0.0 && eb > 0.0) {
    const double nf = std::pow(1e-40 / (2.0 * c5a), 0.4) / (2.0 * eb);
    const double nm = std::pow(1e-30 / (15.0 * c5a * eb), 2.0 / 3.0) / (2.0 * eb);
    ns = std::min(nf, nm);
  }
  return std::min(ns, 1e30);
}

}  // namespace egpe
