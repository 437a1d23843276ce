// Host-side constant tables shared by every engine and by the allocation-free
// entry point: FFT twiddles, the Gauss-Legendre rule of the LHY u-integral
// with its per-node constants (Eq. 1 LHY term, Sec. II branch potentials), and
// the per-instance threshold below which the FP64 kernels drop LHY terms.
// Everything is computed in long double and rounded once to field precision.
#pragma once
#include <math.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
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
// With `subset`, only those node indices are written (same order rule).
template <class R> inline int lhy_node_table(const egpe_params& p, LhyNode<R>* out,
                                             const std::vector<int>* subset = nullptr) {
  const int Q = p.lhy_nodes;
  std::vector<long double> u, w;
  gauss_legendre01(Q, u, w);
  const long double c5 = (long double)p.lhy_kappa * powl((long double)p.lhy_eta_scale, -2.5L);
  std::vector<int> all;
  if (!subset) {
    for (int q = 0; q < Q; ++q) all.push_back(q);
    subset = &all;
  }
  std::vector<LhyNode<R>> pos, neg;
  for (int q : *subset) {
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

// ---------------------------------------------------------------------------
// Interpolation tables of the LHY chemical potentials and second derivatives.
//
// V_+- are homogeneous of degree 1 in (n1, n2), so each node's term
// W max(V,0)^{5/2} of the LHY density is homogeneous of degree 5/2.  With
// n = n1 + n2 and a = sqrt(min(n1, n2) / n) in [0, 1/sqrt(2)]:
//   mu_LHY,i(n1, n2) = n^{3/2} m_i(a),   d^2 F / dn_i dn_j = n^{1/2} h_ij(a),
// with one set of functions of a per half (half 0: n1 <= n2, half 1:
// n1 > n2).  Summed over the nodes they are tabulated as piecewise
// polynomials: NI equal intervals of a, Chebyshev interpolation in long
// double stored as monomial coefficients in the local coordinate
// x = 2 (a NI sqrt(2) - i) - 1 of interval i.  The FP64 engine's tables have
// degree 11 and are checked to 2e-15; the FP32 engine's have degree 7 (two
// 16-byte loads per function) and are checked to 1e-9, below FP32 rounding.  A node's terms are analytic in
// a on the closed half except for the branch points of
// s = sqrt(delta^2 + 4 eta12^2 n1 n2), which sit at a distance of about
// d = |eta_jj| / (2 |eta12|) from a = 0 (j the majority component); nodes with
// d below four interval widths are left out of the tables and evaluated
// exactly per point.  Each table is then checked against the exact sums at
// the interval ends and midway between the interpolation nodes, and further
// nodes (smallest d first) move to the exact list until every function
// matches to the tolerance of its largest magnitude on that half.
// ---------------------------------------------------------------------------
constexpr int kTabFun = 5;  // mu1, mu2, H11, H12, H22
// Degree and check tolerance of the tables for field type R.
template <class R> struct TabSpec;
template <> struct TabSpec<double> {
  static constexpr int deg = 11;
  static constexpr long double tol = 2e-15L;
};
template <> struct TabSpec<float> {
  static constexpr int deg = 7;
  static constexpr long double tol = 1e-9L;
};

// Node q's contributions (W-weighted) to mu1, mu2, H11, H12, H22 at (n1, n2):
// F_q = W sum_+- max(V_+-,0)^{5/2}, V_+- = A +- s (see lhy.cuh for the
// notation), dV/dn_i = eta_ii +- sigma_i/s, d^2 V/dn_i dn_j = +- d^2 s/dn_i dn_j
// with d^2 s/dn1^2 = (eta11^2 - (sigma1/s)^2)/s, d^2 s/dn2^2 = (eta22^2 -
// (sigma2/s)^2)/s, d^2 s/dn1 dn2 = (2 eta12^2 - eta11 eta22 - sigma1 sigma2/s^2)/s
// (terms / s are 0 where s = 0); then dF/dn_i = (5/2) W V^{3/2} V_i and
// d^2 F/dn_i dn_j = W ((15/4) V^{1/2} V_i V_j + (5/2) V^{3/2} V_ij) per branch.
inline void lhy_node_terms(long double e11, long double e22, long double e12, long double W, long double n1,
                           long double n2, long double (&o)[kTabFun]) {
  const long double d = e11 * n1 - e22 * n2;
  const long double s = sqrtl(d * d + 4.0L * e12 * e12 * n1 * n2);
  const long double A = e11 * n1 + e22 * n2;
  long double q1 = 0, q2 = 0, d11 = 0, d22 = 0, d12 = 0;
  if (s > 0) {
    q1 = (d * e11 + 2.0L * e12 * e12 * n2) / s;
    q2 = (-d * e22 + 2.0L * e12 * e12 * n1) / s;
    d11 = (e11 * e11 - q1 * q1) / s;
    d22 = (e22 * e22 - q2 * q2) / s;
    d12 = (2.0L * e12 * e12 - e11 * e22 - q1 * q2) / s;
  }
  for (int sg = 1; sg >= -1; sg -= 2) {
    const long double V = A + sg * s;
    if (!(V > 0)) continue;
    const long double sv = sqrtl(V), v32 = V * sv;
    const long double V1 = e11 + sg * q1, V2 = e22 + sg * q2;
    o[0] += W * 2.5L * v32 * V1;
    o[1] += W * 2.5L * v32 * V2;
    o[2] += W * (3.75L * sv * V1 * V1 + 2.5L * v32 * sg * d11);
    o[3] += W * (3.75L * sv * V1 * V2 + 2.5L * v32 * sg * d12);
    o[4] += W * (3.75L * sv * V2 * V2 + 2.5L * v32 * sg * d22);
  }
}

struct LhyTableHost {
  int ni = 0;                      // intervals per half; 0: no table (every node exact)
  int deg = 0;                     // polynomial degree (deg + 1 coefficients per function)
  std::vector<long double> coef;   // [half][interval][function][coefficient]
  std::vector<int> exact;          // node indices evaluated exactly per point
};

namespace tab_detail {
struct NodeEta {
  long double e11, e22, e12, W;
};
inline void sums(const std::vector<NodeEta>& nd, const std::vector<char>& use, long double n1, long double n2,
                 long double (&o)[kTabFun]) {
  for (int k = 0; k < kTabFun; ++k) o[k] = 0;
  for (size_t q = 0; q < nd.size(); ++q)
    if (use[q]) lhy_node_terms(nd[q].e11, nd[q].e22, nd[q].e12, nd[q].W, n1, n2, o);
}
inline void point(int half, long double a, long double& n1, long double& n2) {
  const long double m = a * a;
  n1 = half == 0 ? m : 1.0L - m;
  n2 = half == 0 ? 1.0L - m : m;
}
}  // namespace tab_detail

// Builds the tables for NI intervals per half; returns false if the check
// failed for some node set it could still shrink (then `worst` names the half
// whose smallest-d regular node should move to the exact list).
template <int DEG>
inline bool lhy_table_try(const std::vector<tab_detail::NodeEta>& nd, const std::vector<char>& regular, int NI,
                          long double tol, std::vector<long double>& coef, int& worst_half) {
  using namespace tab_detail;
  constexpr int NC = DEG + 1, NR = kTabFun * NC;
  const long double amax = sqrtl(0.5L), h = amax / NI;
  const long double pi = 3.141592653589793238462643383279502884L;
  coef.assign((size_t)2 * NI * NR, 0.0L);
  long double xs[NC], T[NC][NC];
  for (int j = 0; j < NC; ++j) {
    xs[j] = cosl(pi * (j + 0.5L) / NC);
    T[j][0] = 1.0L;
    T[j][1] = xs[j];
    for (int k = 2; k < NC; ++k) T[j][k] = 2.0L * xs[j] * T[j][k - 1] - T[j][k - 2];
  }
  // monomial coefficients of the Chebyshev polynomials: mono[k][m] = [x^m] T_k
  long double mono[NC][NC] = {};
  mono[0][0] = 1.0L;
  mono[1][1] = 1.0L;
  for (int k = 2; k < NC; ++k)
    for (int m = 0; m < NC; ++m)
      mono[k][m] = (m > 0 ? 2.0L * mono[k - 1][m - 1] : 0.0L) - mono[k - 2][m];
  std::vector<char> all(nd.size(), 1);
  bool ok = true;
  long double worst = 0;
  worst_half = 0;
  for (int half = 0; half < 2; ++half) {
    long double scale[kTabFun] = {}, err[kTabFun] = {};
    for (int i = 0; i < NI; ++i) {
      long double f[NC][kTabFun];
      for (int j = 0; j < NC; ++j) {
        long double n1, n2;
        point(half, i * h + (xs[j] + 1.0L) * 0.5L * h, n1, n2);
        sums(nd, regular, n1, n2, f[j]);
      }
      long double* out = &coef[((size_t)half * NI + i) * NR];
      for (int fn = 0; fn < kTabFun; ++fn) {
        long double c[NC];
        for (int k = 0; k < NC; ++k) {
          long double acc = 0;
          for (int j = 0; j < NC; ++j) acc += f[j][fn] * T[j][k];
          c[k] = acc * 2.0L / NC;
        }
        c[0] *= 0.5L;
        for (int m = 0; m < NC; ++m) {
          long double b = 0;
          for (int k = m; k < NC; ++k) b += c[k] * mono[k][m];
          out[fn * NC + m] = b;
        }
      }
      // check at both ends and midway between consecutive interpolation nodes
      for (int j = -1; j < NC; ++j) {
        long double x;
        if (j < 0) x = -1.0L;
        else if (j == NC - 1) x = 1.0L;
        else x = 0.5L * (xs[j] + xs[j + 1]);
        long double n1, n2, ex[kTabFun], full[kTabFun];
        point(half, i * h + (x + 1.0L) * 0.5L * h, n1, n2);
        sums(nd, regular, n1, n2, ex);
        sums(nd, all, n1, n2, full);
        for (int fn = 0; fn < kTabFun; ++fn) {
          long double p = out[fn * NC + DEG];
          for (int m = DEG - 1; m >= 0; --m) p = p * x + out[fn * NC + m];
          err[fn] = std::max(err[fn], fabsl(p - ex[fn]));
          scale[fn] = std::max(scale[fn], fabsl(full[fn]));
        }
      }
    }
    for (int fn = 0; fn < kTabFun; ++fn) {
      const long double r = scale[fn] > 0 ? err[fn] / scale[fn] : 0.0L;
      if (r > tol) ok = false;
      if (r > worst) {
        worst = r;
        worst_half = half;
      }
    }
  }
  return ok;
}

// Tables for the couplings p (NI = 32 or 64 intervals per half, whichever
// leaves fewer nodes to exact evaluation; ties go to 32) for field type R.
template <class R> inline LhyTableHost lhy_interp_table(const egpe_params& p) {
  using namespace tab_detail;
  const int Q = p.lhy_nodes;
  std::vector<long double> u, w;
  gauss_legendre01(Q, u, w);
  const long double c5 = (long double)p.lhy_kappa * powl((long double)p.lhy_eta_scale, -2.5L);
  std::vector<NodeEta> nd(Q);
  std::vector<long double> dist[2];
  for (int q = 0; q < Q; ++q) {
    const long double s = 3.0L * u[q] * u[q] - 1.0L;
    nd[q] = {p.g[0][0] + p.gdd[0][0] * s, p.g[1][1] + p.gdd[1][1] * s, p.g[0][1] + p.gdd[0][1] * s, c5 * w[q]};
    const long double e12 = fabsl(nd[q].e12);
    // half 0 (n1 minor): majority component 2; half 1: component 1
    dist[0].push_back(e12 > 0 ? fabsl(nd[q].e22) / (2.0L * e12) : HUGE_VALL);
    dist[1].push_back(e12 > 0 ? fabsl(nd[q].e11) / (2.0L * e12) : HUGE_VALL);
  }
  LhyTableHost best;
  best.exact.resize(Q + 1);  // worse than any outcome
  for (int NI : {32, 64}) {
    if (best.exact.empty()) break;  // 32 intervals already cover every node
    const long double h = sqrtl(0.5L) / NI;
    std::vector<char> regular(Q, 1);
    for (int q = 0; q < Q; ++q)
      if (dist[0][q] < 4.0L * h || dist[1][q] < 4.0L * h) regular[q] = 0;
    std::vector<long double> coef;
    int half = 0;
    while (true) {
      int nreg = 0;
      for (char r : regular) nreg += r;
      if (nreg == 0) break;
      if (lhy_table_try<TabSpec<R>::deg>(nd, regular, NI, TabSpec<R>::tol, coef, half)) break;
      int qmin = -1;
      for (int q = 0; q < Q; ++q)
        if (regular[q] && (qmin < 0 || dist[half][q] < dist[half][qmin])) qmin = q;
      regular[qmin] = 0;
    }
    std::vector<int> exact;
    for (int q = 0; q < Q; ++q)
      if (!regular[q]) exact.push_back(q);
    if (exact.size() < best.exact.size()) {
      best.exact = exact;
      best.ni = (int)exact.size() == Q ? 0 : NI;
      best.deg = TabSpec<R>::deg;
      best.coef = best.ni ? coef : std::vector<long double>();
    }
  }
  return best;
}

// The tables of one parameter set and field type, built once per process
// (repeated handles share the build); returned by value, so a later eviction
// cannot invalidate a caller's copy.
template <class R> inline LhyTableHost lhy_interp_table_cached(const egpe_params& p) {
  static std::mutex mu;
  static std::map<std::vector<double>, LhyTableHost> memo;
  const std::vector<double> key = {p.g[0][0], p.g[0][1], p.g[1][0], p.g[1][1], p.gdd[0][0], p.gdd[0][1],
                                   p.gdd[1][0], p.gdd[1][1], p.lhy_kappa, p.lhy_eta_scale, (double)p.lhy_nodes};
  std::lock_guard<std::mutex> lock(mu);
  auto it = memo.find(key);
  if (it != memo.end()) return it->second;
  if (memo.size() >= 1024) memo.clear();
  return memo.emplace(key, lhy_interp_table<R>(p)).first->second;
}

}  // namespace egpe
