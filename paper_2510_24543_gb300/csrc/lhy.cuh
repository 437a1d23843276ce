// Lee-Huang-Yang terms of the binary dipolar eGPE, evaluated per grid point
// over a Gauss-Legendre rule on u in [0,1] (Eq. 1 LHY term, Sec. II branch
// potentials and mu_LHY, Sec. V second variations).
//
// At node u: eta_ij = g_ij + gdd_ij (3u^2 - 1), delta = eta11 n1 - eta22 n2,
// s = sqrt(delta^2 + 4 eta12 eta21 n1 n2), V_+- = eta11 n1 + eta22 n2 +- s.
// Negative V contributes max(V,0)^{5/2}; where s = 0 every term divided by s
// is 0 (the two branches coincide there).  One rsqrt gives both s and 1/s.
#pragma once
#include "common.cuh"

namespace egpe {

__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }

// Smallest s^2 treated as nonzero (below it the rsqrt of the field precision
// would overflow or lose its meaning).
template <class R> __device__ __forceinline__ R s2_min();
template <> __device__ __forceinline__ double s2_min<double>() { return 1e-300; }
template <> __device__ __forceinline__ float s2_min<float>() { return 1e-36f; }

// F = sum_q w_q sum_+- max(V,0)^{5/2};  mu_i = dF/dn_i
//   = sum_q w_q (5/2) sum_+- max(V,0)^{3/2} (eta_ii +- sigma_i/s),
// sigma_1 = eta11 delta + 2 eta12 eta21 n2, sigma_2 = -eta22 delta + 2 eta12 eta21 n1.
// The weights already include kappa eta_s^{-5/2}.
template <class R>
__device__ __forceinline__ void lhy_point(const LhyNode<R>* __restrict__ nd, int Q, R n1, R n2, R& F, R& mu1,
                                          R& mu2) {
  R f = 0, m1 = 0, m2 = 0;
  for (int q = 0; q < Q; ++q) {
    const R e11 = nd[q].e11, e22 = nd[q].e22, e2 = nd[q].e2, w = nd[q].w;
    const R a1 = e11 * n1, a2 = e22 * n2;
    const R A = a1 + a2, d = a1 - a2;
    const R s2 = d * d + R(2) * e2 * n1 * n2;
    R rs = 0, s = 0;
    if (s2 > s2_min<R>()) {
      rs = rsqrt_(s2);
      s = s2 * rs;
    }
    const R vp = A + s, vm = A - s;
    R p32 = 0, m32 = 0, p52 = 0, m52 = 0;
    if (vp > R(0)) {
      const R sq = sqrt_(vp);
      p32 = vp * sq;
      p52 = vp * p32;
    }
    if (vm > R(0)) {
      const R sq = sqrt_(vm);
      m32 = vm * sq;
      m52 = vm * m32;
    }
    f += w * (p52 + m52);
    const R sum32 = p32 + m32, dif32 = p32 - m32;
    const R q1 = (e11 * d + e2 * n2) * rs;
    const R q2 = (e2 * n1 - e22 * d) * rs;
    m1 += w * (e11 * sum32 + q1 * dif32);
    m2 += w * (e22 * sum32 + q2 * dif32);
  }
  F = f;
  mu1 = R(2.5) * m1;
  mu2 = R(2.5) * m2;
}

// Second variation of F along n(alpha) with first variations n1', n2' and the
// second variations n'' removed (they enter through mu_LHY, see the line-search
// assembly):  sum_q w_q (5/2) sum_+- [ 2 max(V,0)^{3/2} K_+- + (3/2) max(V,0)^{1/2} (V1_+-)^2 ],
// V1_+- = eta11 n1' + eta22 n2' +- t1,  t1 = (delta delta1 + 2 eta12 eta21 (n1 n2' + n1' n2))/s,
// K_+- = +-(delta1^2 + 4 eta12 eta21 n1' n2' - t1^2)/(2s),  delta1 = eta11 n1' - eta22 n2'
// (the n''-free part of the paper's V^2_+-, Sec. V auxiliaries).
template <class R>
__device__ __forceinline__ R lhy_hess(const LhyNode<R>* __restrict__ nd, int Q, R n1, R n2, R n1p, R n2p) {
  R h = 0;
  for (int q = 0; q < Q; ++q) {
    const R e11 = nd[q].e11, e22 = nd[q].e22, e2 = nd[q].e2, w = nd[q].w;
    const R a1 = e11 * n1, a2 = e22 * n2;
    const R A = a1 + a2, d = a1 - a2;
    const R s2 = d * d + R(2) * e2 * n1 * n2;
    R rs = 0, s = 0;
    if (s2 > s2_min<R>()) {
      rs = rsqrt_(s2);
      s = s2 * rs;
    }
    const R d1 = e11 * n1p - e22 * n2p;
    const R A1 = e11 * n1p + e22 * n2p;
    const R t1 = (d * d1 + e2 * (n1 * n2p + n1p * n2)) * rs;
    const R K = (d1 * d1 + R(2) * e2 * n1p * n2p - t1 * t1) * R(0.5) * rs;
    const R vp = A + s, vm = A - s;
    R acc = 0;
    if (vp > R(0)) {
      const R sq = sqrt_(vp);
      const R v1 = A1 + t1;
      acc += R(2) * vp * sq * K + R(1.5) * sq * v1 * v1;
    }
    if (vm > R(0)) {
      const R sq = sqrt_(vm);
      const R v1 = A1 - t1;
      acc += R(-2) * vm * sq * K + R(1.5) * sq * v1 * v1;
    }
    h += w * acc;
  }
  return R(2.5) * h;
}

}  // namespace egpe
