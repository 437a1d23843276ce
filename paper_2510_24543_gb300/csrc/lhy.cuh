// Lee-Huang-Yang terms of the binary dipolar eGPE, evaluated per grid point
// over a Gauss-Legendre rule on u in [0,1] (Eq. 1 LHY term, Sec. II branch
// potentials and mu_LHY, Sec. V second variations).
//
// At node u, with w = 3u^2 - 1: eta_ij = g_ij + gdd_ij w,
//   A = eta11 n1 + eta22 n2 = A0 + A1 w,  delta = eta11 n1 - eta22 n2 = D0 + D1 w,
//   s = sqrt(delta^2 + 4 eta12^2 n1 n2),  V_+- = A +- s   (eta12 = eta21: the couplings
// are symmetric).  Negative V contributes max(V,0)^{5/2}; where s = 0 every
// term divided by s is 0 (the two branches coincide there).  Because eta is
// linear in w, the per-point coefficients A0, A1, D0, D1 and the polynomial
// coefficients of sigma_i(w) are formed once per point, and the node loop only
// carries what depends on the square roots.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace egpe {

__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }

// Smallest s^2 treated as nonzero (below it the rsqrt of the field precision
// would overflow or lose its meaning).
template <class R> __device__ __forceinline__ R s2_min();
template <> __device__ __forceinline__ double s2_min<double>() { return 1e-300; }
template <> __device__ __forceinline__ float s2_min<float>() { return 1e-36f; }

// sqrt(v) of a clamped v >= 0 without branches.  FP64: the library square
// root; FP32: the translation unit is built with the approximate square root
// (MUFU, a few ulp).
__device__ __forceinline__ double sqrt_pos(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_pos(float v) { return sqrtf(v); }

// 1/s (0 where s^2 is below the threshold) and s = s^2 / s.
template <class R> __device__ __forceinline__ void inv_s(R s2, R& rs, R& s) {
  const R r = rsqrt_(s2 > s2_min<R>() ? s2 : R(1));
  rs = s2 > s2_min<R>() ? r : R(0);
  s = s2 * rs;
}

// 1/s with a tiny offset instead of a branch: where s^2 is 0 the quantities
// multiplied by it, (V+^{3/2} - V-^{3/2}), vanish with it.
template <class R> __device__ __forceinline__ R s2_eps();
template <> __device__ __forceinline__ double s2_eps<double>() { return 1e-300; }
template <> __device__ __forceinline__ float s2_eps<float>() { return 1e-30f; }

// Two FP32 values in one 64-bit register pair, operated on by the packed FP32
// instructions (add/sub/mul/fma .f32x2: both lanes in one issue slot, each
// rounded like its scalar counterpart, denormals flushed like the rest of the
// FP32 path).  The FP32 node loops below are bound by instruction issue and
// evaluate two grid points per instruction with them; square roots, min and
// max stay scalar.
struct f32x2 {
  unsigned long long v;
};
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(f32x2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {  // a b + c
  f32x2 r;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f32x2 rsqrt2(f32x2 a) {
  float x, y;
  upk2(a, x, y);
  return pk2(rsqrtf(x), rsqrtf(y));
}
__device__ __forceinline__ f32x2 max0_2(f32x2 a) {
  float x, y;
  upk2(a, x, y);
  return pk2(fmaxf(x, 0.f), fmaxf(y, 0.f));
}
__device__ __forceinline__ f32x2 min2(f32x2 a, f32x2 b) {
  float x, y, u, v;
  upk2(a, x, y);
  upk2(b, u, v);
  return pk2(fminf(x, u), fminf(y, v));
}

// A quadrature node with every value in both lanes, for the packed loops.
struct __align__(16) LhyNodeP {
  f32x2 w, W, Ww, e12sq, gq, Www, pad0, pad1;
};

// Shared-memory staging of the node table: the LhyNode<R> entries, followed
// for FP32 by the same nodes in packed form (the FP32 node loops read them at
// nd + Q).  The staged table must start on a 16-byte boundary.
template <class R> __host__ __device__ constexpr size_t lhy_stage_bytes(int Q) {
  return (size_t)Q * sizeof(LhyNode<R>) + (std::is_same<R, float>::value ? (size_t)Q * sizeof(LhyNodeP) : 0);
}
template <class R> __device__ __forceinline__ void stage_lhy_nodes(LhyNode<R>* dst, const LhyNode<R>* src, int Q) {
  for (int i = threadIdx.x; i < Q; i += blockDim.x) {
    const LhyNode<R> e = src[i];
    dst[i] = e;
    if constexpr (std::is_same<R, float>::value) {
      LhyNodeP& q = reinterpret_cast<LhyNodeP*>(dst + Q)[i];
      q.w = pk2(e.w, e.w);
      q.W = pk2(e.W, e.W);
      q.Ww = pk2(e.Ww, e.Ww);
      q.e12sq = pk2(e.e12sq, e.e12sq);
      q.gq = pk2(e.gq, e.gq);
      q.Www = pk2(e.Www, e.Www);
      q.pad0 = q.pad1 = pk2(0.f, 0.f);
    }
  }
}

// Per-point coefficients.
template <class R> struct LhyPt {
  R A0, A1, D0, D1, q4;  // q4 = 4 n1 n2
};
template <class R> __device__ __forceinline__ LhyPt<R> lhy_pt(const LhyCoef<R>& c, R n1, R n2) {
  LhyPt<R> p;
  p.A0 = c.g11 * n1 + c.g22 * n2;
  p.A1 = c.d11 * n1 + c.d22 * n2;
  p.D0 = c.g11 * n1 - c.g22 * n2;
  p.D1 = c.d11 * n1 - c.d22 * n2;
  p.q4 = R(4) * n1 * n2;
  return p;
}

// F = sum_q W_q sum_+- max(V,0)^{5/2};  mu_i = dF/dn_i
//   = sum_q W_q (5/2) sum_+- max(V,0)^{3/2} (eta_ii +- sigma_i/s),
// sigma_1 = eta11 delta + 2 eta12^2 n2, sigma_2 = -eta22 delta + 2 eta12^2 n1
// (the paper's mu_LHY, Sec. II).  With S_k = sum W w^k (V+^{3/2} + V-^{3/2}) and
// T_k = sum W w^k (V+^{3/2} - V-^{3/2})/s, and sigma_i(w) quadratic in w:
//   mu_i = 5/2 (g_ii S_0 + gdd_ii S_1 + sigma_i0 T_0 + sigma_i1 T_1 + sigma_i2 T_2).
// W_q already includes kappa eta_s^{-5/2}.  NP points are evaluated together
// (independent dependency chains per node).
template <class R, int NP>
__device__ __forceinline__ void lhy_points(const LhyNode<R>* __restrict__ nd, int Q, int Qm, const LhyCoef<R>& c,
                                           const R (&n1)[NP], const R (&n2)[NP], R (&F)[NP], R (&mu1)[NP],
                                           R (&mu2)[NP]) {
  if constexpr (std::is_same<R, double>::value) {
    // every term below FP64 rounding (see LhyCoef::nskip).  FP64 only: the FP32
    // transforms leave a round-off floor of ~1e-7 in amplitude everywhere, so
    // FP32 densities never fall below the threshold and the test only costs.
    bool any = false;
#pragma unroll
    for (int j = 0; j < NP; ++j) any |= n1[j] + n2[j] > c.nskip;
    if (!any) {
#pragma unroll
      for (int j = 0; j < NP; ++j) F[j] = mu1[j] = mu2[j] = R(0);
      return;
    }
  }
  LhyPt<R> p[NP];
  R S0[NP], S1[NP], T0[NP], T1[NP], T2[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    p[j] = lhy_pt(c, n1[j], n2[j]);
    S0[j] = S1[j] = T0[j] = T1[j] = T2[j] = R(0);
  }
  // nodes [0, Qm): det eta > 0, both branches; [Qm, Q): det eta <= 0, where
  // V+ V- = 4 n1 n2 det(eta) <= 0 makes max(V-, 0) = 0 at every point.  With
  // both branches, one reciprocal square root of V+ gives sqrt(V+) and
  // sqrt(V-) = gq sqrt(n1 n2) / sqrt(V+) (clamped to sqrt(V+)).
  R sq[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) sq[j] = sqrt_pos(n1[j] * n2[j]);
  auto node = [&](const LhyNode<R>& e, auto minus) {
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const R A = p[j].A0 + p[j].A1 * e.w;
      const R d = p[j].D0 + p[j].D1 * e.w;
      const R s2 = d * d + e.e12sq * p[j].q4;
      const R rs = rsqrt_(s2 + s2_eps<R>());
      const R s = s2 * rs;
      const R vp = fmax(A + s, R(0));
      R p32, m32 = R(0);
      if constexpr (decltype(minus)::value) {
        const R rp = rsqrt_(vp + s2_eps<R>());
        const R P1 = vp * rp;
        const R M1 = fmin(e.gq * sq[j] * rp, P1);
        p32 = vp * P1;
        m32 = M1 * M1 * M1;
      } else {
        p32 = vp * sqrt_pos(vp);
      }
      const R sum32 = p32 + m32;
      const R t = (p32 - m32) * rs;
      S0[j] += e.W * sum32;
      S1[j] += e.Ww * sum32;
      T0[j] += e.W * t;
      T1[j] += e.Ww * t;
      T2[j] += e.Www * t;
    }
  };
  if constexpr (std::is_same<R, float>::value) {
    // FP32: one loop over all nodes with both branches (sqrt(V-) as above; the
    // clamp also makes it 0 where V+ is clamped to 0), points j = 2h, 2h + 1 in
    // the two lanes
    static_assert(NP % 2 == 0, "the packed FP32 loop takes points in pairs");
    constexpr int NH = NP / 2;
    const LhyNodeP* np = reinterpret_cast<const LhyNodeP*>(nd + Q);
    f32x2 A0[NH], A1[NH], D0[NH], D1[NH], q4[NH], sq2[NH], s0[NH], s1[NH], t0[NH], t1[NH], t2[NH];
    const f32x2 eps = pk2(s2_eps<float>(), s2_eps<float>()), zero = pk2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      A0[h] = pk2(p[2 * h].A0, p[2 * h + 1].A0);
      A1[h] = pk2(p[2 * h].A1, p[2 * h + 1].A1);
      D0[h] = pk2(p[2 * h].D0, p[2 * h + 1].D0);
      D1[h] = pk2(p[2 * h].D1, p[2 * h + 1].D1);
      q4[h] = pk2(p[2 * h].q4, p[2 * h + 1].q4);
      sq2[h] = pk2(sq[2 * h], sq[2 * h + 1]);
      s0[h] = s1[h] = t0[h] = t1[h] = t2[h] = zero;
    }
#pragma unroll 2
    for (int k = 0; k < Q; ++k) {
      const LhyNodeP e = np[k];
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const f32x2 A = fma2(A1[h], e.w, A0[h]);
        const f32x2 d = fma2(D1[h], e.w, D0[h]);
        const f32x2 s2 = fma2(d, d, mul2(e.e12sq, q4[h]));
        const f32x2 rs = rsqrt2(add2(s2, eps));
        const f32x2 vp = max0_2(fma2(s2, rs, A));
        const f32x2 rp = rsqrt2(add2(vp, eps));
        const f32x2 P1 = mul2(vp, rp);
        const f32x2 M1 = min2(mul2(mul2(e.gq, sq2[h]), rp), P1);
        const f32x2 p32 = mul2(vp, P1), m32 = mul2(mul2(M1, M1), M1);
        const f32x2 sum32 = add2(p32, m32);
        const f32x2 t = mul2(sub2(p32, m32), rs);
        s0[h] = fma2(e.W, sum32, s0[h]);
        s1[h] = fma2(e.Ww, sum32, s1[h]);
        t0[h] = fma2(e.W, t, t0[h]);
        t1[h] = fma2(e.Ww, t, t1[h]);
        t2[h] = fma2(e.Www, t, t2[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      upk2(s0[h], S0[2 * h], S0[2 * h + 1]);
      upk2(s1[h], S1[2 * h], S1[2 * h + 1]);
      upk2(t0[h], T0[2 * h], T0[2 * h + 1]);
      upk2(t1[h], T1[2 * h], T1[2 * h + 1]);
      upk2(t2[h], T2[2 * h], T2[2 * h + 1]);
    }
  } else {
#pragma unroll 2
    for (int k = 0; k < Qm; ++k) node(nd[k], std::true_type{});
#pragma unroll 2
    for (int k = Qm; k < Q; ++k) node(nd[k], std::false_type{});
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    // sigma_1(w) = (g11 + d11 w)(D0 + D1 w) + 2 n2 (g12 + d12 w)^2, sigma_2 likewise
    const R n2x2 = R(2) * n2[j], n1x2 = R(2) * n1[j];
    const R s10 = c.g11 * p[j].D0 + n2x2 * c.g12 * c.g12;
    const R s11 = c.g11 * p[j].D1 + c.d11 * p[j].D0 + R(2) * n2x2 * c.g12 * c.d12;
    const R s12 = c.d11 * p[j].D1 + n2x2 * c.d12 * c.d12;
    const R s20 = -c.g22 * p[j].D0 + n1x2 * c.g12 * c.g12;
    const R s21 = -c.g22 * p[j].D1 - c.d22 * p[j].D0 + R(2) * n1x2 * c.g12 * c.d12;
    const R s22 = -c.d22 * p[j].D1 + n1x2 * c.d12 * c.d12;
    mu1[j] = R(2.5) * (c.g11 * S0[j] + c.d11 * S1[j] + s10 * T0[j] + s11 * T1[j] + s12 * T2[j]);
    mu2[j] = R(2.5) * (c.g22 * S0[j] + c.d22 * S1[j] + s20 * T0[j] + s21 * T1[j] + s22 * T2[j]);
    // V+- are homogeneous of degree 1 in (n1, n2), so F is of degree 5/2 and
    // Euler's theorem gives F = (2/5)(n1 mu1 + n2 mu2) exactly
    F[j] = R(0.4) * (n1[j] * mu1[j] + n2[j] * mu2[j]);
  }
}

// Second variation of F along n(alpha) with first variations n1', n2' and the
// second variations n'' removed (they enter through mu_LHY in the line-search
// assembly):  sum_q W_q (5/2) sum_+- [ 2 max(V,0)^{3/2} K_+- + (3/2) max(V,0)^{1/2} (V1_+-)^2 ],
// V1_+- = eta11 n1' + eta22 n2' +- t1,  t1 = (delta delta1 + 2 eta12^2 (n1 n2' + n1' n2))/s,
// K_+- = +-(delta1^2 + 4 eta12^2 n1' n2' - t1^2)/(2s),  delta1 = eta11 n1' - eta22 n2'
// (the n''-free part of the paper's V^2_+-, Sec. V auxiliaries).  NP points together.
template <class R, int NP>
__device__ __forceinline__ void lhy_hess(const LhyNode<R>* __restrict__ nd, int Q, int Qm, const LhyCoef<R>& c,
                                         const R (&n1)[NP], const R (&n2)[NP], const R (&n1p)[NP],
                                         const R (&n2p)[NP], R (&H)[NP]) {
  if constexpr (std::is_same<R, double>::value) {  // as in lhy_points
    bool any = false;
#pragma unroll
    for (int j = 0; j < NP; ++j) any |= n1[j] + n2[j] > c.nskip;
    if (!any) {
#pragma unroll
      for (int j = 0; j < NP; ++j) H[j] = R(0);
      return;
    }
  }
  LhyPt<R> p[NP];
  R B0[NP], B1[NP], E0[NP], E1[NP], m[NP], mp[NP], h[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    p[j] = lhy_pt(c, n1[j], n2[j]);
    B0[j] = c.g11 * n1p[j] + c.g22 * n2p[j];  // A1(w) = B0 + B1 w
    B1[j] = c.d11 * n1p[j] + c.d22 * n2p[j];
    E0[j] = c.g11 * n1p[j] - c.g22 * n2p[j];  // delta1(w) = E0 + E1 w
    E1[j] = c.d11 * n1p[j] - c.d22 * n2p[j];
    m[j] = R(2) * (n1[j] * n2p[j] + n1p[j] * n2[j]);  // 2 eta12^2 (n1 n2' + n1' n2) = eta12^2 m
    mp[j] = R(4) * n1p[j] * n2p[j];                   // 4 eta12^2 n1' n2' = eta12^2 mp
    h[j] = R(0);
  }
  R sq[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) sq[j] = sqrt_pos(n1[j] * n2[j]);
  auto node = [&](const LhyNode<R>& e, auto minus) {
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const R A = p[j].A0 + p[j].A1 * e.w;
      const R d = p[j].D0 + p[j].D1 * e.w;
      const R s2 = d * d + e.e12sq * p[j].q4;
      R rs, s;
      inv_s(s2, rs, s);
      const R vp = fmax(A + s, R(0));
      R sp, rp = R(0);
      if constexpr (decltype(minus)::value) {
        rp = rsqrt_(vp + s2_eps<R>());  // see lhy_points for sqrt(V-)
        sp = vp * rp;
      } else {
        sp = sqrt_pos(vp);
      }
      const R A1 = B0[j] + B1[j] * e.w;
      const R d1 = E0[j] + E1[j] * e.w;
      const R t1 = (d * d1 + e.e12sq * m[j]) * rs;
      const R K = (d1 * d1 + e.e12sq * mp[j] - t1 * t1) * (R(0.5) * rs);
      const R v1p = A1 + t1;
      R acc = R(2) * K * (vp * sp) + R(1.5) * (sp * v1p * v1p);
      if constexpr (decltype(minus)::value) {
        const R sm = fmin(e.gq * sq[j] * rp, sp);
        const R vm = sm * sm;
        const R v1m = A1 - t1;
        acc += R(-2) * K * (vm * sm) + R(1.5) * (sm * v1m * v1m);
      }
      h[j] += e.W * acc;
    }
  };
  if constexpr (std::is_same<R, float>::value) {
    // FP32: sqrt(V-) from sqrt(V+) as in lhy_points, and the two branches summed
    // in closed form: with P1,M1 = sqrt(V+-), P3,M3 = V+-^{3/2}, V1+- = A1 +- t1,
    //   sum_+- [2 K+- V^{3/2} + 3/2 V^{1/2} V1^2]
    //     = (Q2 - t1^2)/s (P3 - M3) + 3/2 [(P1 + M1)(A1^2 + t1^2) + 2 A1 t1 (P1 - M1)]
    // with K+- = +-(Q2 - t1^2)/(2s), Q2 = delta1^2 + 4 eta12^2 n1' n2'.
    // Points j = 2i, 2i + 1 in the two lanes of the packed instructions.
    static_assert(NP % 2 == 0, "the packed FP32 loop takes points in pairs");
    constexpr int NH = NP / 2;
    const LhyNodeP* np = reinterpret_cast<const LhyNodeP*>(nd + Q);
    f32x2 A0[NH], A1c[NH], D0[NH], D1[NH], q4[NH], sq2[NH], b0[NH], b1[NH], e0[NH], e1[NH], m2[NH], mp2[NH],
        hh[NH];
    const f32x2 eps = pk2(s2_eps<float>(), s2_eps<float>()), c15 = pk2(1.5f, 1.5f);
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const int j0 = 2 * i, j1 = 2 * i + 1;
      A0[i] = pk2(p[j0].A0, p[j1].A0);
      A1c[i] = pk2(p[j0].A1, p[j1].A1);
      D0[i] = pk2(p[j0].D0, p[j1].D0);
      D1[i] = pk2(p[j0].D1, p[j1].D1);
      q4[i] = pk2(p[j0].q4, p[j1].q4);
      sq2[i] = pk2(sq[j0], sq[j1]);
      b0[i] = pk2(B0[j0], B0[j1]);
      b1[i] = pk2(B1[j0], B1[j1]);
      e0[i] = pk2(E0[j0], E0[j1]);
      e1[i] = pk2(E1[j0], E1[j1]);
      m2[i] = pk2(m[j0], m[j1]);
      mp2[i] = pk2(mp[j0], mp[j1]);
      hh[i] = pk2(0.f, 0.f);
    }
#pragma unroll 2
    for (int k = 0; k < Q; ++k) {
      const LhyNodeP e = np[k];
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        const f32x2 A = fma2(A1c[i], e.w, A0[i]);
        const f32x2 d = fma2(D1[i], e.w, D0[i]);
        const f32x2 s2 = fma2(d, d, mul2(e.e12sq, q4[i]));
        const f32x2 rs = rsqrt2(add2(s2, eps));
        const f32x2 vp = max0_2(fma2(s2, rs, A));
        const f32x2 rp = rsqrt2(add2(vp, eps));
        const f32x2 P1 = mul2(vp, rp);
        const f32x2 M1 = min2(mul2(mul2(e.gq, sq2[i]), rp), P1);
        const f32x2 dP3 = sub2(mul2(vp, P1), mul2(mul2(M1, M1), M1));
        const f32x2 a1 = fma2(b1[i], e.w, b0[i]);
        const f32x2 d1 = fma2(e1[i], e.w, e0[i]);
        const f32x2 t1 = mul2(fma2(d, d1, mul2(e.e12sq, m2[i])), rs);
        const f32x2 tt = mul2(t1, t1);
        const f32x2 K2 = mul2(sub2(fma2(d1, d1, mul2(e.e12sq, mp2[i])), tt), rs);
        const f32x2 br = fma2(add2(P1, M1), fma2(a1, a1, tt), mul2(mul2(add2(a1, a1), t1), sub2(P1, M1)));
        hh[i] = fma2(e.W, fma2(c15, br, mul2(K2, dP3)), hh[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < NH; ++i) upk2(hh[i], h[2 * i], h[2 * i + 1]);
  } else {
#pragma unroll 2
    for (int k = 0; k < Qm; ++k) node(nd[k], std::true_type{});
#pragma unroll 2
    for (int k = Qm; k < Q; ++k) node(nd[k], std::false_type{});
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) H[j] = R(2.5) * h[j];
}

// F and its partial derivatives with respect to the entries of
// eta(u) = g + gdd (3u^2 - 1), summed over the u-rule (one point; the
// parameter-derivative pass):  o[0] = F,  o[1..3] = dF/d(g11, g22, g12),
// o[4..6] = dF/d(gdd11, gdd22, gdd12).  With V_+- = A +- s and f_+- =
// (5/2) max(V_+-,0)^{3/2}:  dV_+-/deta11 = n1 +- delta n1/s,
// dV_+-/deta22 = n2 -+ delta n2/s, dV_+-/deta12 = +-4 eta12 n1 n2/s (g12 = g21
// moved together); terms / s are 0 where s = 0.
template <class R>
__device__ __forceinline__ void lhy_eta_sums(const LhyNode<R>* __restrict__ nd, int Q, const LhyCoef<R>& c, R n1,
                                             R n2, R (&o)[7]) {
#pragma unroll
  for (int k = 0; k < 7; ++k) o[k] = R(0);
  if constexpr (std::is_same<R, double>::value)
    if (!(n1 + n2 > c.nskip)) return;
  const LhyPt<R> p = lhy_pt(c, n1, n2);
  for (int q = 0; q < Q; ++q) {
    const LhyNode<R>& e = nd[q];
    const R A = p.A0 + p.A1 * e.w;
    const R d = p.D0 + p.D1 * e.w;
    const R s2 = d * d + e.e12sq * p.q4;
    R rs, s;
    inv_s(s2, rs, s);
    const R e12 = c.g12 + c.d12 * e.w;
    const R vp = fmax(A + s, R(0)), vm = fmax(A - s, R(0));
    const R rp = sqrt_pos(vp), rm = sqrt_pos(vm);
    const R fp = R(2.5) * vp * rp, fm = R(2.5) * vm * rm;
    o[0] += e.W * (vp * vp * rp + vm * vm * rm);
    const R sum = fp + fm, dif = fp - fm;
    const R t11 = sum * n1 + dif * d * n1 * rs;
    const R t22 = sum * n2 - dif * d * n2 * rs;
    const R t12 = dif * R(4) * e12 * n1 * n2 * rs;
    o[1] += e.W * t11;
    o[2] += e.W * t22;
    o[3] += e.W * t12;
    o[4] += e.Ww * t11;
    o[5] += e.Ww * t22;
    o[6] += e.Ww * t12;
  }
}

// ----------------------------------------------------------------------------
// Interpolated LHY terms.  The LHY density is homogeneous of degree 5/2 in
// (n1, n2), so with n = n1 + n2 and a = sqrt(min(n1, n2)/n):
//   mu_LHY,i = n^{3/2} m_i(a),   d^2 F/dn_i dn_j = n^{1/2} h_ij(a),
// where m_i, h_ij are the quadrature sums over the table's nodes, stored per
// half (n1 <= n2, n1 > n2) as polynomials on equal intervals of a (the host
// builds and checks them).  A record holds, per interval, the coefficients of
// m1, m2, h11, h12, h22 in the local coordinate x in [-1,1].
// ----------------------------------------------------------------------------
// Coefficients per function: degree 11 for FP64 fields, degree 7 for FP32.
template <class R> struct LhyTabDim;
template <> struct LhyTabDim<double> {
  static constexpr int coef = 12, rec = 5 * coef;
};
template <> struct LhyTabDim<float> {
  static constexpr int coef = 8, rec = 5 * coef;
};

template <class R> struct LhyTab {
  const R* tab;  // [half][interval][function][coefficient], 16-byte aligned records
  int ni;        // intervals per half (0: no table)
  R tscale;      // ni sqrt(2): a tscale is the interval coordinate
};

// The interval polynomial at x (Horner), coefficients from global memory
// through the read-only path in 16-byte loads: degree 7 in FP32, 11 in FP64.
__device__ __forceinline__ float horner_tab(const float* c, float x) {
  const float4* v = reinterpret_cast<const float4*>(c);
  const float4 a = __ldg(v), b = __ldg(v + 1);
  float p = b.w;
  p = fmaf(p, x, b.z);
  p = fmaf(p, x, b.y);
  p = fmaf(p, x, b.x);
  p = fmaf(p, x, a.w);
  p = fmaf(p, x, a.z);
  p = fmaf(p, x, a.y);
  return fmaf(p, x, a.x);
}
__device__ __forceinline__ double horner_tab(const double* c, double x) {
  const double2* v = reinterpret_cast<const double2*>(c);
  double2 k[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) k[i] = __ldg(v + i);
  double p = k[5].y;
  p = fma(p, x, k[5].x);
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    p = fma(p, x, k[i].y);
    p = fma(p, x, k[i].x);
  }
  return p;
}

// Interval record of (n1, n2) and its local coordinate x; rs = 1/sqrt(n) (1
// where n = 0, whose terms vanish with their n-power prefactor).
template <class R>
__device__ __forceinline__ const R* lhy_tab_locate(const LhyTab<R>& t, R n1, R n2, R& x, R& rs) {
  const R n = n1 + n2;
  rs = rsqrt_(n > R(0) ? n : R(1));
  const bool h = n1 > n2;
  const R a = sqrt_pos(h ? n2 : n1) * rs;
  const R tt = a * t.tscale;
  int i = (int)tt;  // a <= 1/sqrt(2) up to rounding: clamp to the last interval (NaN converts to 0)
  i = i < 0 ? 0 : (i < t.ni - 1 ? i : t.ni - 1);
  x = R(2) * (tt - (R)i) - R(1);
  return t.tab + (size_t)((h ? t.ni : 0) + i) * LhyTabDim<R>::rec;
}

// The table's part of mu_LHY,1 and mu_LHY,2 at NP points.
template <class R, int NP>
__device__ __forceinline__ void lhy_tab_mu(const LhyTab<R>& t, const R (&n1)[NP], const R (&n2)[NP], R (&m1)[NP],
                                           R (&m2)[NP]) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    R x, rs;
    const R* c = lhy_tab_locate(t, n1[j], n2[j], x, rs);
    const R n = n1[j] + n2[j];
    const R n32 = n * n * rs;
    m1[j] = n32 * horner_tab(c, x);
    m2[j] = n32 * horner_tab(c + LhyTabDim<R>::coef, x);
  }
}

// The table's part of n'^T (d^2 F/dn dn) n' at NP points.
template <class R, int NP>
__device__ __forceinline__ void lhy_tab_hess(const LhyTab<R>& t, const R (&n1)[NP], const R (&n2)[NP],
                                             const R (&n1p)[NP], const R (&n2p)[NP], R (&H)[NP]) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    R x, rs;
    const R* c = lhy_tab_locate(t, n1[j], n2[j], x, rs);
    const R n = n1[j] + n2[j];
    const R h11 = horner_tab(c + 2 * LhyTabDim<R>::coef, x);
    const R h12 = horner_tab(c + 3 * LhyTabDim<R>::coef, x);
    const R h22 = horner_tab(c + 4 * LhyTabDim<R>::coef, x);
    H[j] = n * rs * (n1p[j] * (h11 * n1p[j] + R(2) * h12 * n2p[j]) + h22 * n2p[j] * n2p[j]);
  }
}

}  // namespace egpe
