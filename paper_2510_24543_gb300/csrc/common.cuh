// Common device types of the eGPE hot path: complex helpers, kernel arguments,
// the on-device solver state and the scalar slots the reductions fill.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace egpe {

template <class R> struct CpxT;
template <> struct CpxT<double> { using T = double2; };
template <> struct CpxT<float> { using T = float2; };
template <class R> using C2 = typename CpxT<R>::T;

template <class C> __host__ __device__ __forceinline__ C cmk(decltype(C::x) x, decltype(C::x) y) {
  C c;
  c.x = x;
  c.y = y;
  return c;
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {
  return cmk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <class C, class R> __device__ __forceinline__ C cscale(C a, R s) { return cmk<C>(a.x * s, a.y * s); }
// Re(conj(a) b)
template <class C> __device__ __forceinline__ auto cdot(C a, C b) -> decltype(a.x) { return a.x * b.x + a.y * b.y; }
template <class C> __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }

// ---------------------------------------------------------------------------
// Scalar slots written by the deterministic reductions (FP64 always).
// ---------------------------------------------------------------------------
enum EgSlot {  // pointwise part of one energy/gradient evaluation (x dV later)
  EG_TRAP = 0, EG_CONTACT, EG_DIPOLAR, EG_LHY, EG_MU1, EG_MU2, EG_NPHI1, EG_NPHI2,
  EG_NMUL1, EG_NMUL2, EG_NORM1, EG_NORM2, EG_NS
};
enum EgzSlot { EGZ_KIN1 = 0, EGZ_KIN2, EGZ_NS };  // Parseval sums of the z pass
enum PcaSlot { PCA_RR1 = 0, PCA_RR2, PCA_NS };     // residual norms (first pass)
enum PcSlot {  // preconditioned residual / beta sums
  PC_SRZ = 0, PC_SRP, PC_ZPSI1, PC_ZPSI2, PC_PPPSI1, PC_PPPSI2, PC_ZR1, PC_ZR2,
  PC_PPR1, PC_PPR2, PC_PSIR1, PC_PSIR2, PC_RR1, PC_RR2, PC_NS
};
enum LcSlot {  // line-coefficient sums
  LC_P1 = 0, LC_P2, LC_PSIP1, LC_PSIP2, LC_PH1, LC_PH2, LC_UPP1, LC_UPP2, LC_SRHO, LC_HLHY, LC_NS
};
enum LczSlot { LCZ_TPP1 = 0, LCZ_TPP2, LCZ_NS };
enum RtSlot { RT_P1 = 0, RT_P2, RT_PSIP1, RT_PSIP2, RT_PSI1, RT_PSI2, RT_NS };
enum PgSlot {  // parameter-derivative sums (x dV later)
  PG_N11 = 0, PG_N12, PG_N22, PG_K11, PG_K12, PG_K22, PG_X2, PG_Y2, PG_Z2,
  PG_F, PG_L11, PG_L22, PG_L12, PG_M11, PG_M22, PG_M12, PG_NS
};
// Default row width in bytes of a column-pass tile (one cache line); the
// autotuner may pick 64 or 256 for the power-of-two lengths.
#define EGPE_COL_BYTES 128
static constexpr int MAX_NS = 16;
static_assert(PG_NS <= MAX_NS, "reduction slots");

// Phases of the on-device solver state machine.
enum Phase { PH_NEW_ITER = 0, PH_TRIAL = 1, PH_DONE = 2 };
// Launch gates: which phases a kernel runs in.
enum Gate { GATE_ALWAYS = 0, GATE_NEW_ITER = 1, GATE_ACTIVE = 2 };

struct SolveOptsDev {
  int precond, restart_period, max_iter, armijo_max, trace_cap, fp32_phase, beta_rule, stall_iters;
  double tol_res, tol_dE, armijo_c1, theta_max, accept_rtol, pv_floor, pc_blend;
};

struct TraceDev {
  int n, kind, armijo, flags;
  double E, E_trial, res, beta, alpha, theta[2], Ep, Epp;
};

// On-device solver/evaluation state.  One per engine (instance x precision).
struct DevState {
  // reduction outputs
  double eg[2][MAX_NS];    // per field-buffer slot
  double egz[2][4];
  double pca[4];
  double pc[MAX_NS];
  double lc[MAX_NS];
  double lcz[4];
  double rt[MAX_NS];
  double pg[MAX_NS];
  // flow control
  int phase, status, n, attempts, restarts, armijo_total, armijo_k, kind;
  int cur, fallback, trace_len, restart_flag;
  int rgiven, pgiven, timeout, pad1;  // timeout: a device wait ran out of its poll budget
  SolveOptsDev opt;
  // current point (slot cur)
  double E, mu[2], shift[2], nmuL[2], norm2[2];
  // iteration scalars
  double res, beta, c[2], alpha0, alpha, alpha_prev, theta[2], pnorm2[2];
  double Ep, Epp, coef_a[2], coef_b[2], E_trial, dE_last, psip[2];
  double rz, rz_prev;  // Re<r, P^{-1} r> of this and of the previous iteration (PR+ beta)
  double dV, invN;
  long long ffts;
  double res_best;     // smallest residual so far and the iteration that reached it
  int n_best, pad2;
};

// Gauss-Legendre node constants of the LHY u-integral, in field precision.
template <class R> struct LhyNode {
  R w;      // 3 u_q^2 - 1
  R W;      // kappa eta_s^{-5/2} times the quadrature weight on [0,1]
  R Ww;     // W w
  R e12sq;  // eta12(u_q)^2 = (g12 + gdd12 w)^2
  R gq;     // 2 sqrt(max(det eta(u_q), 0)): V+ V- = 4 n1 n2 det eta, so sqrt(V-) = gq sqrt(n1 n2) / sqrt(V+)
  R Www;    // W w^2
  R pad0, pad1;
};

// Couplings entering the LHY terms (symmetric: eta12 = eta21).
template <class R> struct LhyCoef {
  R g11, g22, g12, d11, d22, d12;
  R nskip;  // FP64: points with n1 + n2 <= nskip contribute below FP64 rounding (set per instance)
};

}  // namespace egpe
