// On-device controller of the NCG loop (Algorithm 1).  Each step runs in
// thread 0 of the last block of the kernel whose reduction it needs, so the
// whole iteration stays on the device and can be replayed as a CUDA graph.
//
// Readings (where the paper is silent or garbled):
// * HS+ beta with the previous projected direction p^{n-1} in the denominator
//   (or PR+ with Re<r^{n-1}, P^{-1} r^{n-1}> of the previous iteration),
//   restart (beta = 0) when n mod K_r == 0, on a zero/non-finite denominator,
//   and when Re<r, p> >= 0 for the resulting direction (Sec. IV.C); if even the
//   restarted direction is not a descent direction the residual itself is used.
// * Step: alpha = -E'/E'' when E'' > 0 (Sec. V), largest theta_i capped at
//   theta_max; accepted on E_trial < E + accept_rtol |E| (a decrease up to the
//   round-off of the energy evaluation); otherwise, or when E'' <= 0, Armijo
//   halving along the same exact path, E(alpha) <= E + c1 alpha E' (+ the same
//   allowance), starting from the previous accepted alpha (pi/(4 max||p_i||) at
//   n = 0) when E'' <= 0 (Sec. V, last paragraph).
#pragma once
#include <math.h>

#include "common.cuh"

namespace egpe {

struct EnergyOut {
  double E, kin[2], trap, contact, dipolar, lhy, mu[2], norm2[2], shift[2], nmuL[2];
};

// Energy terms from the raw sums of one evaluation (sums are over grid points;
// the kinetic sums are Parseval sums of |k|^2/2 |psi^|^2 over the unnormalised DFT).
__host__ __device__ inline void finalize_energy(const double* eg, const double* egz, double dV, double invN,
                                                EnergyOut& o) {
  o.kin[0] = egz[EGZ_KIN1] * dV * invN;
  o.kin[1] = egz[EGZ_KIN2] * dV * invN;
  o.trap = eg[EG_TRAP] * dV;
  o.contact = eg[EG_CONTACT] * dV;
  o.dipolar = eg[EG_DIPOLAR] * dV;
  o.lhy = eg[EG_LHY] * dV;
  o.E = o.kin[0] + o.kin[1] + o.trap + o.contact + o.dipolar + o.lhy;
  o.mu[0] = eg[EG_MU1] * dV;
  o.mu[1] = eg[EG_MU2] * dV;
  o.norm2[0] = eg[EG_NORM1] * dV;
  o.norm2[1] = eg[EG_NORM2] * dV;
  // alpha_i = mu_i - Re<psi_i, Phi_i psi_i>  (preconditioner shift)
  o.shift[0] = o.mu[0] - eg[EG_NPHI1] * dV;
  o.shift[1] = o.mu[1] - eg[EG_NPHI2] * dV;
  o.nmuL[0] = eg[EG_NMUL1] * dV;
  o.nmuL[1] = eg[EG_NMUL2] * dV;
}

struct LineOut {
  double Ep, Epp, pnorm2[2], psip[2];
};

// E' = 2 sum_i Re<p_i, H_i psi_i>;
// E'' = sum_i 2(-||p_i||^2 mu_i + <p_i|T|p_i> + <p_i|U_i|p_i>) + 4 int sum_ij rho_i (g_ij rho_j + Phi_ij[rho_j])
//       + int LHY second variation (n''-free part),
// which regroups the paper's E'_i, E''_ij, E'_LHY, E''_LHY (Sec. V): the n''
// terms of E''_LHY combine with the H_MF terms into the full H_i (incl. mu_LHY).
__host__ __device__ inline void finalize_line(const double* lc, const double* lcz, const double mu[2], double dV,
                                              double invN, LineOut& o) {
  double Epp = 0.0;
  for (int i = 0; i < 2; ++i) {
    o.pnorm2[i] = lc[LC_P1 + i] * dV;
    o.psip[i] = lc[LC_PSIP1 + i] * dV;
    const double tpp = lcz[LCZ_TPP1 + i] * dV * invN;
    const double upp = lc[LC_UPP1 + i] * dV;
    Epp += 2.0 * (-o.pnorm2[i] * mu[i] + tpp + upp);
  }
  Epp += 4.0 * lc[LC_SRHO] * dV + lc[LC_HLHY] * dV;
  o.Ep = 2.0 * (lc[LC_PH1] + lc[LC_PH2]) * dV;
  o.Epp = Epp;
}

#ifdef __CUDACC__
__device__ __forceinline__ bool finite_(double x) { return isfinite(x); }

__device__ inline void set_retraction(DevState* st) {
  for (int i = 0; i < 2; ++i) {
    const double pn = sqrt(st->pnorm2[i]);
    const double th = st->alpha * pn;
    st->theta[i] = th;
    double s, c;
    sincos(th, &s, &c);
    if (pn > 0.0) {
      const double nrm2 = c * c * st->norm2[i] + s * s + 2.0 * c * s * st->psip[0 + i] / pn;
      const double inv = 1.0 / sqrt(nrm2);
      st->coef_a[i] = c * inv;
      st->coef_b[i] = s * inv / pn;
    } else {
      st->coef_a[i] = 1.0 / sqrt(st->norm2[i]);
      st->coef_b[i] = 0.0;
    }
  }
}

// A device wait that ran out of its budget ends the run with EGPE_ERR_TIMEOUT
// whatever the controller step would decide from the (incomplete) sums.
__device__ inline bool ctrl_timed_out(DevState* st) {
  if (!st->timeout) return false;
  st->status = 7;  // EGPE_ERR_TIMEOUT
  st->phase = PH_DONE;
  return true;
}

__device__ inline void load_point(DevState* st, int slot) {
  EnergyOut o;
  finalize_energy(st->eg[slot], st->egz[slot], st->dV, st->invN, o);
  st->E = o.E;
  for (int i = 0; i < 2; ++i) {
    st->mu[i] = o.mu[i];
    st->shift[i] = fabs(o.shift[i]);
    st->nmuL[i] = o.nmuL[i];
    st->norm2[i] = o.norm2[i];
  }
}

// After an energy/gradient evaluation.  mode 0: evaluation of the current
// point (start of a solve, or a standalone call); mode 1: trial point.
__device__ inline void ctrl_after_eg(DevState* st, int mode, TraceDev* trace) {
  if (ctrl_timed_out(st)) return;
  if (mode == 0) {
    load_point(st, st->cur);
    st->phase = finite_(st->E) ? PH_NEW_ITER : PH_DONE;
    if (!finite_(st->E)) st->status = 4;  // EGPE_ERR_NONFINITE
    return;
  }
  const int slot = st->cur ^ 1;
  EnergyOut o;
  finalize_energy(st->eg[slot], st->egz[slot], st->dV, st->invN, o);
  st->attempts += 1;
  st->E_trial = o.E;
  const SolveOptsDev& op = st->opt;
  const double tau = op.accept_rtol * fabs(st->E);
  bool ok;
  if (st->kind == 0 && st->armijo_k == 0) ok = o.E < st->E + tau;
  else ok = o.E <= st->E + op.armijo_c1 * st->alpha * st->Ep + tau;
  if (!finite_(o.E)) ok = false;
  if (trace && st->trace_len < op.trace_cap) {
    TraceDev& t = trace[st->trace_len];
    t.n = st->n;
    t.kind = st->kind;
    t.armijo = st->armijo_k;
    t.flags = (ok ? 1 : 0) | (st->restart_flag ? 2 : 0) | (st->fallback ? 4 : 0) | (op.fp32_phase ? 8 : 0);
    t.E = st->E;
    t.E_trial = o.E;
    t.res = st->res;
    t.beta = st->beta;
    t.alpha = st->alpha;
    t.theta[0] = st->theta[0];
    t.theta[1] = st->theta[1];
    t.Ep = st->Ep;
    t.Epp = st->Epp;
    st->trace_len += 1;
  }
  if (!finite_(o.E)) {
    st->status = 4;
    st->phase = PH_DONE;
    return;
  }
  if (ok) {
    const double Eold = st->E;
    st->rz_prev = st->rz;
    st->cur = slot;
    load_point(st, slot);
    st->dE_last = st->E - Eold;
    st->alpha_prev = st->alpha;
    st->n += 1;
    st->phase = PH_NEW_ITER;
    if (op.tol_dE > 0.0 && fabs(st->dE_last) < op.tol_dE) {
      st->status = 0;
      st->phase = PH_DONE;
    }
  } else {
    st->armijo_k += 1;
    st->armijo_total += 1;
    if (st->armijo_k > op.armijo_max) {
      st->status = 6;  // EGPE_ERR_STAGNATED
      st->phase = PH_DONE;
      return;
    }
    st->alpha = st->alpha0 / (double)(1ll << st->armijo_k);
    set_retraction(st);
    st->phase = PH_TRIAL;
  }
}

// End of one imaginary-time step: the energy of the renormalised state, the
// |E^{k+1} - E^k| < tol_dE stopping rule of the ITE comparison (Sec. VI.A).
__device__ inline void ctrl_after_ite(DevState* st) {
  if (ctrl_timed_out(st)) return;
  const double Eold = st->E;
  load_point(st, st->cur);
  st->dE_last = st->E - Eold;
  st->n += 1;
  if (!finite_(st->E)) {
    st->status = 4;
    st->phase = PH_DONE;
  } else if (fabs(st->dE_last) < st->opt.tol_dE) {
    st->status = 0;
    st->phase = PH_DONE;
  } else if (st->n >= st->opt.max_iter) {
    st->status = 5;
    st->phase = PH_DONE;
  }
}

// After the preconditioned residual and its sums: convergence test, beta,
// projection coefficients, restart rules.
__device__ inline void ctrl_after_pc(DevState* st) {
  if (ctrl_timed_out(st)) return;
  const double* pc = st->pc;
  const double dV = st->dV;
  const SolveOptsDev& op = st->opt;
  st->res = sqrt((pc[PC_RR1] + pc[PC_RR2]) * dV);
  if (!finite_(st->res)) {
    st->status = 4;
    st->phase = PH_DONE;
    return;
  }
  if (st->res < op.tol_res) {
    st->status = 0;
    st->phase = PH_DONE;
    return;
  }
  if (st->n >= op.max_iter) {
    st->status = 5;  // EGPE_ERR_NOT_CONVERGED
    st->phase = PH_DONE;
    return;
  }
  // FP32 fields: stop once the residual has stalled at its round-off floor
  // (no 10% decrease of the best residual within stall_iters iterations).
  if (op.stall_iters > 0) {
    if (st->n == 0 || st->res < 0.9 * st->res_best) {
      st->res_best = st->res;
      st->n_best = st->n;
    } else if (st->n - st->n_best >= op.stall_iters) {
      st->status = 5;
      st->phase = PH_DONE;
      return;
    }
  }
  bool restart = (op.restart_period <= 0) ? (st->n == 0) : (st->n % op.restart_period == 0);
  double beta = 0.0;
  st->rz = (pc[PC_ZR1] + pc[PC_ZR2]) * dV;
  if (!restart) {
    // HS+: Re<r - r_prev, z> / Re<r - r_prev, p_prev>;  PR+: Re<r - r_prev, z> / Re<r_prev, z_prev>
    const double num = pc[PC_SRZ] * dV;
    const double den = op.beta_rule == 1 ? st->rz_prev : pc[PC_SRP] * dV;
    if (den == 0.0 || !finite_(den) || !finite_(num)) restart = true;
    else beta = fmax(num / den, 0.0);
  }
  double c[2], descent = 0.0;
  for (int i = 0; i < 2; ++i) {
    c[i] = -pc[PC_ZPSI1 + i] + beta * pc[PC_PPPSI1 + i];
    descent += -pc[PC_ZR1 + i] + beta * pc[PC_PPR1 + i] - c[i] * pc[PC_PSIR1 + i];
  }
  if (descent >= 0.0 && beta != 0.0) {
    beta = 0.0;
    descent = 0.0;
    for (int i = 0; i < 2; ++i) {
      c[i] = -pc[PC_ZPSI1 + i];
      descent += -pc[PC_ZR1 + i] - c[i] * pc[PC_PSIR1 + i];
    }
  }
  st->fallback = 0;
  if (descent >= 0.0) {
    // p = -(r - Re<r,psi> psi): c_i = Re<-r_i, psi_i>
    st->fallback = 1;
    for (int i = 0; i < 2; ++i) c[i] = -pc[PC_PSIR1 + i];
  }
  st->beta = beta;
  st->restart_flag = (beta == 0.0) ? 1 : 0;
  if (beta == 0.0) st->restarts += 1;
  st->c[0] = c[0] * dV;
  st->c[1] = c[1] * dV;
}

// After the line-search sums: E', E'', alpha, theta, retraction coefficients.
__device__ inline void ctrl_after_lc(DevState* st) {
  if (ctrl_timed_out(st)) return;
  LineOut o;
  finalize_line(st->lc, st->lcz, st->mu, st->dV, st->invN, o);
  st->Ep = o.Ep;
  st->Epp = o.Epp;
  st->pnorm2[0] = o.pnorm2[0];
  st->pnorm2[1] = o.pnorm2[1];
  st->psip[0] = o.psip[0];
  st->psip[1] = o.psip[1];
  const double pmax = fmax(sqrt(o.pnorm2[0]), sqrt(o.pnorm2[1]));
  if (!(pmax > 0.0) || !finite_(pmax)) {
    st->status = (finite_(pmax)) ? 6 : 4;
    st->phase = PH_DONE;
    return;
  }
  double a0;
  if (o.Epp > 0.0 && finite_(o.Epp) && finite_(o.Ep)) {
    a0 = -o.Ep / o.Epp;
    st->kind = 0;
  } else {
    a0 = (st->n > 0 && st->alpha_prev > 0.0) ? st->alpha_prev : 3.14159265358979323846 / (4.0 * pmax);
    st->kind = 1;
  }
  if (a0 * pmax > st->opt.theta_max) a0 = st->opt.theta_max / pmax;
  st->alpha0 = a0;
  st->alpha = a0;
  st->armijo_k = 0;
  set_retraction(st);
}
#endif

}  // namespace egpe
