// C ABI of the eGPE hot path (declared in include/egpe.h).  Validates every
// argument before any launch, maps CUDA failures to status codes, and drives
// the per-precision engines.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "egpe.h"
#include "engine.h"
#include "host_tables.h"

namespace egpe {

static thread_local std::string g_last_error;

void set_error(const char* what, cudaError_t e) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
}
void set_error_msg(const std::string& msg) { g_last_error = msg; }

// cast kernels for the mixed-precision hand-over (defined in engine units)
}  // namespace egpe

using egpe::Engine;

struct egpe_handle {
  int n_inst = 0;
  egpe_precision prec = EGPE_FP64;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // default-stream ordering of an owned stream
  std::vector<Engine<double>*> e64;
  std::vector<Engine<float>*> e32;
  std::vector<egpe_grid> grids;
};

namespace {

__global__ void cast_d2f(size_t n, const double2* in, float2* out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void cast_f2d(size_t n, const float2* in, double2* out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    out[i] = make_double2((double)v.x, (double)v.y);
  }
}

bool len_supported(int n) {
  return n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 48 || n == 80 || n == 96;
}

egpe_status validate(const egpe_grid& g, const egpe_params& p) {
  for (int a = 0; a < 3; ++a) {
    if (!len_supported(g.n[a])) {
      egpe::set_error_msg("grid size must be one of 16, 32, 48, 64, 80, 96, 128, 256 on every axis");
      return EGPE_ERR_INVALID_ARG;
    }
    if (!(g.L[a] > 0.0) || !std::isfinite(g.L[a])) {
      egpe::set_error_msg("box half-lengths must be positive and finite");
      return EGPE_ERR_INVALID_ARG;
    }
    if (!std::isfinite(p.trap[a])) {
      egpe::set_error_msg("trap frequencies must be finite");
      return EGPE_ERR_INVALID_ARG;
    }
  }
  if ((size_t)g.n[0] * g.n[1] * g.n[2] > (size_t)1 << 28) {
    egpe::set_error_msg("grid too large");
    return EGPE_ERR_INVALID_ARG;
  }
  if (p.g[0][1] != p.g[1][0] || p.gdd[0][1] != p.gdd[1][0]) {
    egpe::set_error_msg("couplings g and gdd must be symmetric");
    return EGPE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      if (!std::isfinite(p.g[i][j]) || !std::isfinite(p.gdd[i][j])) {
        egpe::set_error_msg("couplings must be finite");
        return EGPE_ERR_INVALID_ARG;
      }
  if (p.lhy_nodes < 1 || p.lhy_nodes > 64 || !(p.lhy_eta_scale > 0.0) || !std::isfinite(p.lhy_kappa)) {
    egpe::set_error_msg("lhy_nodes must be in [1,64], lhy_eta_scale > 0, lhy_kappa finite");
    return EGPE_ERR_INVALID_ARG;
  }
  return EGPE_OK;
}

bool bad_inst(egpe_handle* h, int inst) { return !h || inst < 0 || inst >= h->n_inst; }

// A handle created without a stream works on a stream of its own, which does
// not synchronise with the legacy default stream by itself.  Every call on
// such a handle is therefore ordered after the work already submitted to the
// legacy default stream (the caller's writes of its input buffers), and the
// legacy default stream after the call's own work (its writes of the output
// buffers), so callers on the default stream need no synchronisation.
struct DefaultStreamJoin {
  egpe_handle* h;
  explicit DefaultStreamJoin(egpe_handle* hh) : h(hh) {
    if (h->own_stream) {
      cudaEventRecord(h->ev_in, cudaStreamLegacy);
      cudaStreamWaitEvent(h->stream, h->ev_in, 0);
    }
  }
  ~DefaultStreamJoin() {
    if (h->own_stream) {
      cudaEventRecord(h->ev_out, h->stream);
      cudaStreamWaitEvent(cudaStreamLegacy, h->ev_out, 0);
    }
  }
  DefaultStreamJoin(const DefaultStreamJoin&) = delete;
  DefaultStreamJoin& operator=(const DefaultStreamJoin&) = delete;
};

egpe_status sync_and_check(egpe_handle* h) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    egpe::set_error("cudaStreamSynchronize", e);
    return EGPE_ERR_CUDA;
  }
  return EGPE_OK;
}

}  // namespace

extern "C" {

int egpe_version(void) { return 103; }

const char* egpe_last_error(void) { return egpe::g_last_error.c_str(); }

const char* egpe_status_string(egpe_status s) {
  switch (s) {
    case EGPE_OK: return "ok";
    case EGPE_ERR_INVALID_ARG: return "invalid argument";
    case EGPE_ERR_CUDA: return "CUDA error";
    case EGPE_ERR_OOM: return "out of device memory";
    case EGPE_ERR_NONFINITE: return "non-finite value";
    case EGPE_ERR_NOT_CONVERGED: return "not converged";
    case EGPE_ERR_STAGNATED: return "stagnated (no acceptable step)";
    case EGPE_ERR_TIMEOUT: return "timeout";
    case EGPE_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

void egpe_default_solve_opts(egpe_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precond = EGPE_PRECOND_KINETIC;
  o->beta_rule = 0;
  o->restart_period = 20;
  o->max_iter = 2000;
  o->armijo_max = 30;
  o->poll_every = 8;
  o->use_graph = 1;
  o->psi_on_host = 0;
  o->tol_res = 1e-8;
  o->tol_dE = 0.0;
  o->armijo_c1 = 1e-4;
  o->theta_max = 1.5707963267948966;
  o->accept_rtol = 1e-13;
  o->accept_rtol_fp32 = 1e-6;
  o->pv_floor = 1e-2;
  o->tol_fp32_switch = 1e-4;
  o->max_iter_fp32 = 2000;
  o->trace_cap = 0;
  o->trace = nullptr;
  o->batch = 1;
  o->stall_iters_fp32 = 0;
  o->pc_blend = 0.5;
}

egpe_status egpe_create(const egpe_grid* grids, const egpe_params* params, int n_inst, egpe_precision prec,
                        void* cuda_stream, egpe_handle** out) {
  if (!out) return EGPE_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grids || !params || n_inst < 1 || n_inst > 4096 || (prec != EGPE_FP64 && prec != EGPE_FP32 && prec != EGPE_MIXED)) {
    egpe::set_error_msg("egpe_create: bad arguments");
    return EGPE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_inst; ++i) {
    egpe_status s = validate(grids[i], params[i]);
    if (s != EGPE_OK) return s;
  }
  egpe_handle* h = new egpe_handle();
  h->n_inst = n_inst;
  h->prec = prec;
  cudaGetDevice(&h->device);
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      egpe::set_error("cudaStreamCreateWithFlags/cudaEventCreateWithFlags", e);
      if (h->ev_in) cudaEventDestroy(h->ev_in);
      if (h->stream) cudaStreamDestroy(h->stream);
      delete h;
      return EGPE_ERR_CUDA;
    }
    h->own_stream = true;
  }
  h->grids.assign(grids, grids + n_inst);
  for (int i = 0; i < n_inst; ++i) {
    if (prec == EGPE_FP64 || prec == EGPE_MIXED) {
      auto* e = new Engine<double>();
      h->e64.push_back(e);
      egpe_status s = e->create(grids[i], params[i], h->stream);
      if (s != EGPE_OK) {
        egpe_destroy(h);
        return s;
      }
    }
    if (prec == EGPE_FP32 || prec == EGPE_MIXED) {
      auto* e = new Engine<float>();
      h->e32.push_back(e);
      egpe_status s = e->create(grids[i], params[i], h->stream);
      if (s != EGPE_OK) {
        egpe_destroy(h);
        return s;
      }
    }
  }
  egpe_status s = sync_and_check(h);
  if (s != EGPE_OK) {
    egpe_destroy(h);
    return s;
  }
  *out = h;
  return EGPE_OK;
}

void egpe_destroy(egpe_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto* e : h->e64) delete e;
  for (auto* e : h->e32) delete e;
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  delete h;
}

egpe_status egpe_energy_terms_eval(egpe_handle* h, int inst, const void* psi, egpe_energy_terms* terms, void* grad) {
  if (bad_inst(h, inst) || !psi) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  if (h->prec == EGPE_FP32)
    return h->e32[inst]->energy_grad((const float2*)psi, terms, (float2*)grad);
  return h->e64[inst]->energy_grad((const double2*)psi, terms, (double2*)grad);
}

egpe_status egpe_energy_grad(egpe_handle* h, int inst, const void* psi, double* E, double mu[2], void* grad) {
  egpe_energy_terms t;
  egpe_status s = egpe_energy_terms_eval(h, inst, psi, &t, grad);
  if (s != EGPE_OK) return s;
  if (E) *E = t.E;
  if (mu) {
    mu[0] = t.mu[0];
    mu[1] = t.mu[1];
  }
  return EGPE_OK;
}

egpe_status egpe_line_coeffs(egpe_handle* h, int inst, const void* psi, const void* p, double coeffs[3]) {
  if (bad_inst(h, inst) || !psi || !p || !coeffs) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  if (h->prec == EGPE_FP32) return h->e32[inst]->line_coeffs((const float2*)psi, (const float2*)p, coeffs);
  return h->e64[inst]->line_coeffs((const double2*)psi, (const double2*)p, coeffs);
}

egpe_status egpe_precondition(egpe_handle* h, int inst, int mode, const void* psi, const void* r, void* z) {
  if (bad_inst(h, inst) || !psi || !z || mode < 0 || mode > 4) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  if (h->prec == EGPE_FP32)
    return h->e32[inst]->precondition(mode, (const float2*)psi, (const float2*)r, (float2*)z);
  return h->e64[inst]->precondition(mode, (const double2*)psi, (const double2*)r, (double2*)z);
}

egpe_status egpe_retract(egpe_handle* h, int inst, const void* psi, const void* p, const double theta[2],
                         void* psi_out) {
  if (bad_inst(h, inst) || !psi || !p || !theta || !psi_out) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  if (!std::isfinite(theta[0]) || !std::isfinite(theta[1])) return EGPE_ERR_INVALID_ARG;
  if (h->prec == EGPE_FP32)
    return h->e32[inst]->retract((const float2*)psi, (const float2*)p, theta, (float2*)psi_out);
  return h->e64[inst]->retract((const double2*)psi, (const double2*)p, theta, (double2*)psi_out);
}

egpe_status egpe_fft(egpe_handle* h, int inst, const void* in, void* out, int nfields, int inverse) {
  if (bad_inst(h, inst) || !in || !out || nfields < 1 || nfields > 64) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  if (h->prec == EGPE_FP32) return h->e32[inst]->fft((const float2*)in, (float2*)out, nfields, inverse ? 1 : 0);
  return h->e64[inst]->fft((const double2*)in, (double2*)out, nfields, inverse ? 1 : 0);
}

egpe_status egpe_profile_attempt(egpe_handle* h, int inst, int engine, const void* psi, int precond, int reps,
                                 int cap, char* names, double* ms, double* bytes, int* count) {
  if (bad_inst(h, inst) || !psi || precond < 0 || precond > 4 || reps < 1 || cap < 1 || !names || !ms || !bytes ||
      !count)
    return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  std::vector<std::string> nm;
  std::vector<double> t, b;
  egpe_status s;
  if (engine == 0 && !h->e64.empty()) {
    s = h->e64[inst]->profile_attempt((const double2*)psi, precond, reps, nm, t, b);
  } else if (engine == 1 && !h->e32.empty()) {
    s = h->e32[inst]->profile_attempt((const float2*)psi, precond, reps, nm, t, b);
  } else {
    return EGPE_ERR_INVALID_ARG;
  }
  if (s != EGPE_OK) return s;
  const int n = (int)std::min<size_t>(nm.size(), (size_t)cap);
  for (int k = 0; k < n; ++k) {
    std::strncpy(names + 48 * k, nm[k].c_str(), 47);
    names[48 * k + 47] = 0;
    ms[k] = t[k];
    bytes[k] = b[k];
  }
  *count = n;
  return EGPE_OK;
}

egpe_status egpe_param_grad(egpe_handle* h, int inst, const void* psi, double* dEdp) {
  if (bad_inst(h, inst) || !psi || !dEdp) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  if (h->prec == EGPE_FP32) return h->e32[inst]->param_grad((const float2*)psi, dEdp);
  return h->e64[inst]->param_grad((const double2*)psi, dEdp);
}

egpe_status egpe_set_params(egpe_handle* h, int inst, const egpe_params* params) {
  if (bad_inst(h, inst) || !params) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  egpe_status s = validate(h->grids[inst], *params);
  if (s != EGPE_OK) return s;
  if (!h->e64.empty()) {
    s = h->e64[inst]->set_params(*params);
    if (s != EGPE_OK) return s;
  }
  if (!h->e32.empty()) s = h->e32[inst]->set_params(*params);
  return s;
}

egpe_status egpe_autotune(egpe_handle* h, int inst, int engine, const void* psi, int precond, int reps,
                          egpe_tuning* out, int cap, int* count) {
  if (bad_inst(h, inst) || !psi || precond < 0 || precond > 4 || reps < 1 || cap < 0 || (cap > 0 && !out))
    return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  std::vector<egpe::TuneResult> res;
  egpe_status s;
  if (engine == 0 && !h->e64.empty()) s = h->e64[inst]->autotune((const double2*)psi, precond, reps, res);
  else if (engine == 1 && !h->e32.empty()) s = h->e32[inst]->autotune((const float2*)psi, precond, reps, res);
  else return EGPE_ERR_INVALID_ARG;
  if (s != EGPE_OK) return s;
  const int n = (int)std::min<size_t>(res.size(), (size_t)cap);
  for (int k = 0; k < n; ++k) {
    egpe_tuning& t = out[k];
    std::memset(&t, 0, sizeof(t));
    std::strncpy(t.key, res[k].key.c_str(), sizeof(t.key) - 1);
    std::strncpy(t.name, res[k].name.c_str(), sizeof(t.name) - 1);
    t.L = res[k].L;
    t.kind = res[k].kind;
    t.choice = res[k].choice;
    t.default_choice = res[k].default_choice;
    t.ms_best = res[k].ms_best;
    t.ms_default = res[k].ms_default;
  }
  if (count) *count = n;
  return EGPE_OK;
}

egpe_status egpe_lhy_table_eval(const egpe_params* params, int precision, int count, const double* n1,
                                const double* n2, double* mu, double* hess, int info[2]) {
  if (!params || count < 0 || (count > 0 && (!n1 || !n2 || !mu || !hess))) return EGPE_ERR_INVALID_ARG;
  if (precision != EGPE_FP64 && precision != EGPE_FP32) return EGPE_ERR_INVALID_ARG;
  const egpe_grid g1 = {{16, 16, 16}, {1.0, 1.0, 1.0}};
  egpe_status s = validate(g1, *params);
  if (s != EGPE_OK) return s;
  const egpe_params& p = *params;
  const egpe::LhyTableHost T = precision == EGPE_FP32 ? egpe::lhy_interp_table_cached<float>(p)
                                                      : egpe::lhy_interp_table_cached<double>(p);
  const int NC = T.deg + 1, NR = egpe::kTabFun * NC;
  if (info) {
    info[0] = T.ni;
    info[1] = (int)T.exact.size();
  }
  std::vector<long double> u, w;
  egpe::gauss_legendre01(p.lhy_nodes, u, w);
  const long double c5 = (long double)p.lhy_kappa * powl((long double)p.lhy_eta_scale, -2.5L);
  const double tscale = T.ni * 1.4142135623730950488;
  for (int k = 0; k < count; ++k) {
    if (!(n1[k] >= 0.0) || !(n2[k] >= 0.0)) return EGPE_ERR_INVALID_ARG;
    long double o[egpe::kTabFun] = {};
    for (int q : T.exact) {
      const long double sw = 3.0L * u[q] * u[q] - 1.0L;
      egpe::lhy_node_terms(p.g[0][0] + p.gdd[0][0] * sw, p.g[1][1] + p.gdd[1][1] * sw, p.g[0][1] + p.gdd[0][1] * sw,
                           c5 * w[q], n1[k], n2[k], o);
    }
    double v[egpe::kTabFun];
    for (int f = 0; f < egpe::kTabFun; ++f) v[f] = (double)o[f];
    const double n = n1[k] + n2[k];
    if (T.ni > 0 && n > 0.0) {  // the device evaluation, in FP64 on the host
      const int half = n1[k] > n2[k];
      const double a = std::sqrt(half ? n2[k] : n1[k]) / std::sqrt(n);
      const double tt = a * tscale;
      const int i = std::min((int)tt, T.ni - 1);
      const double x = 2.0 * (tt - i) - 1.0;
      const long double* c = &T.coef[((size_t)half * T.ni + i) * NR];
      for (int f = 0; f < egpe::kTabFun; ++f) {
        double pv = (double)c[f * NC + T.deg];
        for (int m = T.deg - 1; m >= 0; --m) pv = std::fma(pv, x, (double)c[f * NC + m]);
        v[f] += (f < 2 ? n * std::sqrt(n) : std::sqrt(n)) * pv;
      }
    }
    mu[2 * k] = v[0];
    mu[2 * k + 1] = v[1];
    hess[3 * k] = v[2];
    hess[3 * k + 1] = v[3];
    hess[3 * k + 2] = v[4];
  }
  return EGPE_OK;
}

egpe_status egpe_set_wait_limit(egpe_handle* h, long long polls) {
  if (!h || polls < 0) return EGPE_ERR_INVALID_ARG;
  for (auto* e : h->e64) e->set_wait_limit(polls);
  for (auto* e : h->e32) e->set_wait_limit(polls);
  return EGPE_OK;
}

egpe_status egpe_set_tuning(egpe_handle* h, int inst, int engine, const egpe_tuning* t, int count) {
  if (bad_inst(h, inst) || count < 0 || (count > 0 && !t)) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  for (int k = 0; k < count; ++k) {
    std::string key(t[k].key, strnlen(t[k].key, sizeof(t[k].key)));
    if (engine == 0 && !h->e64.empty()) h->e64[inst]->set_tuning(key, t[k].choice);
    else if (engine == 1 && !h->e32.empty()) h->e32[inst]->set_tuning(key, t[k].choice);
    else return EGPE_ERR_INVALID_ARG;
  }
  return EGPE_OK;
}

static bool opts_ok(const egpe_solve_opts& o) {
  return !(o.precond < 0 || o.precond > 4 || !(o.pc_blend >= 0.0 && o.pc_blend <= 1.0) || o.beta_rule < 0 || o.beta_rule > 1 || o.max_iter < 0 || o.armijo_max < 0 ||
           o.armijo_max > 60 || !(o.tol_res >= 0.0) || !(o.theta_max > 0.0) || !(o.pv_floor > 0.0) ||
           o.trace_cap < 0 || (o.trace_cap > 0 && !o.trace) || o.stall_iters_fp32 < 0);
}

egpe_status egpe_solver_start(egpe_handle* h, int inst, int engine, const void* psi, const egpe_solve_opts* opts) {
  if (bad_inst(h, inst) || !psi || !opts || !opts_ok(*opts)) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  const egpe_solve_opts& o = *opts;
  if (engine == 0 && !h->e64.empty()) {
    auto* e = h->e64[inst];
    egpe_status s = e->load_psi(psi, cudaMemcpyDeviceToDevice);
    if (s != EGPE_OK) return s;
    return e->solve_begin(o, 0, o.max_iter, o.tol_res, o.accept_rtol, false, 0);
  }
  if (engine == 1 && !h->e32.empty()) {
    auto* e = h->e32[inst];
    egpe_status s = e->load_psi(psi, cudaMemcpyDeviceToDevice);
    if (s != EGPE_OK) return s;
    return e->solve_begin(o, 1, o.max_iter, o.tol_res, o.accept_rtol_fp32, false, 0);
  }
  return EGPE_ERR_INVALID_ARG;
}

egpe_status egpe_solver_step(egpe_handle* h, int inst, int engine, int attempts) {
  if (bad_inst(h, inst) || attempts < 0) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  if (engine == 0 && !h->e64.empty()) return h->e64[inst]->solve_launch(attempts);
  if (engine == 1 && !h->e32.empty()) return h->e32[inst]->solve_launch(attempts);
  return EGPE_ERR_INVALID_ARG;
}

egpe_status egpe_solver_read(egpe_handle* h, int inst, int engine, egpe_report* report, void* psi_out) {
  if (bad_inst(h, inst) || !report) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  egpe::SolveRun run{};
  egpe_status s;
  if (engine == 0 && !h->e64.empty()) {
    s = h->e64[inst]->solve_finish(run, nullptr, 0, 0);
    if (s == EGPE_OK && psi_out) s = h->e64[inst]->store_psi(psi_out, cudaMemcpyDeviceToDevice);
  } else if (engine == 1 && !h->e32.empty()) {
    s = h->e32[inst]->solve_finish(run, nullptr, 0, 0);
    if (s == EGPE_OK && psi_out) s = h->e32[inst]->store_psi(psi_out, cudaMemcpyDeviceToDevice);
  } else {
    return EGPE_ERR_INVALID_ARG;
  }
  if (s != EGPE_OK) return s;
  std::memset(report, 0, sizeof(*report));
  report->status = run.status;
  report->iters = run.n;
  report->iters_fp32 = engine == 1 ? run.n : 0;
  report->attempts = run.attempts;
  report->restarts = run.restarts;
  report->armijo_steps = run.armijo_total;
  report->graph_launches = run.launches;
  report->E = run.E;
  report->mu[0] = run.mu[0];
  report->mu[1] = run.mu[1];
  report->res = run.res;
  report->ffts = run.ffts;
  report->kernels = run.kernels;
  return EGPE_OK;
}

}  // extern "C"

namespace {

// All instances advance together (batch.cuh); same phases as the sequential
// path per precision.
egpe_status ncg_solve_batched(egpe_handle* h, void* const* psi_inout, const egpe_solve_opts& o,
                              egpe_report* reports) {
  const auto t0 = std::chrono::steady_clock::now();
  const int n = h->n_inst;
  const cudaMemcpyKind kin = o.psi_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = o.psi_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  egpe_trace_entry* trace = (egpe_trace_entry*)o.trace;
  std::vector<egpe::SolveRun> runs, r32;
  egpe_status s = EGPE_OK;
  if (h->prec == EGPE_FP64) {
    for (int i = 0; i < n && s == EGPE_OK; ++i) s = h->e64[i]->load_psi(psi_inout[i], kin);
    if (s == EGPE_OK)
      s = egpe::batch_solve<double>(h->e64, h->stream, o, 0, o.max_iter, o.tol_res, o.accept_rtol, runs, trace,
                                    o.trace_cap, nullptr);
    for (int i = 0; i < n && s == EGPE_OK; ++i) s = h->e64[i]->store_psi(psi_inout[i], kout);
  } else if (h->prec == EGPE_FP32) {
    for (int i = 0; i < n && s == EGPE_OK; ++i) s = h->e32[i]->load_psi(psi_inout[i], kin);
    if (s == EGPE_OK)
      s = egpe::batch_solve<float>(h->e32, h->stream, o, 1, o.max_iter, o.tol_res, o.accept_rtol_fp32, runs, trace,
                                   o.trace_cap, nullptr);
    for (int i = 0; i < n && s == EGPE_OK; ++i) s = h->e32[i]->store_psi(psi_inout[i], kout);
  } else {  // MIXED: batched FP32 phase, then batched FP64 polish
    for (int i = 0; i < n && s == EGPE_OK; ++i) {
      s = h->e64[i]->load_psi(psi_inout[i], kin);
      if (s == EGPE_OK) {
        cast_d2f<<<256, 256, 0, h->stream>>>(2 * h->e64[i]->N, (const double2*)h->e64[i]->psi_slot0(),
                                             h->e32[i]->psi_slot0());
        if (cudaGetLastError() != cudaSuccess) s = EGPE_ERR_CUDA;
      }
    }
    if (s == EGPE_OK)
      s = egpe::batch_solve<float>(h->e32, h->stream, o, 1, o.max_iter_fp32, std::max(o.tol_res, o.tol_fp32_switch),
                                   o.accept_rtol_fp32, r32, trace, o.trace_cap, nullptr);
    for (int i = 0; i < n && s == EGPE_OK; ++i) {
      cast_f2d<<<256, 256, 0, h->stream>>>(2 * h->e64[i]->N, h->e32[i]->current_psi(), h->e64[i]->psi_slot0());
      if (cudaGetLastError() != cudaSuccess) s = EGPE_ERR_CUDA;
      if (s == EGPE_OK) s = h->e64[i]->normalise_current();
    }
    const int t32 = (trace && !r32.empty()) ? r32[0].trace_len : 0;
    const int tcap2 = trace ? std::max(0, o.trace_cap - t32) : 0;
    if (s == EGPE_OK)
      s = egpe::batch_solve<double>(h->e64, h->stream, o, 0, o.max_iter, o.tol_res, o.accept_rtol, runs,
                                    tcap2 > 0 ? trace + t32 : nullptr, tcap2, nullptr);
    for (int i = 0; i < n && s == EGPE_OK; ++i) s = h->e64[i]->store_psi(psi_inout[i], kout);
  }
  if (s != EGPE_OK) return s;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  egpe_status first_bad = EGPE_OK;
  for (int i = 0; i < n; ++i) {
    egpe::SolveRun run = runs[i];
    egpe_report rep;
    std::memset(&rep, 0, sizeof(rep));
    if (h->prec == EGPE_MIXED) {
      rep.iters_fp32 = r32[i].n;
      run.n += r32[i].n;
      run.attempts += r32[i].attempts;
      run.restarts += r32[i].restarts;
      run.armijo_total += r32[i].armijo_total;
      run.launches += r32[i].launches;
      run.ffts += r32[i].ffts;
      run.kernels += r32[i].kernels;
      run.trace_len += r32[i].trace_len;
    }
    if (h->prec == EGPE_FP32) rep.iters_fp32 = run.n;
    rep.status = run.status;
    rep.iters = run.n;
    rep.attempts = run.attempts;
    rep.restarts = run.restarts;
    rep.armijo_steps = run.armijo_total;
    rep.trace_len = i == 0 ? run.trace_len : 0;
    rep.graph_launches = run.launches;
    rep.E = run.E;
    rep.mu[0] = run.mu[0];
    rep.mu[1] = run.mu[1];
    rep.res = run.res;
    rep.seconds = secs;
    rep.ffts = run.ffts;
    rep.kernels = run.kernels;
    if (reports) reports[i] = rep;
    if (rep.status != EGPE_OK && first_bad == EGPE_OK) first_bad = (egpe_status)rep.status;
  }
  return first_bad;
}

// One instance, one precision path (FP64, FP32, or MIXED: FP32 phase then
// FP64 polish), from psi (device or host per o.psi_on_host) back into psi.
egpe_status solve_one(egpe_handle* h, int i, void* psi, const egpe_solve_opts& o, egpe_trace_entry* tr, int tcap,
                      egpe_report& rep) {
  const auto t0 = std::chrono::steady_clock::now();
  std::memset(&rep, 0, sizeof(rep));
  egpe::SolveRun run{};
  egpe_status s = EGPE_OK;
  const cudaMemcpyKind kin = o.psi_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = o.psi_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (h->prec == EGPE_FP64) {
    auto* e = h->e64[i];
    s = e->load_psi(psi, kin);
    if (s == EGPE_OK) s = e->solve(o, 0, o.max_iter, o.tol_res, o.accept_rtol, run, tr, tcap, 0);
    if (s == EGPE_OK) s = e->store_psi(psi, kout);
  } else if (h->prec == EGPE_FP32) {
    auto* e = h->e32[i];
    s = e->load_psi(psi, kin);
    if (s == EGPE_OK) s = e->solve(o, 1, o.max_iter, o.tol_res, o.accept_rtol_fp32, run, tr, tcap, 0);
    if (s == EGPE_OK) s = e->store_psi(psi, kout);
  } else {  // MIXED: FP32 phase, then FP64 polish
    auto* e64 = h->e64[i];
    auto* e32 = h->e32[i];
    s = e64->load_psi(psi, kin);
    const size_t n2 = 2 * e64->N;
    if (s == EGPE_OK) {
      cast_d2f<<<256, 256, 0, h->stream>>>(n2, (const double2*)e64->psi_slot0(), e32->psi_slot0());
      if (cudaGetLastError() != cudaSuccess) s = EGPE_ERR_CUDA;
    }
    egpe::SolveRun r32{};
    if (s == EGPE_OK)
      s = e32->solve(o, 1, o.max_iter_fp32, std::max(o.tol_res, o.tol_fp32_switch), o.accept_rtol_fp32, r32, tr,
                     tcap, 0);
    if (s == EGPE_OK) {
      cast_f2d<<<256, 256, 0, h->stream>>>(n2, e32->current_psi(), e64->psi_slot0());
      if (cudaGetLastError() != cudaSuccess) s = EGPE_ERR_CUDA;
    }
    if (s == EGPE_OK) s = e64->normalise_current();
    egpe_trace_entry* tr2 = tr ? tr + r32.trace_len : nullptr;
    const int tcap2 = tr ? std::max(0, tcap - r32.trace_len) : 0;
    if (s == EGPE_OK)
      s = e64->solve(o, 0, o.max_iter, o.tol_res, o.accept_rtol, run, tcap2 > 0 ? tr2 : nullptr, tcap2, 0);
    if (s == EGPE_OK) s = e64->store_psi(psi, kout);
    rep.iters_fp32 = r32.n;
    run.n += r32.n;
    run.attempts += r32.attempts;
    run.restarts += r32.restarts;
    run.armijo_total += r32.armijo_total;
    run.launches += r32.launches;
    run.ffts += r32.ffts;
    run.kernels += r32.kernels;
    run.trace_len += r32.trace_len;
  }
  const auto t1 = std::chrono::steady_clock::now();
  if (s != EGPE_OK) {
    rep.status = s;
  } else {
    rep.status = run.status;
  }
  rep.iters = run.n;
  if (h->prec == EGPE_FP32) rep.iters_fp32 = run.n;
  rep.attempts = run.attempts;
  rep.restarts = run.restarts;
  rep.armijo_steps = run.armijo_total;
  rep.trace_len = run.trace_len;
  rep.graph_launches = run.launches;
  rep.E = run.E;
  rep.mu[0] = run.mu[0];
  rep.mu[1] = run.mu[1];
  rep.res = run.res;
  rep.seconds = std::chrono::duration<double>(t1 - t0).count();
  rep.ffts = run.ffts;
  rep.kernels = run.kernels;
  return s;
}

}  // namespace

extern "C" {

egpe_status egpe_ncg_solve(egpe_handle* h, void* const* psi_inout, const egpe_solve_opts* opts,
                           egpe_report* reports) {
  if (!h || !psi_inout || !opts) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  const egpe_solve_opts& o = *opts;
  if (!opts_ok(o)) {
    egpe::set_error_msg("egpe_ncg_solve: bad options");
    return EGPE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < h->n_inst; ++i)
    if (!psi_inout[i]) return EGPE_ERR_INVALID_ARG;
  if (h->n_inst > 1 && o.batch) return ncg_solve_batched(h, psi_inout, o, reports);
  egpe_status first_bad = EGPE_OK;
  egpe_trace_entry* trace = (egpe_trace_entry*)o.trace;
  for (int i = 0; i < h->n_inst; ++i) {
    egpe_report rep;
    // the trace follows the first instance
    const egpe_status s = solve_one(h, i, psi_inout[i], o, i == 0 ? trace : nullptr, i == 0 ? o.trace_cap : 0, rep);
    if (reports) reports[i] = rep;
    if (s != EGPE_OK) return s;
    if (rep.status != EGPE_OK && first_bad == EGPE_OK) first_bad = (egpe_status)rep.status;
  }
  return first_bad;
}

egpe_status egpe_ncg_continuation(egpe_handle* h, int inst, const egpe_params* path, int npoints, void* psi_inout,
                                  void* const* psi_out, const egpe_solve_opts* opts, egpe_report* reports) {
  if (bad_inst(h, inst) || !path || npoints < 1 || !psi_inout || !opts) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  const egpe_solve_opts& o = *opts;
  if (!opts_ok(o)) {
    egpe::set_error_msg("egpe_ncg_continuation: bad options");
    return EGPE_ERR_INVALID_ARG;
  }
  for (int k = 0; k < npoints; ++k) {
    const egpe_status v = validate(h->grids[inst], path[k]);
    if (v != EGPE_OK) return v;
  }
  const size_t bytes = 2 * (h->prec == EGPE_FP32 ? h->e32[inst]->N * sizeof(float2) : h->e64[inst]->N * sizeof(double2));
  egpe_status first_bad = EGPE_OK;
  for (int k = 0; k < npoints; ++k) {
    egpe_status s = egpe_set_params(h, inst, &path[k]);
    if (s != EGPE_OK) return s;
    egpe_report rep;
    s = solve_one(h, inst, psi_inout, o, nullptr, 0, rep);  // warm start: psi_inout holds the last state
    if (reports) reports[k] = rep;
    if (s != EGPE_OK) return s;
    if (psi_out && psi_out[k]) {
      if (o.psi_on_host) {
        std::memcpy(psi_out[k], psi_inout, bytes);
      } else {
        cudaError_t e = cudaMemcpyAsync(psi_out[k], psi_inout, bytes, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
          egpe::set_error("egpe_ncg_continuation copy", e);
          return EGPE_ERR_CUDA;
        }
      }
    }
    if (rep.status != EGPE_OK && first_bad == EGPE_OK) first_bad = (egpe_status)rep.status;
  }
  return first_bad;
}

void egpe_default_ite_opts(egpe_ite_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->dtau = 1e-3;
  o->tol_dE = 1e-10;
  o->max_steps = 100000;
  o->poll_every = 32;
  o->use_graph = 1;
  o->psi_on_host = 0;
}

egpe_status egpe_ite_solve(egpe_handle* h, void* const* psi_inout, const egpe_ite_opts* opts,
                           egpe_report* reports) {
  if (!h || !psi_inout || !opts) return EGPE_ERR_INVALID_ARG;
  DefaultStreamJoin join(h);
  const egpe_ite_opts& o = *opts;
  if (!(o.dtau > 0.0) || !std::isfinite(o.dtau) || !(o.tol_dE > 0.0) || o.max_steps <= 0 || o.poll_every < 0) {
    egpe::set_error_msg("egpe_ite_solve: dtau and tol_dE must be positive and finite, max_steps > 0");
    return EGPE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < h->n_inst; ++i)
    if (!psi_inout[i]) return EGPE_ERR_INVALID_ARG;
  egpe_status first_bad = EGPE_OK;
  const cudaMemcpyKind kin = o.psi_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = o.psi_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  for (int i = 0; i < h->n_inst; ++i) {
    const auto t0 = std::chrono::steady_clock::now();
    egpe::SolveRun run{};
    egpe_status s;
    if (h->prec == EGPE_FP32) {
      auto* e = h->e32[i];
      s = e->load_psi(psi_inout[i], kin);
      if (s == EGPE_OK) s = e->ite(o.dtau, o.tol_dE, o.max_steps, o.poll_every, o.use_graph != 0, run);
      if (s == EGPE_OK) s = e->store_psi(psi_inout[i], kout);
    } else {
      auto* e = h->e64[i];
      s = e->load_psi(psi_inout[i], kin);
      if (s == EGPE_OK) s = e->ite(o.dtau, o.tol_dE, o.max_steps, o.poll_every, o.use_graph != 0, run);
      if (s == EGPE_OK) s = e->store_psi(psi_inout[i], kout);
    }
    const auto t1 = std::chrono::steady_clock::now();
    egpe_report rep;
    std::memset(&rep, 0, sizeof(rep));
    rep.status = (s != EGPE_OK) ? s : run.status;
    rep.iters = run.n;
    if (h->prec == EGPE_FP32) rep.iters_fp32 = run.n;
    rep.graph_launches = run.launches;
    rep.E = run.E;
    rep.mu[0] = run.mu[0];
    rep.mu[1] = run.mu[1];
    rep.res = run.res;
    rep.seconds = std::chrono::duration<double>(t1 - t0).count();
    rep.ffts = run.ffts;
    rep.kernels = run.kernels;
    if (reports) reports[i] = rep;
    if (s != EGPE_OK) return s;
    if (rep.status != EGPE_OK && first_bad == EGPE_OK) first_bad = (egpe_status)rep.status;
  }
  return first_bad;
}

}  // extern "C"
