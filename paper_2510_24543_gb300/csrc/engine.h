// Host-side engine of one eGPE instance in one field precision: owns the
// device workspace, the twiddle and quadrature tables, the launch shapes and
// the captured CUDA graph of one solver attempt.  Implemented in engine_impl.cuh
// and instantiated for double and float in their own translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "egpe.h"
#include "common.cuh"

namespace egpe {

template <class R> struct KArgs;
template <class R> struct KBatch;
template <class R> class BatchRunner;

// One recorded launch of a pipeline pass (batched replay, see batch.cuh): the
// instance's kernel arguments and how to launch the pass for several
// instances at once.
template <class R> struct LaunchRec {
  int arg = -1;                       // index of its KArgs in the recording's argument list
  const CUtensorMap* tm = nullptr;    // column-pass tensor map (TMA launches)
  const void* fn = nullptr;           // the batched kernel: one KBatch<R> parameter
  int block = 0;
  size_t smem = 0;
  long long units = 0;                // blocks' worth of work per instance
  // launch-shape tuning (autotune): the single-instance kernels and shape data
  int kind = 0;                       // 0 row pass, 1 column pass, 2 pointwise
  const char* key = nullptr;          // identifies the op instantiation
  const char* name = nullptr;
  int L = 0;
  const void* fn1 = nullptr;          // row pass / plain column pass (KArgs parameter)
  const void* fn1_tma = nullptr;      // column pass fed by TMA (CUtensorMap, KArgs)
  int tpl = 0, max_threads = 0, mx = 0;
  size_t rowbytes = 0, smem_fixed = 0, smem_plain = 0, smem_tma = 0;
  long long rows = 0;
};

// Key of the tuning entry that sets the column tile width (kind 2).
inline const char* const kColBytesKey = "column tile row bytes";

// One tuned launch shape: rows per block (row passes), 1 = TMA-fed / 0 =
// plain loads (column passes), or the column tile row width in bytes.

struct TuneResult {
  std::string key, name;
  int L = 0, kind = 0, choice = 0, default_choice = 0;
  double ms_best = 0.0, ms_default = 0.0;
};

void set_error(const char* what, cudaError_t e);
void set_error_msg(const std::string& msg);

struct SolveRun {
  int status, n, attempts, restarts, armijo_total, trace_len, launches, phase;
  double E, mu[2], res;
  long long ffts, kernels;
};

template <class R> class Engine {
 public:
  using C = C2<R>;
  Engine() = default;
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;
  ~Engine() { destroy(); }

  egpe_status create(const egpe_grid& g, const egpe_params& p, cudaStream_t stream);
  void destroy();

  // Standalone evaluations (synchronous; device pointers of this precision).
  egpe_status energy_grad(const C* psi, egpe_energy_terms* out, C* grad);
  egpe_status line_coeffs(const C* psi, const C* p, double coeffs[3]);
  egpe_status precondition(int mode, const C* psi, const C* r, C* z);
  egpe_status retract(const C* psi, const C* p, const double theta[2], C* out);
  egpe_status fft(const C* in, C* out, int nf, int inverse);
  egpe_status normalise_current();
  // Partial derivatives of E at psi with respect to the parameters (index
  // EGPE_P_*), and an in-place change of the parameters (same grid).
  egpe_status param_grad(const C* psi, double out[EGPE_NPARAM]);
  egpe_status set_params(const egpe_params& p);

  // Solver: psi start must already be in psi buffer 0 (load_psi / cast).
  egpe_status load_psi(const void* src, cudaMemcpyKind kind);
  egpe_status store_psi(void* dst, cudaMemcpyKind kind);
  egpe_status solve(const egpe_solve_opts& o, int fp32_phase, int max_iter, double tol_res, double accept_rtol,
                    SolveRun& run, egpe_trace_entry* trace_out, int trace_cap, int trace_offset);
  // Per-kernel device times of `reps` solver attempts from psi (CUDA events
  // around every launch, no graph): names, mean ms and algorithmic bytes.
  egpe_status profile_attempt(const C* psi, int precond, int reps, std::vector<std::string>& names,
                              std::vector<double>& ms, std::vector<double>& bytes);
  // Stepping interface (the same phases egpe_ncg_solve runs): begin loads
  // nothing -- psi must be in slot 0 -- evaluates the start and prepares the
  // graph; launch enqueues attempts without waiting; finish reads the state.
  egpe_status solve_begin(const egpe_solve_opts& o, int fp32_phase, int max_iter, double tol_res,
                          double accept_rtol, bool want_trace, int trace_cap);
  egpe_status solve_launch(int attempts);
  egpe_status solve_poll(int& phase);
  egpe_status solve_finish(SolveRun& run, egpe_trace_entry* trace_out, int trace_cap, int trace_offset);
  // Imaginary-time evolution (the baseline of the paper's comparison): Strang
  // steps of size dtau from the state in slot 0 until |E^{k+1} - E^k| < tol_dE
  // or max_steps; the same begin / launch / poll / finish phases as the solver.
  egpe_status ite_begin(double dtau, double tol_dE, int max_steps, bool use_graph);
  egpe_status ite(double dtau, double tol_dE, int max_steps, int poll_every, bool use_graph, SolveRun& run);
  // Launch-shape autotuning: times every candidate shape of each kernel of one
  // attempt from psi (reps launches each, controller off) and keeps the fastest.
  egpe_status autotune(const C* psi, int precond, int reps, std::vector<TuneResult>& out);
  // Applies previously tuned shapes (by key); unknown keys are ignored.
  void set_tuning(const std::string& key, int choice) {
    if (key == kColBytesKey) return set_col_bytes(choice);
    tune_[key] = choice;
    drop_graphs();
  }
  void clear_tuning() {
    tune_.clear();
    set_col_bytes(EGPE_COL_BYTES);
    drop_graphs();
  }
  // Row width in bytes (64, 128 or 256; anything else: the default) of the
  // column-pass tiles of the power-of-two lengths; rebuilds the tensor maps.
  void set_col_bytes(int bytes);
  // Poll budget of the device-side TMA waits (default kTmaWaitPolls; 0 gives
  // up before the first poll, which tests use to reach the timeout path).
  void set_wait_limit(long long polls);
  // Captured graphs hold launch shapes: drop them when the shapes change.
  void drop_graphs();
  // Records (instead of launching) the kernels of one solver attempt.
  egpe_status record_attempt(int mode, std::vector<LaunchRec<R>>& recs, std::vector<KArgs<R>>& args);
  C* current_psi();  // valid after solve (device)
  C* psi_slot0();    // psi buffer 0 (start of a solve)

  size_t N = 0;
  int nx = 0, ny = 0, nz = 0;
  cudaStream_t stream = nullptr;
  double dV = 0.0;

 private:
  egpe_status enq_eg(int trial, int gate, int ctrl);
  egpe_status enq_pc(int mode, int gate, int ctrl, int rgiven);
  egpe_status enq_lc(int gate, int ctrl, int pgiven);
  egpe_status enq_attempt(int mode);
  egpe_status enq_kin(int potential, int gate);
  egpe_status enq_pg(int gate);
  egpe_status apply_params(const egpe_params& p);
  egpe_status enq_ite_step(int gate);
  egpe_status reset_state(const egpe_solve_opts* o, int fp32_phase, int max_iter, double tol_res,
                          double accept_rtol);
  egpe_status read_state(DevState& hs, bool report_timeout = true);
  template <class Op> egpe_status launch_x(KArgs<R> a);
  egpe_status launch_point(void (*kern)(KArgs<R>), void (*kern_b)(KBatch<R>), const char* name, double bytes,
                           const KArgs<R>& a, long long units);
  egpe_status record(const KArgs<R>& a, const CUtensorMap* tm, const void* fn, int block, size_t smem,
                     long long units);
  template <class Op> egpe_status launch_col(KArgs<R> a, const CUtensorMap* tm);
  template <template <class, int> class OpT> egpe_status dispatch_x(int L, const KArgs<R>& a);
  template <template <class, int> class OpT> egpe_status dispatch_col(int L, const KArgs<R>& a, const CUtensorMap* tm);
  egpe_status plain_x(int inverse, const KArgs<R>& a);
  egpe_status plain_col(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm);
  // Launches for a list of line lengths (engine_impl.cuh).  The lengths 48 and
  // 96 (suffix mr), 80 (mr5) and 128, 256 (big) are compiled in translation
  // units of their own (engine_ext.cuh) to spread the compile time.
  template <template <class, int> class OpT, int... Ls> egpe_status dispatch_x_in(int L, const KArgs<R>& a);
  template <template <class, int> class OpT, int... Ls>
  egpe_status dispatch_col_in(int L, const KArgs<R>& a, const CUtensorMap* tm);
  template <int... Ls> egpe_status plain_x_in(int inverse, const KArgs<R>& a);
  template <int... Ls> egpe_status plain_col_in(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm);
  template <template <class, int> class OpT> egpe_status dispatch_x_mr(int L, const KArgs<R>& a);
  template <template <class, int> class OpT>
  egpe_status dispatch_col_mr(int L, const KArgs<R>& a, const CUtensorMap* tm);
  egpe_status plain_x_mr(int inverse, const KArgs<R>& a);
  egpe_status plain_col_mr(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm);
  template <template <class, int> class OpT> egpe_status dispatch_x_mr5(int L, const KArgs<R>& a);
  template <template <class, int> class OpT>
  egpe_status dispatch_col_mr5(int L, const KArgs<R>& a, const CUtensorMap* tm);
  egpe_status plain_x_mr5(int inverse, const KArgs<R>& a);
  egpe_status plain_col_mr5(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm);
  template <template <class, int> class OpT> egpe_status dispatch_x_big(int L, const KArgs<R>& a);
  template <template <class, int> class OpT>
  egpe_status dispatch_col_big(int L, const KArgs<R>& a, const CUtensorMap* tm);
  egpe_status plain_x_big(int inverse, const KArgs<R>& a);
  egpe_status plain_col_big(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm);
  const CUtensorMap* tmy() const { return have_maps_ ? &tmW_y_ : nullptr; }
  const CUtensorMap* tmz() const { return have_maps_ ? &tmW_z_ : nullptr; }
  int occupancy(const void* fn, int block, size_t smem);
  void t_begin(const char* name, int L, double bytes);
  void t_end();

  struct KTime {
    std::string name;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<KTime> tlog_;
  bool timing_ = false;
  // strided passes fed by TMA (tensor maps over the workspace W)
  bool use_tma_ = true;
  bool have_maps_ = false;
  int col_bytes_ = EGPE_COL_BYTES;  // column tile row width (set_col_bytes)
  CUtensorMap tmW_y_{}, tmW_z_{};
  size_t tpos_ = 0;

  KArgs<R>* base_ = nullptr;  // host copy of the common kernel arguments
  egpe_grid grid_{};
  egpe_params prm_{};
  void* arena_ = nullptr;
  C* twx_ = nullptr;
  C* twy_ = nullptr;
  C* twz_ = nullptr;
  LhyNode<R>* nodes_ = nullptr;
  int nodes_q_ = 0;
  LhyNode<R>* xnodes_ = nullptr;    // nodes evaluated exactly beside the LHY table
  R* tab_ = nullptr;                // LHY interpolation table (host_tables.h)
  size_t tab_elems_ = 0;
  double* partials_ = nullptr;
  unsigned* counter_ = nullptr;
  DevState* st_ = nullptr;
  DevState* st_host_ = nullptr;  // pinned mirror
  TraceDev* trace_ = nullptr;
  int trace_alloc_ = 0;
  int nsm_ = 0;
  int Qm_ = 0;  // LHY nodes with det eta > 0 (stored first)
  long long kernels_ = 0;
  std::unordered_map<unsigned long long, int> occ_;
  cudaGraphExec_t graph_[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int run_mode_ = 0, run_graph_ = 1;
  long long run_k0_ = 0, run_launches_ = 0, per_attempt_ = 0;
  int graph_max_iter_[5] = {0, 0, 0, 0, 0};
  R* kin_tab_ = nullptr;            // ITE kinetic half-step factors and dtau
  std::vector<R> kin_host_;
  cudaGraphExec_t graph_ite_ = nullptr;
  int ite_per_step_ = 0;
  bool run_ite_ = false;
  std::unordered_map<std::string, int> tune_;  // tuned launch shapes by op key
  std::vector<LaunchRec<R>>* rec_ = nullptr;  // recording mode when set
  std::vector<KArgs<R>>* rec_args_ = nullptr;
  friend class BatchRunner<R>;
};

// Solves all instances together with batched launches (batch.cuh).  Engines
// of one precision on stream s; psi starts in each engine's slot 0.
template <class R>
egpe_status batch_solve(const std::vector<Engine<R>*>& eng, cudaStream_t s, const egpe_solve_opts& o, int fp32_phase,
                        int max_iter, double tol_res, double accept_rtol, std::vector<SolveRun>& runs,
                        egpe_trace_entry* trace_out, int trace_cap, int* graph_builds);

}  // namespace egpe
