// Batched solver runtime: many independent instances (a parameter scan, with
// uneven grids) advanced together.  Each pass of a solver attempt is ONE
// launch per group of up to KB_MAX instances of the same grid shape: the
// launch's blockIdx.y selects the instance, whose kernel arguments (and
// column-pass tensor map) travel in the parameter block.  Every instance keeps
// its own workspace, reductions and on-device controller, so the arithmetic is
// exactly that of a single-instance solve.  The host replays a captured graph
// of one attempt for all live instances, gathers the instances' phases in one
// small copy per poll, and rebuilds the graph whenever instances finish, so
// finished instances drop out of the launches instead of occupying them.
// The launch chains of different groups are independent: with `concurrent`
// they are captured as parallel branches of the graph (one forked stream per
// group), each launch sized by its group's share of the live grid points, so
// the groups of uneven grids fill the GPU together; otherwise one after the
// other, each launch filling one wave by itself.
// Included by engine_f64.cu and engine_f32.cu only.
#pragma once
#include <map>
#include <memory>
#include <tuple>

#include "engine_impl.cuh"

namespace egpe {

template <class R> __global__ void phase_gather_kernel(DevState* const* sts, int n, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __ldcg(&sts[i]->phase);
}

template <class R> class BatchRunner {
 public:
  BatchRunner(const std::vector<Engine<R>*>& eng, cudaStream_t s, bool concurrent)
      : eng_(eng), stream_(s), concurrent_(concurrent) {}
  ~BatchRunner() { release(); }

  // Solves every instance from the state in its psi slot 0; options as in
  // Engine::solve.  runs[i] receives instance i's result.
  egpe_status solve(const egpe_solve_opts& o, int fp32_phase, int max_iter, double tol_res, double accept_rtol,
                    std::vector<SolveRun>& runs, egpe_trace_entry* trace_out, int trace_cap) {
    const int n = (int)eng_.size();
    runs.assign(n, SolveRun{});
    EGPE_TRY(alloc());
    egpe_solve_opts oo = o;
    oo.use_graph = 0;
    for (int i = 0; i < n; ++i)
      EGPE_TRY(eng_[i]->solve_begin(oo, fp32_phase, max_iter, tol_res, accept_rtol, i == 0 && trace_out != nullptr,
                                    trace_cap));
    std::vector<int> phase;
    EGPE_TRY(gather(phase));
    std::vector<int> active = live(phase);
    const int mode = o.precond;
    const int poll = std::max(1, o.poll_every);
    const long long max_launch = (long long)(max_iter + 2) * (long long)(o.armijo_max + 2) + 4;
    long long replays = 0, kernels = 0;
    while (!active.empty() && replays < max_launch) {
      if (active != built_) EGPE_TRY(rebuild(active, mode));
      for (int k = 0; k < poll; ++k) {
        EGPE_CUDA(cudaGraphLaunch(graph_, stream_));
        ++replays;
        kernels += per_replay_;
      }
      EGPE_TRY(gather(phase));
      active = live(phase);
    }
    for (int i = 0; i < n; ++i) {
      Engine<R>& e = *eng_[i];
      e.run_launches_ = replays;
      e.kernels_ += kernels;
      EGPE_TRY(e.solve_finish(runs[i], i == 0 ? trace_out : nullptr, trace_cap, 0));
    }
    return EGPE_OK;
  }

  int graph_builds() const { return builds_; }

 private:
  std::vector<Engine<R>*> eng_;
  cudaStream_t stream_ = nullptr;
  bool concurrent_ = false;
  std::vector<cudaStream_t> branch_;  // forked capture streams, one per group (concurrent mode)
  std::vector<cudaEvent_t> join_;     // [0]: fork point, [1 + g]: end of group g's chain
  cudaGraphExec_t graph_ = nullptr;
  std::vector<int> built_;
  long long per_replay_ = 0;
  int builds_ = 0;
  DevState** d_sts_ = nullptr;
  int* d_phase_ = nullptr;
  int* h_phase_ = nullptr;

  void release() {
    if (graph_) cudaGraphExecDestroy(graph_);
    graph_ = nullptr;
    for (cudaStream_t b : branch_) cudaStreamDestroy(b);
    for (cudaEvent_t e : join_) cudaEventDestroy(e);
    branch_.clear();
    join_.clear();
    if (d_sts_) cudaFree(d_sts_);
    if (d_phase_) cudaFree(d_phase_);
    if (h_phase_) cudaFreeHost(h_phase_);
    d_sts_ = nullptr;
    d_phase_ = nullptr;
    h_phase_ = nullptr;
  }

  egpe_status alloc() {
    if (d_sts_) return EGPE_OK;
    const int n = (int)eng_.size();
    std::vector<DevState*> h(n);
    for (int i = 0; i < n; ++i) h[i] = eng_[i]->st_;
    EGPE_CUDA(cudaMalloc(&d_sts_, n * sizeof(DevState*)));
    EGPE_CUDA(cudaMemcpy(d_sts_, h.data(), n * sizeof(DevState*), cudaMemcpyHostToDevice));
    EGPE_CUDA(cudaMalloc(&d_phase_, n * sizeof(int)));
    EGPE_CUDA(cudaMallocHost(&h_phase_, n * sizeof(int)));
    return EGPE_OK;
  }

  egpe_status gather(std::vector<int>& phase) {
    const int n = (int)eng_.size();
    phase_gather_kernel<R><<<(n + 127) / 128, 128, 0, stream_>>>(d_sts_, n, d_phase_);
    EGPE_CUDA(cudaGetLastError());
    EGPE_CUDA(cudaMemcpyAsync(h_phase_, d_phase_, n * sizeof(int), cudaMemcpyDeviceToHost, stream_));
    EGPE_CUDA(cudaStreamSynchronize(stream_));
    phase.assign(h_phase_, h_phase_ + n);
    return EGPE_OK;
  }

  static std::vector<int> live(const std::vector<int>& phase) {
    std::vector<int> a;
    for (int i = 0; i < (int)phase.size(); ++i)
      if (phase[i] != PH_DONE) a.push_back(i);
    return a;
  }

  // Groups the live instances by grid shape (chunks of at most KB_MAX),
  // records each one's attempt and captures one graph that launches every
  // pass once per chunk.
  egpe_status rebuild(const std::vector<int>& active, int mode) {
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;
    for (int i : active) groups[std::make_tuple(eng_[i]->nx, eng_[i]->ny, eng_[i]->nz)].push_back(i);
    struct Launch {
      const void* fn;
      dim3 grid;
      int block;
      size_t smem;
      std::unique_ptr<KBatch<R>> kb;
      int branch;
    };
    std::vector<Launch> launches;
    double live_points = 0.0;
    for (int i : active) live_points += (double)eng_[i]->N;
    int branch = 0;
    std::vector<std::vector<LaunchRec<R>>> recs;
    std::vector<std::vector<KArgs<R>>> args;
    for (auto& g : groups) {
      const std::vector<int>& ids = g.second;
      for (size_t c0 = 0; c0 < ids.size(); c0 += KB_MAX) {
        const int nc = (int)std::min<size_t>(KB_MAX, ids.size() - c0);
        recs.assign(nc, {});
        args.assign(nc, {});
        for (int c = 0; c < nc; ++c) EGPE_TRY(eng_[ids[c0 + c]]->record_attempt(mode, recs[c], args[c]));
        for (int c = 1; c < nc; ++c)
          if (recs[c].size() != recs[0].size()) {
            set_error_msg("batched solve: instances recorded different launch sequences");
            return EGPE_ERR_UNSUPPORTED;
          }
        Engine<R>& e0 = *eng_[ids[c0]];
        for (size_t j = 0; j < recs[0].size(); ++j) {
          const LaunchRec<R>& r0 = recs[0][j];
          Launch L;
          L.fn = r0.fn;
          L.block = r0.block;
          L.smem = r0.smem;
          L.kb.reset(new KBatch<R>());
          std::memset((void*)L.kb.get(), 0, sizeof(KBatch<R>));
          for (int c = 0; c < nc; ++c) {
            const LaunchRec<R>& rc = recs[c][j];
            if (rc.fn != r0.fn || (rc.tm == nullptr) != (r0.tm == nullptr)) {
              set_error_msg("batched solve: instances recorded different kernels");
              return EGPE_ERR_UNSUPPORTED;
            }
            L.kb->k[c] = args[c][rc.arg];
            if (rc.tm) L.kb->tm[c] = *rc.tm;
          }
          // sequential chunks: one full wave over the chunk's instances (a
          // rounded-up share would spill a few blocks into a second wave);
          // concurrent chunks: the wave shared in proportion to grid points
          const int occ = e0.occupancy(r0.fn, r0.block, r0.smem);
          const long long wave = (long long)occ * e0.nsm_;
          const long long fill = concurrent_ ? (long long)(wave * ((double)e0.N / live_points)) : wave / nc;
          const long long gx = std::max<long long>(1, std::min<long long>(r0.units, std::min<long long>(fill, 16384)));
          L.grid = dim3((unsigned)gx, (unsigned)nc, 1);
          L.branch = branch;
          launches.push_back(std::move(L));
        }
        ++branch;
      }
    }
    if (concurrent_) {
      // capture streams and events for every branch (kept across rebuilds)
      if (join_.empty()) {
        cudaEvent_t e;
        EGPE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        join_.push_back(e);
      }
      while ((int)branch_.size() < branch) {
        cudaStream_t b;
        cudaEvent_t e;
        EGPE_CUDA(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
        branch_.push_back(b);
        EGPE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        join_.push_back(e);
      }
    }
    if (graph_) cudaGraphExecDestroy(graph_);
    graph_ = nullptr;
    cudaGraph_t g = nullptr;
    EGPE_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    if (concurrent_) {
      // fork: every branch stream waits on the capture origin, then joins back
      le = cudaEventRecord(join_[0], stream_);
      for (int b = 0; b < branch && le == cudaSuccess; ++b) le = cudaStreamWaitEvent(branch_[b], join_[0], 0);
    }
    for (Launch& L : launches) {
      if (le != cudaSuccess) break;
      void* params[1] = {(void*)L.kb.get()};
      cudaStream_t s = concurrent_ ? branch_[L.branch] : stream_;
      le = cudaLaunchKernel(L.fn, L.grid, dim3((unsigned)L.block), params, L.smem, s);
    }
    if (concurrent_) {
      for (int b = 0; b < branch && le == cudaSuccess; ++b) {
        le = cudaEventRecord(join_[1 + b], branch_[b]);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(stream_, join_[1 + b], 0);
      }
    }
    cudaError_t ce = cudaStreamEndCapture(stream_, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      set_error(le != cudaSuccess ? "batched launch" : "cudaStreamEndCapture", le != cudaSuccess ? le : ce);
      return EGPE_ERR_CUDA;
    }
    cudaError_t ie = cudaGraphInstantiate(&graph_, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      graph_ = nullptr;
      set_error("cudaGraphInstantiate", ie);
      return EGPE_ERR_CUDA;
    }
    per_replay_ = (long long)launches.size();
    built_ = active;
    ++builds_;
    return EGPE_OK;
  }
};

template <class R>
egpe_status batch_solve(const std::vector<Engine<R>*>& eng, cudaStream_t s, const egpe_solve_opts& o, int fp32_phase,
                        int max_iter, double tol_res, double accept_rtol, std::vector<SolveRun>& runs,
                        egpe_trace_entry* trace_out, int trace_cap, int* graph_builds) {
  BatchRunner<R> br(eng, s, o.batch >= 2);
  const egpe_status st = br.solve(o, fp32_phase, max_iter, tol_res, accept_rtol, runs, trace_out, trace_cap);
  if (graph_builds) *graph_builds = br.graph_builds();
  return st;
}

}  // namespace egpe
