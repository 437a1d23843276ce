// Implementation of Engine<R> (see engine.h).  Included by engine_f64.cu and
// engine_f32.cu only.
#pragma once
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <limits>
#include <mutex>
#include <typeinfo>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "host_tables.h"
#include "kernels.cuh"

namespace egpe {

#define EGPE_CUDA(call)                       \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) {                  \
      set_error(#call, e_);                   \
      return e_ == cudaErrorMemoryAllocation ? EGPE_ERR_OOM : EGPE_ERR_CUDA; \
    }                                         \
  } while (0)

#define EGPE_TRY(x)                 \
  do {                              \
    egpe_status s_ = (x);           \
    if (s_ != EGPE_OK) return s_;   \
  } while (0)

typedef CUresult (*TmaEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library).
static TmaEncodeFn tma_encode_fn() {
  static TmaEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmaEncodeFn>(p);
  }
  return fn;
}

// Columns per tile of the strided passes: tile rows of col_bytes (64, 128 or
// 256; EGPE_COL_BYTES = 128, one cache line, unless the autotuner chose
// another width) for the power-of-two lengths, whose kernels are bound to 512
// threads, and of 128 bytes for the mixed-radix lengths (bound to that width);
// whole warps, and the TMA-fed pass's tiles within 200 KB of shared memory.
template <class C> static inline int col_tile_width(int L, int nx, int col_bytes) {
  const int TPL = L / 8;
  const bool pow2 = (L & (L - 1)) == 0;
  int M = pow2 ? std::min((int)(col_bytes / sizeof(C)), 512 / TPL) : (int)(128 / sizeof(C));
  while (pow2 && M > 1 && (size_t)(kColStages + 1) * M * L * sizeof(C) > 200 * 1024) M /= 2;
  M = std::min(std::max(M, whole_warp_rows(L)), nx);
  while (M > whole_warp_rows(L) && nx % M != 0) M /= 2;  // whole tiles across x
  return M;
}

// Tensor map of `nfields` consecutive complex fields (nx, ny, nz), box = one
// column tile of the y (axis 1) or z (axis 2) pass.
template <class C>
static bool make_col_map(CUtensorMap& tm, const void* base, int nx, int ny, int nz, int nfields, int axis,
                         int col_bytes) {
  TmaEncodeFn fn = tma_encode_fn();
  if (!fn) return false;
  const int L = axis == 1 ? ny : nz;
  const int M = col_tile_width<C>(L, nx, col_bytes);
  const cuuint64_t esz = sizeof(C) / 8;
  cuuint64_t dims[3] = {(cuuint64_t)nx * esz, (cuuint64_t)ny, (cuuint64_t)nz * nfields};
  cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(C), (cuuint64_t)nx * ny * sizeof(C)};
  cuuint32_t box[3] = {(cuuint32_t)(M * esz), axis == 1 ? (cuuint32_t)L : 1u, axis == 1 ? 1u : (cuuint32_t)L};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(&tm, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Lets a kernel take every byte of dynamic shared memory the device allows.
// The attribute belongs to the function, process-wide, so it is set once to
// the maximum rather than per launch shape (engines that launch one kernel
// with different shapes would otherwise lower it under each other).
inline cudaError_t allow_max_dynamic_smem(const void* fn) {
  static std::mutex mu;
  static std::unordered_map<const void*, cudaError_t> done;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(fn);
  if (it != done.end()) return it->second;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  done[fn] = e;
  return e;
}

static inline bool supported_len(int n) {
  return n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 48 || n == 80 || n == 96;
}

// Couplings, trap and LHY node table of the instance (at create, and again
// when the parameters change: egpe_set_params).  The node table keeps its
// nodes with det eta > 0 first (Qm_ of them).
template <class R> egpe_status Engine<R>::apply_params(const egpe_params& p) {
  prm_ = p;
  const int Q = p.lhy_nodes;
  std::vector<LhyNode<R>> h(Q);
  Qm_ = lhy_node_table<R>(p, h.data());
  // kernels still reading the old table finish first
  EGPE_CUDA(cudaStreamSynchronize(stream));
  if (nodes_ && nodes_q_ != Q) {
    cudaFree(nodes_);
    nodes_ = nullptr;
  }
  if (!nodes_) {
    EGPE_CUDA(cudaMalloc(&nodes_, Q * sizeof(LhyNode<R>)));
    nodes_q_ = Q;
  }
  EGPE_CUDA(cudaMemcpy(nodes_, h.data(), Q * sizeof(LhyNode<R>), cudaMemcpyHostToDevice));
  // interpolated LHY sums and the nodes left to exact evaluation
  const LhyTableHost T = lhy_interp_table_cached<R>(p);
  static_assert(TabSpec<R>::deg + 1 == LhyTabDim<R>::coef, "table layout");
  std::vector<R> tab(T.coef.begin(), T.coef.end());
  if (tab_ && tab_elems_ != tab.size()) {
    cudaFree(tab_);
    tab_ = nullptr;
    tab_elems_ = 0;
  }
  if (!tab_ && !tab.empty()) {
    EGPE_CUDA(cudaMalloc(&tab_, tab.size() * sizeof(R)));
    tab_elems_ = tab.size();
  }
  if (!tab.empty()) EGPE_CUDA(cudaMemcpy(tab_, tab.data(), tab.size() * sizeof(R), cudaMemcpyHostToDevice));
  std::vector<LhyNode<R>> xh(std::max<size_t>(T.exact.size(), 1));
  const int Qxm = lhy_node_table<R>(p, xh.data(), &T.exact);
  if (!xnodes_) EGPE_CUDA(cudaMalloc(&xnodes_, 64 * sizeof(LhyNode<R>)));
  if (!T.exact.empty())
    EGPE_CUDA(cudaMemcpy(xnodes_, xh.data(), T.exact.size() * sizeof(LhyNode<R>), cudaMemcpyHostToDevice));
  KArgs<R>& a = *base_;
  a.xnodes = xnodes_;
  a.Qx = (int)T.exact.size();
  a.Qxm = Qxm;
  a.tab.tab = T.ni ? tab_ : nullptr;
  a.tab.ni = T.ni;
  a.tab.tscale = (R)(T.ni * 1.4142135623730950488);
  a.vx = (R)(0.5 * p.trap[0] * p.trap[0]);
  a.vy = (R)(0.5 * p.trap[1] * p.trap[1]);
  a.vz = (R)(0.5 * p.trap[2] * p.trap[2]);
  a.g11 = (R)p.g[0][0];
  a.g12 = (R)p.g[0][1];
  a.g21 = (R)p.g[1][0];
  a.g22 = (R)p.g[1][1];
  a.d11 = (R)p.gdd[0][0];
  a.d12 = (R)p.gdd[0][1];
  a.d21 = (R)p.gdd[1][0];
  a.d22 = (R)p.gdd[1][1];
  a.Q = Q;
  a.Qm = Qm_;
  a.nodes = nodes_;
  a.nskip = (R)lhy_skip_threshold(p);
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::set_params(const egpe_params& p) {
  EGPE_TRY(apply_params(p));
  drop_graphs();  // captured launches hold the old couplings
  return EGPE_OK;
}

// Parameter-derivative pass: one packed density field through the dipolar
// kernel (4 transform passes) and the sums of the last row pass.
template <class R> egpe_status Engine<R>::enq_pg(int gate) {
  KArgs<R> a = *base_;
  a.gate = gate;
  a.flag = 0;
  a.ctrl = 0;
  a.nf = 1;
  a.f0 = 0;
  EGPE_TRY(dispatch_x<XFwdPG>(nx, a));
  KArgs<R> y = a;
  y.gin = a.W;
  y.gout = a.W;
  EGPE_TRY(plain_col(1, 0, y, tmy()));
  EGPE_TRY(dispatch_col<ZPg>(nz, a, tmz()));
  EGPE_TRY(plain_col(1, 1, y, tmy()));
  return dispatch_x<XInvPG>(nx, a);
}

template <class R> egpe_status Engine<R>::param_grad(const C* psi, double out[EGPE_NPARAM]) {
  EGPE_TRY(reset_state(nullptr, 0, 0, 0.0, 0.0));
  EGPE_CUDA(cudaMemcpyAsync(base_->psi[0], psi, 2 * N * sizeof(C), cudaMemcpyDeviceToDevice, stream));
  EGPE_TRY(enq_pg(GATE_ALWAYS));
  DevState hs;
  EGPE_TRY(read_state(hs));
  const double* s = hs.pg;
  const double kap = prm_.lhy_kappa, eta = prm_.lhy_eta_scale;
  out[EGPE_P_G11] = dV * (0.5 * s[PG_N11] + s[PG_L11]);
  out[EGPE_P_G12] = dV * (s[PG_N12] + s[PG_L12]);
  out[EGPE_P_G22] = dV * (0.5 * s[PG_N22] + s[PG_L22]);
  out[EGPE_P_GDD11] = dV * (0.5 * s[PG_K11] + s[PG_M11]);
  out[EGPE_P_GDD12] = dV * (s[PG_K12] + s[PG_M12]);
  out[EGPE_P_GDD22] = dV * (0.5 * s[PG_K22] + s[PG_M22]);
  out[EGPE_P_KAPPA] = kap != 0.0 ? dV * s[PG_F] / kap : std::numeric_limits<double>::quiet_NaN();
  out[EGPE_P_ETA_S] = -2.5 * dV * s[PG_F] / eta;
  out[EGPE_P_TRAP_X] = prm_.trap[0] * dV * s[PG_X2];
  out[EGPE_P_TRAP_Y] = prm_.trap[1] * dV * s[PG_Y2];
  out[EGPE_P_TRAP_Z] = prm_.trap[2] * dV * s[PG_Z2];
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::create(const egpe_grid& g, const egpe_params& p, cudaStream_t s) {
  grid_ = g;
  prm_ = p;
  stream = s;
  nx = g.n[0];
  ny = g.n[1];
  nz = g.n[2];
  N = (size_t)nx * ny * nz;
  int dev = 0;
  EGPE_CUDA(cudaGetDevice(&dev));
  EGPE_CUDA(cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev));
  const size_t fb = N * sizeof(C);
  // psi[2], hp[2], ax[2], rb[2], pb[2]: 2 fields each; z: 2; W: 3  -> 25 fields
  EGPE_CUDA(cudaMalloc(&arena_, 25 * fb));
  EGPE_CUDA(cudaMemsetAsync(arena_, 0, 25 * fb, stream));
  C* f = reinterpret_cast<C*>(arena_);
  base_ = new KArgs<R>();
  std::memset((void*)base_, 0, sizeof(KArgs<R>));
  KArgs<R>& a = *base_;
  for (int b = 0; b < 2; ++b) a.psi[b] = f + (0 + 2 * b) * N;
  for (int b = 0; b < 2; ++b) a.hp[b] = f + (4 + 2 * b) * N;
  for (int b = 0; b < 2; ++b) a.ax[b] = f + (8 + 2 * b) * N;
  for (int b = 0; b < 2; ++b) a.rb[b] = f + (12 + 2 * b) * N;
  for (int b = 0; b < 2; ++b) a.pb[b] = f + (16 + 2 * b) * N;
  a.z = f + 20 * N;
  a.W = f + 22 * N;
  // twiddles W_L^m = exp(-2 pi i m / L), long double on the host
  C** tws[3] = {&twx_, &twy_, &twz_};
  for (int ax = 0; ax < 3; ++ax) {
    const int L = g.n[ax];
    std::vector<C> h(L);
    twiddle_table<R>(L, h.data());
    EGPE_CUDA(cudaMalloc(tws[ax], L * sizeof(C)));
    EGPE_CUDA(cudaMemcpy(*tws[ax], h.data(), L * sizeof(C), cudaMemcpyHostToDevice));
  }
  EGPE_CUDA(cudaMalloc(&partials_, (size_t)16384 * MAX_NS * sizeof(double)));
  EGPE_CUDA(cudaMalloc(&counter_, 64 * sizeof(unsigned)));
  EGPE_CUDA(cudaMemset(counter_, 0, 64 * sizeof(unsigned)));
  EGPE_CUDA(cudaMalloc(&st_, sizeof(DevState)));
  EGPE_CUDA(cudaMallocHost(&st_host_, sizeof(DevState)));
  EGPE_CUDA(cudaMalloc(&kin_tab_, (size_t)(nx + ny + nz + 1) * sizeof(R)));
  EGPE_CUDA(cudaMemsetAsync(kin_tab_, 0, (size_t)(nx + ny + nz + 1) * sizeof(R), stream));
  const double hx = 2.0 * g.L[0] / nx, hy = 2.0 * g.L[1] / ny, hz = 2.0 * g.L[2] / nz;
  dV = hx * hy * hz;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.N = (int)N;
  a.hx = (R)hx;
  a.hy = (R)hy;
  a.hz = (R)hz;
  a.Lx = (R)g.L[0];
  a.Ly = (R)g.L[1];
  a.Lz = (R)g.L[2];
  const double pi = 3.14159265358979323846;
  a.dkx = (R)(pi / g.L[0]);
  a.dky = (R)(pi / g.L[1]);
  a.dkz = (R)(pi / g.L[2]);
  a.invN = (R)(1.0 / (double)N);
  EGPE_TRY(apply_params(p));
  a.twx = twx_;
  a.twy = twy_;
  a.twz = twz_;
  a.partials = partials_;
  a.counter = counter_;
  a.st = st_;
  a.trace = nullptr;
  a.kin_tab = kin_tab_;
  a.wait_polls = kTmaWaitPolls;
  a.gate = GATE_ALWAYS;
  have_maps_ = make_col_map<C>(tmW_y_, a.W, nx, ny, nz, 3, 1, col_bytes_) &&
               make_col_map<C>(tmW_z_, a.W, nx, ny, nz, 3, 2, col_bytes_);
  return reset_state(nullptr, 0, 0, 0.0, 0.0);
}

template <class R> void Engine<R>::set_col_bytes(int b) {
  if (b != 64 && b != 128 && b != 256) b = EGPE_COL_BYTES;
  if (b == col_bytes_) return;
  col_bytes_ = b;
  have_maps_ = make_col_map<C>(tmW_y_, base_->W, nx, ny, nz, 3, 1, b) &&
               make_col_map<C>(tmW_z_, base_->W, nx, ny, nz, 3, 2, b);
  drop_graphs();
}

template <class R> void Engine<R>::set_wait_limit(long long polls) {
  base_->wait_polls = polls;
  drop_graphs();  // captured launches hold the old budget
}

template <class R> void Engine<R>::drop_graphs() {
  for (auto& gx : graph_)
    if (gx) {
      cudaGraphExecDestroy(gx);
      gx = nullptr;
    }
  if (graph_ite_) cudaGraphExecDestroy(graph_ite_);
  graph_ite_ = nullptr;
}

template <class R> void Engine<R>::destroy() {
  for (auto& k : tlog_) {
    cudaEventDestroy(k.a);
    cudaEventDestroy(k.b);
  }
  tlog_.clear();
  for (auto& gx : graph_)
    if (gx) {
      cudaGraphExecDestroy(gx);
      gx = nullptr;
    }
  if (graph_ite_) cudaGraphExecDestroy(graph_ite_);
  graph_ite_ = nullptr;
  if (kin_tab_) cudaFree(kin_tab_);
  kin_tab_ = nullptr;
  if (arena_) cudaFree(arena_);
  if (twx_) cudaFree(twx_);
  if (twy_) cudaFree(twy_);
  if (twz_) cudaFree(twz_);
  if (nodes_) cudaFree(nodes_);
  if (xnodes_) cudaFree(xnodes_);
  if (tab_) cudaFree(tab_);
  if (partials_) cudaFree(partials_);
  if (counter_) cudaFree(counter_);
  if (st_) cudaFree(st_);
  if (st_host_) cudaFreeHost(st_host_);
  if (trace_) cudaFree(trace_);
  delete base_;
  arena_ = nullptr;
  twx_ = twy_ = twz_ = nullptr;
  nodes_ = nullptr;
  xnodes_ = nullptr;
  tab_ = nullptr;
  tab_elems_ = 0;
  partials_ = nullptr;
  counter_ = nullptr;
  st_ = nullptr;
  st_host_ = nullptr;
  trace_ = nullptr;
  base_ = nullptr;
}

// Status of the launch just issued, naming the pass and its shape on failure.
// Passes run whole warps (full-mask shuffles); the geometry rules guarantee it.
static inline egpe_status check_whole_warps(const char* name, int L, int block) {
  if (block % 32 == 0) return EGPE_OK;
  set_error_msg(std::string(name) + " L=" + std::to_string(L) + ": block of " + std::to_string(block) +
                " threads is not whole warps");
  return EGPE_ERR_UNSUPPORTED;
}

static inline egpe_status launch_status(const char* name, int L, int block, size_t smem) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return EGPE_OK;
  set_error_msg(std::string("launch of ") + name + " L=" + std::to_string(L) + " (block " + std::to_string(block) +
                ", " + std::to_string(smem) + " B shared): " + cudaGetErrorString(e));
  return EGPE_ERR_CUDA;
}

template <class R> int Engine<R>::occupancy(const void* fn, int block, size_t smem) {
  const unsigned long long key = ((unsigned long long)(uintptr_t)fn) ^ ((unsigned long long)block << 48) ^
                                 ((unsigned long long)smem << 20);
  auto it = occ_.find(key);
  if (it != occ_.end()) return it->second;
  if (smem > 48 * 1024) allow_max_dynamic_smem(fn);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, smem) != cudaSuccess || occ < 1) occ = 1;
  occ_[key] = occ;
  return occ;
}

template <class R> void Engine<R>::t_begin(const char* name, int L, double bytes) {
  if (tpos_ >= tlog_.size()) {
    KTime k;
    cudaEventCreate(&k.a);
    cudaEventCreate(&k.b);
    tlog_.push_back(k);
  }
  KTime& k = tlog_[tpos_];
  k.name = std::string(name) + (L ? " L=" + std::to_string(L) : std::string());
  k.bytes = bytes;
  cudaEventRecord(k.a, stream);
}

template <class R> void Engine<R>::t_end() {
  cudaEventRecord(tlog_[tpos_].b, stream);
  ++tpos_;
}

template <class R>
egpe_status Engine<R>::profile_attempt(const C* psi, int precond, int reps, std::vector<std::string>& names,
                                       std::vector<double>& ms, std::vector<double>& bytes) {
  egpe_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  o.precond = precond;
  o.restart_period = 20;
  o.armijo_max = 30;
  o.armijo_c1 = 1e-4;
  o.theta_max = 1.5707963267948966;
  o.pv_floor = 1e-2;
  EGPE_CUDA(cudaMemcpyAsync(base_->psi[0], psi, 2 * N * sizeof(C), cudaMemcpyDeviceToDevice, stream));
  EGPE_TRY(reset_state(&o, sizeof(R) == 4, 1 << 30, 0.0, sizeof(R) == 4 ? 1e-6 : 1e-13));
  EGPE_CUDA(cudaMemsetAsync(base_->rb[0], 0, 8 * N * sizeof(C), stream));
  EGPE_TRY(enq_eg(0, GATE_ALWAYS, 1));
  EGPE_CUDA(cudaStreamSynchronize(stream));
  names.clear();
  ms.clear();
  bytes.clear();
  timing_ = true;
  for (int r = 0; r < reps; ++r) {
    tpos_ = 0;
    egpe_status s = enq_attempt(o.precond);
    if (s != EGPE_OK) {
      timing_ = false;
      return s;
    }
    EGPE_CUDA(cudaStreamSynchronize(stream));
    if (names.empty()) {
      for (size_t k = 0; k < tpos_; ++k) {
        names.push_back(tlog_[k].name);
        bytes.push_back(tlog_[k].bytes);
        ms.push_back(0.0);
      }
    }
    for (size_t k = 0; k < tpos_ && k < ms.size(); ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, tlog_[k].a, tlog_[k].b);
      ms[k] += t / reps;
    }
  }
  timing_ = false;
  return EGPE_OK;
}

// The batched kernel of a row pass (one pass for several instances).
template <class Op> static const void* xb_fn() {
  if constexpr (MinBlocks<Op>::v > 1) return (const void*)xpass_kernel_bmb<Op>;
  else return (const void*)xpass_kernel_b<Op>;
}

template <class R>
egpe_status Engine<R>::record(const KArgs<R>& a, const CUtensorMap* tm, const void* fn, int block, size_t smem,
                              long long units) {
  LaunchRec<R> r;
  r.arg = (int)rec_args_->size();
  rec_args_->push_back(a);
  r.tm = tm;
  r.fn = fn;
  r.block = block;
  r.smem = smem;
  r.units = units;
  rec_->push_back(r);
  return fn ? EGPE_OK : EGPE_ERR_UNSUPPORTED;
}

template <class R>
egpe_status Engine<R>::record_attempt(int mode, std::vector<LaunchRec<R>>& recs, std::vector<KArgs<R>>& args) {
  recs.clear();
  args.clear();
  rec_ = &recs;
  rec_args_ = &args;
  const egpe_status s = enq_attempt(mode);
  rec_ = nullptr;
  rec_args_ = nullptr;
  return s;
}

// Launch-shape autotuning.  The kernels of one attempt are recorded and the
// whole sequence is replayed (controller off, gates open) with CUDA events
// around it, so each kernel runs with the caches its predecessors leave, as in
// a solve; a kernel timed alone finds its own inputs in L2 and prefers shapes
// that lose in the pipeline.  Candidates are tried one op key at a time
// (coordinate descent over the keys in launch order), then the column tile
// width; a candidate replaces the current choice only if the sequence gets
// faster by more than 0.3%.  Choices go to tune_ (by op key) and col_bytes_,
// and are used by every later launch, recording and graph capture.
template <class R>
egpe_status Engine<R>::autotune(const C* psi, int precond, int reps, std::vector<TuneResult>& out) {
  out.clear();
  reps = std::max(1, reps);
  egpe_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  o.precond = precond;
  o.restart_period = 20;
  o.armijo_max = 30;
  o.armijo_c1 = 1e-4;
  o.theta_max = 1.5707963267948966;
  o.pv_floor = 1e-2;
  EGPE_CUDA(cudaMemcpyAsync(base_->psi[0], psi, 2 * N * sizeof(C), cudaMemcpyDeviceToDevice, stream));
  EGPE_TRY(reset_state(&o, sizeof(R) == 4, 1 << 30, 0.0, sizeof(R) == 4 ? 1e-6 : 1e-13));
  EGPE_CUDA(cudaMemsetAsync(base_->rb[0], 0, 8 * N * sizeof(C), stream));
  EGPE_TRY(enq_eg(0, GATE_ALWAYS, 1));
  EGPE_TRY(enq_attempt(o.precond));  // realistic coefficients in the state
  EGPE_CUDA(cudaStreamSynchronize(stream));
  tune_.clear();
  set_col_bytes(EGPE_COL_BYTES);
  std::vector<LaunchRec<R>> recs;
  std::vector<KArgs<R>> args;
  EGPE_TRY(record_attempt(o.precond, recs, args));
  cudaEvent_t e0, e1;
  EGPE_CUDA(cudaEventCreate(&e0));
  EGPE_CUDA(cudaEventCreate(&e1));
  egpe_status st = EGPE_OK;
  // shape of a recorded launch under the current choices (kind 0/1 only)
  auto choice_of = [&](const LaunchRec<R>& r) {
    auto it = tune_.find(r.key);
    return it != tune_.end() ? it->second : r.mx;
  };
  // min over reps of the device time of the whole recorded sequence
  auto time_seq = [&](const std::vector<LaunchRec<R>>& rs, const std::vector<KArgs<R>>& as) -> double {
    double tmin = 1e30;
    for (int k = 0; k <= reps && st == EGPE_OK; ++k) {
      cudaEventRecord(e0, stream);
      for (const LaunchRec<R>& r : rs) {
        if (r.kind > 1 || !r.key) continue;  // pointwise passes have one shape
        KArgs<R> a = as[r.arg];
        a.ctrl = 0;
        a.gate = GATE_ALWAYS;
        const int c = choice_of(r);
        const void* fn;
        int block;
        size_t smem;
        long long units;
        CUtensorMap tmc;
        void* params[2];
        if (r.kind == 0) {
          a.MX = c;
          fn = r.fn1;
          block = c * r.tpl;
          smem = r.smem_fixed + (size_t)c * r.rowbytes;
          units = (r.rows + c - 1) / c;
          params[0] = &a;
        } else {
          const bool tma = c != 0 && r.tm && use_tma_;
          fn = tma ? r.fn1_tma : r.fn1;
          block = r.block;
          smem = tma ? r.smem_tma : r.smem_plain;
          units = r.units;
          if (tma) {
            tmc = *r.tm;
            params[0] = &tmc;
            params[1] = &a;
          } else {
            params[0] = &a;
          }
        }
        const int occ = occupancy(fn, block, smem);
        const dim3 grid((unsigned)std::max<long long>(1, std::min<long long>(units, std::min(occ * nsm_, 16384))));
        const cudaError_t le = cudaLaunchKernel(fn, grid, dim3((unsigned)block), params, smem, stream);
        if (le != cudaSuccess) {
          set_error("autotune launch", le);
          st = EGPE_ERR_CUDA;
          break;
        }
      }
      cudaEventRecord(e1, stream);
      if (st != EGPE_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        set_error("autotune", cudaGetLastError());
        st = EGPE_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (k > 0) tmin = std::min(tmin, (double)ms);  // the first replay warms up
    }
    return tmin;
  };
  constexpr double kGain = 0.997;  // a change must save more than 0.3%
  double cur = time_seq(recs, args);
  std::unordered_map<std::string, int> seen;
  for (const LaunchRec<R>& r : recs) {
    if (st != EGPE_OK) break;
    if (r.kind > 1 || !r.key || seen.count(r.key)) continue;
    seen[r.key] = 1;
    std::vector<int> cand;
    if (r.kind == 0) {
      for (int mx = r.mx; mx >= 1; mx /= 2)
        if ((mx * r.tpl) % 32 == 0) cand.push_back(mx);  // whole warps only
      const int up = r.mx * 2;
      if (up * r.tpl <= r.max_threads && (size_t)up * r.rowbytes + r.smem_fixed <= 200 * 1024) cand.push_back(up);
    } else {
      cand.push_back(0);
      if (r.tm && use_tma_) cand.push_back(1);
    }
    TuneResult tr;
    tr.key = r.key;
    tr.name = r.name ? r.name : "";
    tr.L = r.L;
    tr.kind = r.kind;
    tr.default_choice = r.mx;
    tr.choice = r.mx;
    tr.ms_default = tr.ms_best = cur;
    for (int c : cand) {
      if (c == r.mx) continue;
      tune_[r.key] = c;
      const double t = time_seq(recs, args);
      if (st != EGPE_OK) break;
      if (t < kGain * tr.ms_best) {
        tr.ms_best = t;
        tr.choice = c;
      }
    }
    if (st != EGPE_OK) break;
    tune_[r.key] = tr.choice;
    cur = tr.ms_best;
    out.push_back(tr);
  }
  // the column tile width: re-recorded at each width (the shapes change)
  if (st == EGPE_OK) {
    TuneResult tr;
    tr.key = kColBytesKey;
    tr.name = "column tile row bytes";
    tr.kind = 2;
    tr.default_choice = tr.choice = EGPE_COL_BYTES;
    tr.ms_default = tr.ms_best = cur;
    for (int w : {64, 256}) {
      set_col_bytes(w);
      std::vector<LaunchRec<R>> wr;
      std::vector<KArgs<R>> wa;
      st = record_attempt(o.precond, wr, wa);
      if (st != EGPE_OK) break;
      const double t = time_seq(wr, wa);
      if (st != EGPE_OK) break;
      if (t < kGain * tr.ms_best) {
        tr.ms_best = t;
        tr.choice = w;
      }
    }
    set_col_bytes(tr.choice);
    if (st == EGPE_OK) out.push_back(tr);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  EGPE_TRY(st);
  drop_graphs();
  // leave a clean state: the next solve starts from its own psi
  EGPE_TRY(reset_state(nullptr, 0, 0, 0.0, 0.0));
  EGPE_CUDA(cudaStreamSynchronize(stream));
  return EGPE_OK;
}

template <class R>
egpe_status Engine<R>::launch_point(void (*kern)(KArgs<R>), void (*kern_b)(KBatch<R>), const char* name,
                                    double bytes, const KArgs<R>& a, long long units) {
  const int occ = occupancy((const void*)kern, 256, 0);
  const int grid = (int)std::min<long long>(units, (long long)std::min(occ * nsm_, 16384));
  if (rec_) return record(a, nullptr, (const void*)kern_b, 256, 0, units);
  if (timing_) t_begin(name, 0, bytes);
  kern<<<grid, 256, 0, stream>>>(a);
  if (timing_) t_end();
  ++kernels_;
  EGPE_CUDA(cudaGetLastError());
  return EGPE_OK;
}

template <class R> template <class Op> egpe_status Engine<R>::launch_x(KArgs<R> a) {
  constexpr int L = Op::L, TPL = L / 8, NF = Op::NF, NS = Op::NS;
  constexpr int LP = row_len_padded<R, L>();
  const size_t rowbytes = (size_t)NF * LP * sizeof(C);
  int mx = whole_warp_rows(L);
  while ((mx * 2) * TPL <= MaxThreads<Op>::v && (size_t)(mx * 2) * rowbytes <= 46 * 1024) mx *= 2;
  const int mx_default = mx;
  if (!tune_.empty()) {
    auto it = tune_.find(typeid(Op).name());
    if (it != tune_.end() && it->second >= 1 && it->second * TPL <= MaxThreads<Op>::v &&
        (it->second * TPL) % 32 == 0 && (size_t)it->second * rowbytes <= 200 * 1024)
      mx = it->second;
  }
  a.MX = mx;
  const int block = mx * TPL;
  EGPE_TRY(check_whole_warps(Op::NAME, L, block));
  const size_t smem_fixed =
      L * sizeof(C) + (Op::USES_LHY ? lhy_stage_bytes<R>(a.Q) : 0) + (NS > 0 ? sizeof(RedSmem<NS>) : 0);
  const size_t smem = smem_fixed + mx * rowbytes;
  const int rows = ny * nz;
  const int groups = (rows + mx - 1) / mx;
  void (*kern)(KArgs<R>);
  if constexpr (MinBlocks<Op>::v > 1) kern = xpass_kernel_mb<Op>;
  else kern = xpass_kernel<Op>;
  if (rec_) {
    EGPE_TRY(record(a, nullptr, xb_fn<Op>(), block, smem, groups));
    LaunchRec<R>& r = rec_->back();
    r.kind = 0;
    r.key = typeid(Op).name();
    r.name = Op::NAME;
    r.L = L;
    r.fn1 = (const void*)kern;
    r.tpl = TPL;
    r.max_threads = MaxThreads<Op>::v;
    r.mx = mx_default;
    r.rowbytes = rowbytes;
    r.smem_fixed = smem_fixed;
    r.rows = rows;
    return EGPE_OK;
  }
  const int occ = occupancy((const void*)kern, block, smem);
  const int grid = std::min(groups, std::min(occ * nsm_, 16384));
  if (timing_) t_begin(Op::NAME, L, Op::alg_bytes(a));
  kern<<<grid, block, smem, stream>>>(a);
  if (timing_) t_end();
  ++kernels_;
  return launch_status(Op::NAME, L, block, smem);
}

template <class R> template <class Op> egpe_status Engine<R>::launch_col(KArgs<R> a, const CUtensorMap* tm) {
  constexpr int L = Op::L, TPL = L / 8, NS = Op::NS;
  const int M = col_tile_width<C>(L, nx, col_bytes_);
  a.M = M;
  const int block = M * TPL;
  EGPE_TRY(check_whole_warps(Op::NAME, L, block));
  const int other = (Op::AXIS == 1) ? nz : ny;
  const int tiles = (nx / M) * other * a.nf;
  const size_t smem_tma = (size_t)(kColStages + 1) * M * L * sizeof(C) + L * sizeof(C) +
                          kColStages * sizeof(uint64_t) + (NS > 0 ? sizeof(RedSmem<NS>) : 0);
  const size_t smem_plain = L * sizeof(C) + 2 * (size_t)M * L * sizeof(C) + (NS > 0 ? sizeof(RedSmem<NS>) : 0);
  bool tma = tm && use_tma_;
  if (tma && !tune_.empty()) {
    auto it = tune_.find(typeid(Op).name());
    if (it != tune_.end()) tma = it->second != 0;
  }
  // the default tile width runs the kernels compiled for it
  constexpr int MD = ColDefaultM<Op>::v;
  const bool cm = M == MD;
  const void* fn_plain = cm ? (const void*)colpass_kernel<Op, MD> : (const void*)colpass_kernel<Op, 0>;
  const void* fn_tma = cm ? (const void*)colpass_tma_kernel<Op, MD> : (const void*)colpass_tma_kernel<Op, 0>;
  if (rec_) {
    const void* fb = tma ? (cm ? (const void*)colpass_tma_kernel_b<Op, MD> : (const void*)colpass_tma_kernel_b<Op, 0>)
                         : (cm ? (const void*)colpass_kernel_b<Op, MD> : (const void*)colpass_kernel_b<Op, 0>);
    EGPE_TRY(record(a, tma ? tm : nullptr, fb, block, tma ? smem_tma : smem_plain, tiles));
    LaunchRec<R>& r = rec_->back();
    r.kind = 1;
    r.key = typeid(Op).name();
    r.name = Op::NAME;
    r.L = L;
    r.fn1 = fn_plain;
    r.fn1_tma = fn_tma;
    r.tm = tm;  // kept for tuning even when this launch uses plain loads
    r.smem_plain = smem_plain;
    r.smem_tma = smem_tma;
    r.mx = (tm && use_tma_) ? 1 : 0;  // the untuned choice
    return EGPE_OK;
  }
  if (tma) {
    const size_t smem = smem_tma;
    const int occ = occupancy(fn_tma, block, smem);
    const int grid = std::min(tiles, std::min(occ * nsm_, 16384));
    if (timing_) t_begin(Op::NAME, L, Op::alg_bytes(a));
    if (cm) colpass_tma_kernel<Op, MD><<<grid, block, smem, stream>>>(*tm, a);
    else colpass_tma_kernel<Op, 0><<<grid, block, smem, stream>>>(*tm, a);
    if (timing_) t_end();
  } else {
    const size_t smem = smem_plain;
    const int occ = occupancy(fn_plain, block, smem);
    const int grid = std::min(tiles, std::min(occ * nsm_, 16384));
    if (timing_) t_begin(Op::NAME, L, Op::alg_bytes(a));
    if (cm) colpass_kernel<Op, MD><<<grid, block, smem, stream>>>(a);
    else colpass_kernel<Op, 0><<<grid, block, smem, stream>>>(a);
    if (timing_) t_end();
  }
  ++kernels_;
  return launch_status(Op::NAME, L, block, tma ? smem_tma : smem_plain);
}

template <class R> template <template <class, int> class OpT, int... Ls>
egpe_status Engine<R>::dispatch_x_in(int L, const KArgs<R>& a) {
  egpe_status s = EGPE_ERR_UNSUPPORTED;
  (void)((L == Ls ? (s = launch_x<OpT<R, Ls>>(a), true) : false) || ...);
  return s;
}

template <class R> template <template <class, int> class OpT, int... Ls>
egpe_status Engine<R>::dispatch_col_in(int L, const KArgs<R>& a, const CUtensorMap* tm) {
  egpe_status s = EGPE_ERR_UNSUPPORTED;
  (void)((L == Ls ? (s = launch_col<OpT<R, Ls>>(a, tm), true) : false) || ...);
  return s;
}

template <class R> template <int... Ls> egpe_status Engine<R>::plain_x_in(int inverse, const KArgs<R>& a) {
  egpe_status s = EGPE_ERR_UNSUPPORTED;
  (void)((nx == Ls ? (s = inverse ? launch_x<XPlain<R, Ls, true>>(a) : launch_x<XPlain<R, Ls, false>>(a), true)
                   : false) ||
         ...);
  return s;
}

template <class R> template <int... Ls>
egpe_status Engine<R>::plain_col_in(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm) {
  const int L = axis == 1 ? ny : nz;
  egpe_status s = EGPE_ERR_UNSUPPORTED;
  (void)((L == Ls ? (s = axis == 1 ? (inverse ? launch_col<ColPlain<R, Ls, 1, true>>(a, tm)
                                              : launch_col<ColPlain<R, Ls, 1, false>>(a, tm))
                                   : (inverse ? launch_col<ColPlain<R, Ls, 2, true>>(a, tm)
                                              : launch_col<ColPlain<R, Ls, 2, false>>(a, tm)),
                     true)
                  : false) ||
         ...);
  return s;
}

template <class R> template <template <class, int> class OpT>
egpe_status Engine<R>::dispatch_x(int L, const KArgs<R>& a) {
  if (L == 128 || L == 256) return dispatch_x_big<OpT>(L, a);
  if (L == 80) return dispatch_x_mr5<OpT>(L, a);
  if (L == 48 || L == 96) return dispatch_x_mr<OpT>(L, a);
  return dispatch_x_in<OpT, 16, 32, 64>(L, a);
}

template <class R> template <template <class, int> class OpT>
egpe_status Engine<R>::dispatch_col(int L, const KArgs<R>& a, const CUtensorMap* tm) {
  if (L == 128 || L == 256) return dispatch_col_big<OpT>(L, a, tm);
  if (L == 80) return dispatch_col_mr5<OpT>(L, a, tm);
  if (L == 48 || L == 96) return dispatch_col_mr<OpT>(L, a, tm);
  return dispatch_col_in<OpT, 16, 32, 64>(L, a, tm);
}

template <class R> egpe_status Engine<R>::plain_x(int inverse, const KArgs<R>& a) {
  if (nx == 128 || nx == 256) return plain_x_big(inverse, a);
  if (nx == 80) return plain_x_mr5(inverse, a);
  if (nx == 48 || nx == 96) return plain_x_mr(inverse, a);
  return plain_x_in<16, 32, 64>(inverse, a);
}

template <class R>
egpe_status Engine<R>::plain_col(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm) {
  const int L = axis == 1 ? ny : nz;
  if (L == 128 || L == 256) return plain_col_big(axis, inverse, a, tm);
  if (L == 80) return plain_col_mr5(axis, inverse, a, tm);
  if (L == 48 || L == 96) return plain_col_mr(axis, inverse, a, tm);
  return plain_col_in<16, 32, 64>(axis, inverse, a, tm);
}

// Energy / gradient pipeline: 6 complex 3D transforms.
template <class R> egpe_status Engine<R>::enq_eg(int trial, int gate, int ctrl) {
  KArgs<R> a = *base_;
  a.gate = gate;
  a.flag = trial;
  a.ctrl = 0;
  a.nf = 3;
  a.f0 = 0;
  EGPE_TRY(dispatch_x<XFwdEG>(nx, a));
  KArgs<R> y = a;
  y.gin = a.W;
  y.gout = a.W;
  EGPE_TRY(plain_col(1, 0, y, tmy()));
  EGPE_TRY(dispatch_col<ZEg>(nz, a, tmz()));
  EGPE_TRY(plain_col(1, 1, y, tmy()));
  a.ctrl = ctrl;
  return dispatch_x<XInvEG>(nx, a);
}

// Preconditioner pipeline: 4 transforms for the kinetic modes, none otherwise.
template <class R> egpe_status Engine<R>::enq_pc(int mode, int gate, int ctrl, int rgiven) {
  KArgs<R> a = *base_;
  a.gate = gate;
  a.flag = rgiven;
  a.diag = (mode == 2 || mode == 3) ? 1 : 0;
  a.blend = mode == 4 ? 1 : 0;
  a.ctrl = 0;
  a.nf = 2;
  a.f0 = 0;
  if (mode == 1 || mode == 3 || mode == 4) {
    EGPE_TRY(dispatch_x<XFwdPC>(nx, a));
    KArgs<R> y = a;
    y.gin = a.W;
    y.gout = a.W;
    EGPE_TRY(plain_col(1, 0, y, tmy()));
    EGPE_TRY(dispatch_col<ZPc>(nz, a, tmz()));
    EGPE_TRY(plain_col(1, 1, y, tmy()));
    a.ctrl = ctrl;
    return dispatch_x<XInvPC>(nx, a);
  }
  a.ctrl = ctrl;
  return launch_point(pc_point_kernel<R>, pc_point_kernel_b<R>, "pointwise precond sums",
                      (a.diag ? 13.0 : 12.0) * N * sizeof(C), a, (long long)((N + 255) / 256));
}

// Line-search pipeline: forward transforms of p_1, p_2 and one packed pair.
template <class R> egpe_status Engine<R>::enq_lc(int gate, int ctrl, int pgiven) {
  KArgs<R> a = *base_;
  a.gate = gate;
  a.flag = pgiven;
  a.ctrl = 0;
  a.nf = 3;
  a.f0 = 0;
  EGPE_TRY(dispatch_x<XFwdLC>(nx, a));
  KArgs<R> y = a;
  y.gin = a.W;
  y.gout = a.W;
  EGPE_TRY(plain_col(1, 0, y, tmy()));
  EGPE_TRY(dispatch_col<ZLc>(nz, a, tmz()));
  y.nf = 1;
  y.f0 = 2;
  EGPE_TRY(plain_col(1, 1, y, tmy()));
  a.ctrl = ctrl;
  return dispatch_x<XInvLC>(nx, a);
}

template <class R> egpe_status Engine<R>::enq_attempt(int mode) {
  EGPE_TRY(enq_pc(mode, GATE_NEW_ITER, 1, 0));
  EGPE_TRY(enq_lc(GATE_NEW_ITER, 1, 0));
  return enq_eg(1, GATE_ACTIVE, 1);
}

template <class R>
egpe_status Engine<R>::reset_state(const egpe_solve_opts* o, int fp32_phase, int max_iter, double tol_res,
                                   double accept_rtol) {
  DevState& h = *st_host_;
  std::memset(&h, 0, sizeof(DevState));
  h.phase = PH_NEW_ITER;
  h.status = EGPE_ERR_NOT_CONVERGED;
  h.cur = 0;
  h.dV = dV;
  h.invN = 1.0 / (double)N;
  h.opt.pv_floor = 1e-2;
  h.opt.pc_blend = 0.5;
  h.opt.armijo_c1 = 1e-4;
  h.opt.theta_max = 1.5707963267948966;
  h.opt.restart_period = 20;
  if (o) {
    h.opt.precond = o->precond;
    h.opt.beta_rule = o->beta_rule;
    h.opt.restart_period = o->restart_period;
    h.opt.max_iter = max_iter;
    h.opt.armijo_max = o->armijo_max;
    h.opt.trace_cap = o->trace ? std::min(o->trace_cap, trace_alloc_) : 0;
    h.opt.fp32_phase = fp32_phase;
    h.opt.tol_res = tol_res;
    h.opt.tol_dE = o->tol_dE;
    h.opt.armijo_c1 = o->armijo_c1;
    h.opt.theta_max = o->theta_max;
    h.opt.accept_rtol = accept_rtol;
    h.opt.pv_floor = o->pv_floor;
    h.opt.pc_blend = o->pc_blend;
    h.opt.stall_iters = fp32_phase ? o->stall_iters_fp32 : 0;
  }
  EGPE_CUDA(cudaMemcpyAsync(st_, &h, sizeof(DevState), cudaMemcpyHostToDevice, stream));
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::read_state(DevState& hs, bool report_timeout) {
  EGPE_CUDA(cudaMemcpyAsync(st_host_, st_, sizeof(DevState), cudaMemcpyDeviceToHost, stream));
  EGPE_CUDA(cudaStreamSynchronize(stream));
  hs = *st_host_;
  if (report_timeout && hs.timeout) {
    set_error_msg("a device-side wait ran out of its poll budget");
    return EGPE_ERR_TIMEOUT;
  }
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::energy_grad(const C* psi, egpe_energy_terms* out, C* grad) {
  EGPE_TRY(reset_state(nullptr, 0, 0, 0.0, 0.0));
  EGPE_CUDA(cudaMemcpyAsync(base_->psi[0], psi, 2 * N * sizeof(C), cudaMemcpyDeviceToDevice, stream));
  EGPE_TRY(enq_eg(0, GATE_ALWAYS, 1));
  if (grad) EGPE_CUDA(cudaMemcpyAsync(grad, base_->hp[0], 2 * N * sizeof(C), cudaMemcpyDeviceToDevice, stream));
  DevState hs;
  EGPE_TRY(read_state(hs));
  if (out) {
    EnergyOut o;
    finalize_energy(hs.eg[0], hs.egz[0], hs.dV, hs.invN, o);
    out->E = o.E;
    for (int i = 0; i < 2; ++i) {
      out->kin[i] = o.kin[i];
      out->mu[i] = o.mu[i];
      out->norm2[i] = o.norm2[i];
      out->shift[i] = o.shift[i];
    }
    out->trap = o.trap;
    out->contact = o.contact;
    out->dipolar = o.dipolar;
    out->lhy = o.lhy;
  }
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::line_coeffs(const C* psi, const C* p, double coeffs[3]) {
  egpe_energy_terms t;
  EGPE_TRY(energy_grad(psi, &t, nullptr));
  EGPE_CUDA(cudaMemcpyAsync(base_->pb[0], p, 2 * N * sizeof(C), cudaMemcpyDeviceToDevice, stream));
  EGPE_TRY(enq_lc(GATE_ALWAYS, 0, 1));
  DevState hs;
  EGPE_TRY(read_state(hs));
  LineOut o;
  finalize_line(hs.lc, hs.lcz, hs.mu, hs.dV, hs.invN, o);
  coeffs[0] = t.E;
  coeffs[1] = o.Ep;
  coeffs[2] = o.Epp;
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::precondition(int mode, const C* psi, const C* r, C* z) {
  EGPE_TRY(energy_grad(psi, nullptr, nullptr));
  if (r) EGPE_CUDA(cudaMemcpyAsync(base_->rb[0], r, 2 * N * sizeof(C), cudaMemcpyDeviceToDevice, stream));
  EGPE_TRY(enq_pc(mode, GATE_ALWAYS, 0, r ? 1 : 0));
  EGPE_CUDA(cudaMemcpyAsync(z, base_->z, 2 * N * sizeof(C), cudaMemcpyDeviceToDevice, stream));
  EGPE_CUDA(cudaStreamSynchronize(stream));
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::retract(const C* psi, const C* p, const double theta[2], C* out) {
  KArgs<R> a = *base_;
  const int grid = (int)std::min<size_t>((N + 255) / 256, (size_t)nsm_ * 8);
  rt_sums_kernel<R><<<grid, 256, 0, stream>>>(a, psi, p);
  ++kernels_;
  EGPE_CUDA(cudaGetLastError());
  DevState hs;
  EGPE_TRY(read_state(hs));
  double ca[2], cb[2];
  for (int i = 0; i < 2; ++i) {
    const double pn = sqrt(hs.rt[RT_P1 + i] * dV);
    const double psip = hs.rt[RT_PSIP1 + i] * dV, nps = hs.rt[RT_PSI1 + i] * dV;
    const double c = cos(theta[i]), s = sin(theta[i]);
    if (pn > 0.0) {
      const double inv = 1.0 / sqrt(c * c * nps + s * s + 2.0 * c * s * psip / pn);
      ca[i] = c * inv;
      cb[i] = s * inv / pn;
    } else {
      ca[i] = 1.0 / sqrt(nps);
      cb[i] = 0.0;
    }
  }
  rt_apply_kernel<R><<<grid, 256, 0, stream>>>(N, psi, p, out, (R)ca[0], (R)cb[0], (R)ca[1], (R)cb[1]);
  ++kernels_;
  EGPE_CUDA(cudaGetLastError());
  EGPE_CUDA(cudaStreamSynchronize(stream));
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::normalise_current() {
  const double th[2] = {0.0, 0.0};
  return retract(base_->psi[0], base_->psi[0], th, base_->psi[0]);
}

template <class R> egpe_status Engine<R>::fft(const C* in, C* out, int nf, int inverse) {
  for (int f = 0; f < nf; ++f) {
    KArgs<R> a = *base_;
    a.gate = GATE_ALWAYS;
    a.nf = 1;
    a.f0 = 0;
    a.gin = in + (size_t)f * N;
    a.gout = out + (size_t)f * N;
    EGPE_TRY(plain_x(inverse, a));
    a.gin = out + (size_t)f * N;
    CUtensorMap my, mz;
    const bool ok = use_tma_ && make_col_map<C>(my, out + (size_t)f * N, nx, ny, nz, 1, 1, col_bytes_) &&
                    make_col_map<C>(mz, out + (size_t)f * N, nx, ny, nz, 1, 2, col_bytes_);
    EGPE_TRY(plain_col(1, inverse, a, ok ? &my : nullptr));
    EGPE_TRY(plain_col(2, inverse, a, ok ? &mz : nullptr));
  }
  EGPE_CUDA(cudaStreamSynchronize(stream));
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::load_psi(const void* src, cudaMemcpyKind kind) {
  EGPE_CUDA(cudaMemcpyAsync(base_->psi[0], src, 2 * N * sizeof(C), kind, stream));
  return EGPE_OK;
}

template <class R> typename Engine<R>::C* Engine<R>::current_psi() { return base_->psi[st_host_->cur]; }
template <class R> typename Engine<R>::C* Engine<R>::psi_slot0() { return base_->psi[0]; }

template <class R> egpe_status Engine<R>::store_psi(void* dst, cudaMemcpyKind kind) {
  EGPE_CUDA(cudaMemcpyAsync(dst, current_psi(), 2 * N * sizeof(C), kind, stream));
  EGPE_CUDA(cudaStreamSynchronize(stream));
  return EGPE_OK;
}

template <class R>
egpe_status Engine<R>::solve_begin(const egpe_solve_opts& o, int fp32_phase, int max_iter, double tol_res,
                                   double accept_rtol, bool want_trace, int trace_cap) {
  const int mode = o.precond;
  if (want_trace && trace_cap > trace_alloc_) {
    // the trace buffer is captured by the graphs: allocate once, generously
    const int want = std::max(trace_cap, 65536);
    for (auto& gx : graph_)
      if (gx) {
        cudaGraphExecDestroy(gx);
        gx = nullptr;
      }
    if (trace_) cudaFree(trace_);
    trace_ = nullptr;
    EGPE_CUDA(cudaMalloc(&trace_, (size_t)want * sizeof(TraceDev)));
    trace_alloc_ = want;
    base_->trace = trace_;
  }
  egpe_solve_opts oo = o;
  oo.trace_cap = want_trace ? trace_cap : 0;
  oo.trace = want_trace ? (void*)1 : nullptr;
  EGPE_TRY(reset_state(&oo, fp32_phase, max_iter, tol_res, accept_rtol));
  // r and p history start at zero (beta = 0 at n = 0 reads them)
  EGPE_CUDA(cudaMemsetAsync(base_->rb[0], 0, 8 * N * sizeof(C), stream));
  EGPE_TRY(enq_eg(0, GATE_ALWAYS, 1));
  run_k0_ = kernels_;
  run_ite_ = false;
  run_mode_ = mode;
  run_graph_ = o.use_graph ? 1 : 0;
  run_launches_ = 0;
  per_attempt_ = 0;
  if (run_graph_) {
    if (!graph_[mode]) {
      cudaGraph_t g = nullptr;
      EGPE_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
      const long long kb = kernels_;
      egpe_status s = enq_attempt(mode);
      cudaError_t ce = cudaStreamEndCapture(stream, &g);
      if (s != EGPE_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (ce != cudaSuccess) {
        set_error("cudaStreamEndCapture", ce);
        return EGPE_ERR_CUDA;
      }
      graph_max_iter_[mode] = (int)(kernels_ - kb);
      cudaError_t ie = cudaGraphInstantiate(&graph_[mode], g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        set_error("cudaGraphInstantiate", ie);
        graph_[mode] = nullptr;
        return EGPE_ERR_CUDA;
      }
      kernels_ = kb;
    }
    per_attempt_ = graph_max_iter_[mode];
  }
  return EGPE_OK;
}

// Kinetic half step e^{-dtau T/2} of both components (4 transforms), with the
// potential step e^{-dtau U} in the prologue when `potential` is set (U from
// the aux fields of the last evaluation).  Leaves the norms in st->rt[0..1].
template <class R> egpe_status Engine<R>::enq_kin(int potential, int gate) {
  KArgs<R> a = *base_;
  a.gate = gate;
  a.flag = potential;
  a.ctrl = 0;
  a.nf = 2;
  a.f0 = 0;
  EGPE_TRY(dispatch_x<XFwdKin>(nx, a));
  KArgs<R> y = a;
  y.gin = a.W;
  y.gout = a.W;
  EGPE_TRY(plain_col(1, 0, y, tmy()));
  EGPE_TRY(dispatch_col<ZKin>(nz, a, tmz()));
  EGPE_TRY(plain_col(1, 1, y, tmy()));
  return dispatch_x<XInvKin>(nx, a);
}

// One Strang step: kinetic half step, evaluation at the half-stepped state
// (dipolar and LHY potentials), potential step fused into the second kinetic
// half step, renormalisation, evaluation of the new state + controller.
template <class R> egpe_status Engine<R>::enq_ite_step(int gate) {
  EGPE_TRY(enq_kin(0, gate));
  EGPE_TRY(enq_eg(0, gate, 0));
  EGPE_TRY(enq_kin(1, gate));
  {
    KArgs<R> a = *base_;
    a.gate = gate;
    EGPE_TRY(launch_point(ite_scale_kernel<R>, ite_scale_kernel_b<R>, "ITE renormalise", 4.0 * N * sizeof(C), a,
                          (long long)((N + 255) / 256)));
  }
  return enq_eg(0, gate, 2);
}

template <class R> egpe_status Engine<R>::ite_begin(double dtau, double tol_dE, int max_steps, bool use_graph) {
  const double pi = 3.14159265358979323846;
  kin_host_.assign((size_t)(nx + ny + nz + 1), R(0));
  const int n3[3] = {nx, ny, nz};
  int off = 0;
  for (int ax = 0; ax < 3; ++ax) {
    const double dk = pi / grid_.L[ax];
    for (int j = 0; j < n3[ax]; ++j) {
      const double k = dk * (double)(j < n3[ax] / 2 ? j : j - n3[ax]);
      kin_host_[off + j] = (R)exp(-0.25 * dtau * k * k);
    }
    off += n3[ax];
  }
  kin_host_[off] = (R)dtau;
  EGPE_CUDA(cudaMemcpyAsync(kin_tab_, kin_host_.data(), kin_host_.size() * sizeof(R), cudaMemcpyHostToDevice,
                            stream));
  egpe_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  o.tol_dE = tol_dE;
  EGPE_TRY(reset_state(&o, sizeof(R) == 4, max_steps, 0.0, 0.0));
  EGPE_TRY(enq_eg(0, GATE_ALWAYS, 1));
  run_k0_ = kernels_;
  run_ite_ = true;
  run_graph_ = use_graph ? 1 : 0;
  run_launches_ = 0;
  per_attempt_ = 0;
  if (run_graph_ && !graph_ite_) {
    cudaGraph_t g = nullptr;
    EGPE_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    const long long kb = kernels_;
    egpe_status s = enq_ite_step(GATE_ACTIVE);
    cudaError_t ce = cudaStreamEndCapture(stream, &g);
    if (s != EGPE_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (ce != cudaSuccess) {
      set_error("cudaStreamEndCapture", ce);
      return EGPE_ERR_CUDA;
    }
    ite_per_step_ = (int)(kernels_ - kb);
    cudaError_t ie = cudaGraphInstantiate(&graph_ite_, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      set_error("cudaGraphInstantiate", ie);
      graph_ite_ = nullptr;
      return EGPE_ERR_CUDA;
    }
    kernels_ = kb;
  }
  return EGPE_OK;
}

template <class R>
egpe_status Engine<R>::ite(double dtau, double tol_dE, int max_steps, int poll_every, bool use_graph, SolveRun& run) {
  EGPE_TRY(ite_begin(dtau, tol_dE, max_steps, use_graph));
  const int poll = std::max(1, poll_every);
  while (run_launches_ < (long long)max_steps) {
    EGPE_TRY(solve_launch((int)std::min<long long>(poll, (long long)max_steps - run_launches_)));
    int phase = 0;
    EGPE_TRY(solve_poll(phase));
    if (phase == PH_DONE) break;
  }
  return solve_finish(run, nullptr, 0, 0);
}

template <class R> egpe_status Engine<R>::solve_launch(int attempts) {
  for (int k = 0; k < attempts; ++k) {
    if (run_ite_) {
      if (run_graph_) {
        EGPE_CUDA(cudaGraphLaunch(graph_ite_, stream));
        kernels_ += ite_per_step_;
      } else {
        EGPE_TRY(enq_ite_step(GATE_ACTIVE));
      }
    } else if (run_graph_) {
      EGPE_CUDA(cudaGraphLaunch(graph_[run_mode_], stream));
      kernels_ += per_attempt_;
    } else {
      EGPE_TRY(enq_attempt(run_mode_));
    }
    ++run_launches_;
  }
  return EGPE_OK;
}

template <class R> egpe_status Engine<R>::solve_poll(int& phase) {
  EGPE_CUDA(cudaMemcpyAsync(&st_host_->phase, &st_->phase, sizeof(int), cudaMemcpyDeviceToHost, stream));
  EGPE_CUDA(cudaStreamSynchronize(stream));
  phase = st_host_->phase;
  return EGPE_OK;
}

template <class R>
egpe_status Engine<R>::solve_finish(SolveRun& run, egpe_trace_entry* trace_out, int trace_cap, int trace_offset) {
  {
    KArgs<R> a = *base_;
    const int grid = (int)std::min<size_t>((N + 255) / 256, (size_t)nsm_ * 8);
    resnorm_kernel<R><<<grid, 256, 0, stream>>>(a);
    ++kernels_;
    EGPE_CUDA(cudaGetLastError());
  }
  DevState hs;
  EGPE_TRY(read_state(hs, false));
  run.status = (hs.phase == PH_DONE) ? hs.status : EGPE_ERR_NOT_CONVERGED;
  if (hs.timeout) run.status = EGPE_ERR_TIMEOUT;
  run.n = hs.n;
  run.attempts = hs.attempts;
  run.restarts = hs.restarts;
  run.armijo_total = hs.armijo_total;
  run.launches = (int)run_launches_;
  run.E = hs.E;
  run.mu[0] = hs.mu[0];
  run.mu[1] = hs.mu[1];
  run.res = sqrt((hs.pca[0] + hs.pca[1]) * dV);
  run.ffts = hs.ffts;
  run.kernels = kernels_ - run_k0_;
  run.trace_len = 0;
  run.phase = hs.phase;
  if (trace_out && hs.trace_len > 0) {
    const int n = std::min(hs.trace_len, trace_cap);
    std::vector<TraceDev> tmp(n);
    EGPE_CUDA(cudaMemcpy(tmp.data(), trace_, n * sizeof(TraceDev), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n && trace_offset + i < trace_cap; ++i) {
      egpe_trace_entry& d = trace_out[trace_offset + i];
      const TraceDev& s = tmp[i];
      d.n = s.n;
      d.kind = s.kind;
      d.armijo = s.armijo;
      d.flags = s.flags;
      d.E = s.E;
      d.E_trial = s.E_trial;
      d.res = s.res;
      d.beta = s.beta;
      d.alpha = s.alpha;
      d.theta[0] = s.theta[0];
      d.theta[1] = s.theta[1];
      d.Ep = s.Ep;
      d.Epp = s.Epp;
      ++run.trace_len;
    }
  }
  return EGPE_OK;
}

template <class R>
egpe_status Engine<R>::solve(const egpe_solve_opts& o, int fp32_phase, int max_iter, double tol_res,
                             double accept_rtol, SolveRun& run, egpe_trace_entry* trace_out, int trace_cap,
                             int trace_offset) {
  EGPE_TRY(solve_begin(o, fp32_phase, max_iter, tol_res, accept_rtol, trace_out != nullptr, trace_cap));
  const int poll = std::max(1, o.poll_every);
  const long long max_launch = (long long)(max_iter + 2) * (long long)(o.armijo_max + 2) + 4;
  while (run_launches_ < max_launch) {
    EGPE_TRY(solve_launch(poll));
    int phase = 0;
    EGPE_TRY(solve_poll(phase));
    if (phase == PH_DONE) break;
  }
  return solve_finish(run, trace_out, trace_cap, trace_offset);
}

}  // namespace egpe
