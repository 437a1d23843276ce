// Engine<double>: the FP64 path.
#include "batch.cuh"
template class egpe::Engine<double>;
template egpe_status egpe::batch_solve<double>(const std::vector<egpe::Engine<double>*>&, cudaStream_t,
                                             const egpe_solve_opts&, int, int, double, double,
                                             std::vector<egpe::SolveRun>&, egpe_trace_entry*, int, int*);

// ---------------------------------------------------------------------------
// egpe_energy_grad_noalloc: the FP64 energy/gradient evaluation without any
// device allocation, for grids of at most 32 points per axis.
//
// Who needs it: host applications whose device memory is owned entirely by
// their own pool allocator (a cudaMalloc from a library would fail or eat into
// a budget the application has already handed out), and latency-sensitive
// loops that must never enter the CUDA allocator.  Such callers cannot create
// a handle (egpe_create allocates the workspaces), so this entry point runs
// the same five kernels as egpe_energy_grad with every workspace carved out of
// one file-scope device array of fixed size.
//
// The array lives for as long as the library is loaded, on every GPU that
// loads it.  Host code cannot hand the array's name to a kernel (in host code
// it names a host-side stand-in), so its device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made with that
// device current, and cached (under a mutex) for later calls; make that first
// call before any stream capture begins.  The cached address stays valid until
// the device is reset (cudaDeviceReset), which invalidates this entry point for
// the rest of the process.  All calls share the array: two calls whose work
// overlaps on the GPU (different streams, or different host threads on one
// device) race on it and must be serialised by the caller.  Each call is
// synchronous: it returns after E and mu have reached the host.
// ---------------------------------------------------------------------------
#include <cmath>
#include <cstring>
#include <mutex>

namespace {

constexpr int kNoAllocMaxN = 32;                         // points per axis
constexpr size_t kNoAllocMaxPoints = 32 * 32 * 32;
constexpr size_t kNoAllocBlocks = 1024;                  // partial-sum slots
constexpr size_t kNoAllocBytes = (size_t)4 << 20;        // 4 MiB

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffW = 0;                                                   // 3 fields
constexpr size_t kOffAx = al256(kOffW + 3 * kNoAllocMaxPoints * sizeof(double2));   // 2 fields
constexpr size_t kOffHp = al256(kOffAx + 2 * kNoAllocMaxPoints * sizeof(double2));  // 2 fields
constexpr size_t kOffPart = al256(kOffHp + 2 * kNoAllocMaxPoints * sizeof(double2));
constexpr size_t kOffSt = al256(kOffPart + kNoAllocBlocks * egpe::MAX_NS * sizeof(double));
constexpr size_t kOffCnt = al256(kOffSt + sizeof(egpe::DevState));
constexpr size_t kOffTw = al256(kOffCnt + 64 * sizeof(unsigned));
constexpr size_t kOffNodes = al256(kOffTw + 3 * kNoAllocMaxN * sizeof(double2));
constexpr size_t kOffEnd = al256(kOffNodes + 64 * sizeof(egpe::LhyNode<double>));
static_assert(kOffEnd <= kNoAllocBytes, "no-alloc scratch layout exceeds its array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
static unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (looked up once).
cudaError_t noalloc_scratch(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t ce = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (ce != cudaSuccess) return ce;
    if (!ptr) return cudaErrorInvalidSymbol;
    g_scratch_ptr[dev] = (unsigned char*)ptr;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <class Op> cudaError_t noalloc_launch_x(egpe::KArgs<double> a, int rows, cudaStream_t s) {
  using namespace egpe;
  constexpr int L = Op::L, TPL = L / 8, NF = Op::NF, NS = Op::NS;
  constexpr int LP = row_len_padded<double, L>();
  const size_t rowbytes = (size_t)NF * LP * sizeof(double2);
  int mx = whole_warp_rows(L);
  while ((mx * 2) * TPL <= MaxThreads<Op>::v && (size_t)(mx * 2) * rowbytes <= 46 * 1024) mx *= 2;
  a.MX = mx;
  const size_t smem = L * sizeof(double2) + (Op::USES_LHY ? lhy_stage_bytes<double>(a.Q) : 0) +
                      mx * rowbytes + (NS > 0 ? sizeof(RedSmem<NS>) : 0);
  const int groups = (rows + mx - 1) / mx;
  const int grid = std::min(groups, (int)kNoAllocBlocks);
  xpass_kernel<Op><<<grid, mx * TPL, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Op> cudaError_t noalloc_launch_col(egpe::KArgs<double> a, int other, cudaStream_t s) {
  using namespace egpe;
  constexpr int L = Op::L, TPL = L / 8, NS = Op::NS;
  int M = std::max((int)(128 / sizeof(double2)), whole_warp_rows(L));
  M = std::min(M, a.nx);
  a.M = M;
  const size_t smem = L * sizeof(double2) + 2 * (size_t)M * L * sizeof(double2) + (NS > 0 ? sizeof(RedSmem<NS>) : 0);
  const int tiles = (a.nx / M) * other * a.nf;
  const int grid = std::min(tiles, (int)kNoAllocBlocks);
  colpass_kernel<Op><<<grid, M * TPL, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LX, int LY, int LZ> cudaError_t noalloc_pipeline(const egpe::KArgs<double>& a, cudaStream_t s) {
  using namespace egpe;
  cudaError_t e;
  const int rows = a.ny * a.nz;
  if ((e = noalloc_launch_x<XFwdEG<double, LX>>(a, rows, s)) != cudaSuccess) return e;
  egpe::KArgs<double> y = a;
  y.gin = a.W;
  y.gout = a.W;
  if ((e = noalloc_launch_col<ColPlain<double, LY, 1, false>>(y, a.nz, s)) != cudaSuccess) return e;
  if ((e = noalloc_launch_col<ZEg<double, LZ>>(a, a.ny, s)) != cudaSuccess) return e;
  if ((e = noalloc_launch_col<ColPlain<double, LY, 1, true>>(y, a.nz, s)) != cudaSuccess) return e;
  return noalloc_launch_x<XInvEG<double, LX>>(a, rows, s);
}

template <int LX, int LY>
cudaError_t noalloc_dispatch_z(int nz, const egpe::KArgs<double>& a, cudaStream_t s) {
  return nz == 16 ? noalloc_pipeline<LX, LY, 16>(a, s) : noalloc_pipeline<LX, LY, 32>(a, s);
}
template <int LX> cudaError_t noalloc_dispatch_y(int ny, int nz, const egpe::KArgs<double>& a, cudaStream_t s) {
  return ny == 16 ? noalloc_dispatch_z<LX, 16>(nz, a, s) : noalloc_dispatch_z<LX, 32>(nz, a, s);
}

}  // namespace

extern "C" egpe_status egpe_energy_grad_noalloc(const egpe_grid* grid, const egpe_params* params, const void* psi,
                                                double* E, double mu[2], void* grad, void* cuda_stream) {
  using namespace egpe;
  if (!grid || !params || !psi) {
    set_error_msg("egpe_energy_grad_noalloc: grid, params and psi are required");
    return EGPE_ERR_INVALID_ARG;
  }
  const egpe_grid& g = *grid;
  const egpe_params& p = *params;
  for (int ax = 0; ax < 3; ++ax) {
    if (g.n[ax] != 16 && g.n[ax] != 32) {
      set_error_msg("egpe_energy_grad_noalloc: each axis must have 16 or 32 points (its fixed scratch holds "
                    "at most 32^3 points); use a handle for larger grids");
      return EGPE_ERR_INVALID_ARG;
    }
    if (!(g.L[ax] > 0.0) || !std::isfinite(g.L[ax]) || !std::isfinite(p.trap[ax])) {
      set_error_msg("egpe_energy_grad_noalloc: box half-lengths must be positive and finite, traps finite");
      return EGPE_ERR_INVALID_ARG;
    }
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      if (!std::isfinite(p.g[i][j]) || !std::isfinite(p.gdd[i][j])) {
        set_error_msg("egpe_energy_grad_noalloc: couplings must be finite");
        return EGPE_ERR_INVALID_ARG;
      }
  if (p.g[0][1] != p.g[1][0] || p.gdd[0][1] != p.gdd[1][0] || p.lhy_nodes < 1 || p.lhy_nodes > 64 ||
      !(p.lhy_eta_scale > 0.0) || !std::isfinite(p.lhy_kappa)) {
    set_error_msg("egpe_energy_grad_noalloc: couplings must be symmetric, lhy_nodes in [1,64], eta_s > 0");
    return EGPE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) {
    set_error("cudaGetDevice", ce);
    return EGPE_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error_msg("egpe_energy_grad_noalloc: device ordinal out of range");
    return EGPE_ERR_INVALID_ARG;
  }
  unsigned char* base = nullptr;
  ce = noalloc_scratch(dev, &base);
  if (ce != cudaSuccess) {
    set_error("cudaGetSymbolAddress", ce);
    return EGPE_ERR_CUDA;
  }
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const size_t N = (size_t)nx * ny * nz;

  // constant tables (host long double, shared with the handle path), staged
  // through fixed host arrays
  double2 tw[3][kNoAllocMaxN];
  for (int ax = 0; ax < 3; ++ax) twiddle_table<double>(g.n[ax], tw[ax]);
  LhyNode<double> nodes[64];
  const int qm = lhy_node_table<double>(p, nodes);
  double2* twd = (double2*)(base + kOffTw);
  for (int ax = 0; ax < 3; ++ax) {
    ce = cudaMemcpyAsync(twd + ax * kNoAllocMaxN, tw[ax], g.n[ax] * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) {
      set_error("cudaMemcpyAsync", ce);
      return EGPE_ERR_CUDA;
    }
  }
  ce = cudaMemcpyAsync(base + kOffNodes, nodes, p.lhy_nodes * sizeof(LhyNode<double>), cudaMemcpyHostToDevice, s);
  // the previous call's state and arrival counter must not leak into this one
  if (ce == cudaSuccess) ce = cudaMemsetAsync(base + kOffSt, 0, kOffTw - kOffSt, s);
  if (ce != cudaSuccess) {
    set_error("cudaMemcpyAsync/cudaMemsetAsync", ce);
    return EGPE_ERR_CUDA;
  }

  KArgs<double> a;
  std::memset((void*)&a, 0, sizeof(a));
  const double hx = 2.0 * g.L[0] / nx, hy = 2.0 * g.L[1] / ny, hz = 2.0 * g.L[2] / nz;
  const double dpi = 3.14159265358979323846;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.N = (int)N;
  a.hx = hx;
  a.hy = hy;
  a.hz = hz;
  a.Lx = g.L[0];
  a.Ly = g.L[1];
  a.Lz = g.L[2];
  a.dkx = dpi / g.L[0];
  a.dky = dpi / g.L[1];
  a.dkz = dpi / g.L[2];
  a.vx = 0.5 * p.trap[0] * p.trap[0];
  a.vy = 0.5 * p.trap[1] * p.trap[1];
  a.vz = 0.5 * p.trap[2] * p.trap[2];
  a.g11 = p.g[0][0];
  a.g12 = p.g[0][1];
  a.g21 = p.g[1][0];
  a.g22 = p.g[1][1];
  a.d11 = p.gdd[0][0];
  a.d12 = p.gdd[0][1];
  a.d21 = p.gdd[1][0];
  a.d22 = p.gdd[1][1];
  a.invN = 1.0 / (double)N;
  a.Q = p.lhy_nodes;
  a.Qm = qm;
  a.nskip = lhy_skip_threshold(p);
  // every node evaluated exactly per point (no interpolation table here)
  a.Qx = a.Q;
  a.Qxm = qm;
  a.tab.tab = nullptr;
  a.tab.ni = 0;
  a.nodes = (const LhyNode<double>*)(base + kOffNodes);
  a.xnodes = a.nodes;
  a.twx = twd;
  a.twy = twd + kNoAllocMaxN;
  a.twz = twd + 2 * kNoAllocMaxN;
  a.psi[0] = (double2*)psi;  // read only: the non-trial prologue never writes it
  a.hp[0] = grad ? (double2*)grad : (double2*)(base + kOffHp);
  a.ax[0] = (double2*)(base + kOffAx);
  a.W = (double2*)(base + kOffW);
  a.partials = (double*)(base + kOffPart);
  a.counter = (unsigned*)(base + kOffCnt);
  a.st = (DevState*)(base + kOffSt);
  a.trace = nullptr;
  a.wait_polls = kTmaWaitPolls;  // (the passes here load tiles without TMA)
  a.gate = GATE_ALWAYS;
  a.flag = 0;
  a.ctrl = 0;
  a.nf = 3;
  a.f0 = 0;

  ce = (nx == 16) ? noalloc_dispatch_y<16>(ny, nz, a, s) : noalloc_dispatch_y<32>(ny, nz, a, s);
  if (ce != cudaSuccess) {
    set_error("egpe_energy_grad_noalloc launch", ce);
    return EGPE_ERR_CUDA;
  }
  double sums[EG_NS + EGZ_NS];
  DevState* st = (DevState*)(base + kOffSt);
  ce = cudaMemcpyAsync(sums, &st->eg[0][0], EG_NS * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(sums + EG_NS, &st->egz[0][0], EGZ_NS * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    set_error("egpe_energy_grad_noalloc readback", ce);
    return EGPE_ERR_CUDA;
  }
  EnergyOut o;
  finalize_energy(sums, sums + EG_NS, hx * hy * hz, 1.0 / (double)N, o);
  if (E) *E = o.E;
  if (mu) {
    mu[0] = o.mu[0];
    mu[1] = o.mu[1];
  }
  return EGPE_OK;
}
