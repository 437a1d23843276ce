// Kernels of the eGPE hot path.  Two kernel shapes carry every 3D transform:
//
// * xpass_kernel<Op>: lines along x (contiguous).  A block owns MX rows; each
//   row is transformed by L/8 threads.  Op supplies the prologue (values at the
//   transform's entry positions, read straight from global memory) and the
//   epilogue (consumes the exit positions: stores, pointwise physics, sums).
// * colpass_kernel<Op>: lines along y or z (strided).  A tile is M adjacent x
//   columns times one line; lanes run along x so every global access is a
//   full 128-byte row of the tile.
//
// Both are persistent (grid-stride over rows / tiles) so that the per-block
// FP64 partial sums stay few; the last block finalises the sums in a fixed
// order and, where a pipeline needs it, runs the controller step.
#pragma once
#include <type_traits>
#include "common.cuh"
#include "ctrl.cuh"
#include "fft.cuh"
#include "lhy.cuh"
#include "reduce.cuh"
#include "tma.cuh"

// Resident blocks per SM asked of the FP32 x-inverse epilogue passes, which
// caps their registers: energy 4 x 128 threads (128 registers, no spills),
// line coefficients 2 x 256 (128 registers, a few spilled bytes),
// preconditioner 1 (at 128 registers it spills ~250 bytes).  At 128^3 the
// energy pass went from 55.5 to 49.5 us and the line pass from 59 to 57 us.
#ifndef EGPE_EG_MINB
#define EGPE_EG_MINB 4
#endif
#ifndef EGPE_LC_MINB
#define EGPE_LC_MINB 2
#endif
#ifndef EGPE_PC_MINB
#define EGPE_PC_MINB 1
#endif

namespace egpe {

template <class R> struct KArgs {
  using C = C2<R>;
  int nx, ny, nz, N;
  R hx, hy, hz, Lx, Ly, Lz;
  R dkx, dky, dkz;           // pi / L_a
  R vx, vy, vz;              // lambda_a^2 / 2
  R g11, g12, g21, g22;      // contact couplings
  R d11, d12, d21, d22;      // k-space dipolar coefficients
  R invN;
  int Q, Qm;  // Gauss-Legendre nodes; the first Qm have det eta > 0
  R nskip;    // LHY terms skipped where n1 + n2 <= nskip (their size is below 1e-30)
  const LhyNode<R>* nodes;   // all Q nodes (parameter derivatives)
  const LhyNode<R>* xnodes;  // the Qx nodes evaluated exactly next to the table (det eta > 0 first: Qxm)
  int Qx, Qxm;
  LhyTab<R> tab;             // interpolated sums over the other nodes (tab.ni = 0: none)
  const C* twx;
  const C* twy;
  const C* twz;
  C* psi[2];                 // psi buffers (2 fields each)
  C* hp[2];                  // H psi buffers
  C* ax[2];                  // aux: field 0 = (Phi1, Phi2), field 1 = (muL1, muL2)
  C* rb[2];                  // residual buffers (current / previous by parity of n)
  C* pb[2];                  // direction buffers (current / previous)
  C* z;                      // preconditioned residual
  C* W;                      // transform workspace, 3 fields
  const C* gin;              // generic in/out of the plain passes
  C* gout;
  double* partials;
  unsigned* counter;
  DevState* st;
  TraceDev* trace;
  const R* kin_tab;          // ITE: e^{-dtau k_a^2/4} per index ([nx] x, [ny] y, [nz] z), then dtau
  int MX, M, nf, f0;         // launch shape: rows per block, columns per tile, fields
  int gate;                  // Gate
  int flag;                  // op-specific (trial / r given / p given)
  int ctrl;                  // run the controller step in the last block
  int diag;                  // P_V part of the preconditioner
  int blend;                 // weighted P_V / P_Delta combination (mode 4)
  long long wait_polls;      // poll budget of a TMA tile wait before the pass reports a timeout
};

template <class R> __device__ __forceinline__ bool gate_open(const KArgs<R>& a) {
  if (a.gate == GATE_ALWAYS) return true;
  const int ph = __ldcg(&a.st->phase);
  return a.gate == GATE_NEW_ITER ? (ph == PH_NEW_ITER) : (ph != PH_DONE);
}

// Batched launches: one launch runs the same pass for up to KB_MAX instances
// of one grid shape, blockIdx.y selecting the instance.  The descriptors (and
// the column passes' tensor maps) travel in the kernel's parameter block.
constexpr int KB_MAX = 16;
template <class R> struct KBatch {
  CUtensorMap tm[KB_MAX];
  KArgs<R> k[KB_MAX];
};
static_assert(sizeof(KBatch<double>) <= 32764, "batched kernel parameters exceed the 32 KB limit");

// Points whose global loads are issued together before any store of the chunk
// (the buffers may alias as far as the compiler knows, so loads and stores are
// grouped explicitly to keep several loads in flight per thread).
template <class R> struct ChunkW;
template <> struct ChunkW<float> { static constexpr int v = 4; };
template <> struct ChunkW<double> { static constexpr int v = 2; };

// Grid points evaluated together in the LHY node loops (independent chains;
// FP32: two pairs of packed lanes).
template <class R> struct LhyNP;
template <> struct LhyNP<float> { static constexpr int v = 4; };
template <> struct LhyNP<double> { static constexpr int v = 2; };

template <class R> __device__ __forceinline__ LhyCoef<R> lhy_coef(const KArgs<R>& a) {
  LhyCoef<R> c;
  c.g11 = a.g11;
  c.g22 = a.g22;
  c.g12 = a.g12;
  c.d11 = a.d11;
  c.d22 = a.d22;
  c.d12 = a.d12;
  c.nskip = a.nskip;
  return c;
}

template <class R> __device__ __forceinline__ R wavenum(int j, int n, R dk) {
  return dk * (R)(j < (n >> 1) ? j : j - n);
}

// Row-pass ops that read their transform outputs back from shared memory.
template <class Op, class = void> struct StageOut {
  static constexpr bool v = false;
};
template <class Op> struct StageOut<Op, std::void_t<decltype(Op::STAGE_OUT)>> {
  static constexpr bool v = Op::STAGE_OUT;
};

// Minimum resident blocks per SM a row-pass op asks the compiler to allow for
// (caps its registers); 1 unless the op says otherwise.
template <class Op, class = void> struct MinBlocks {
  static constexpr int v = 1;
};
template <class Op> struct MinBlocks<Op, std::void_t<decltype(Op::MINB)>> {
  static constexpr int v = Op::MINB;
};

// Row-pass ops whose LHY terms come from the interpolation table plus the
// exactly evaluated nodes (they stage the exact nodes only).
template <class Op, class = void> struct LhyTabOp {
  static constexpr bool v = false;
};
template <class Op> struct LhyTabOp<Op, std::void_t<decltype(Op::LHY_TAB)>> {
  static constexpr bool v = Op::LHY_TAB;
};

// Every pass runs whole warps: the block reductions and the warp exchanges use
// full-mask shuffles.  A row (x) pass gives each row L/8 threads and a column
// pass each column L/8 threads, so a block holds a multiple of
// whole_warp_rows(L) rows or columns.
__host__ __device__ constexpr int gcd_i(int a, int b) { return b == 0 ? a : gcd_i(b, a % b); }
__host__ __device__ constexpr int whole_warp_rows(int L) { return 32 / gcd_i(L / 8, 32); }

// Threads per block of a row pass: 256 unless the op asks for fewer, rounded
// down to whole warps of whole rows (at least one such group).
template <class Op, class = void> struct MaxThreadsWant {
  static constexpr int v = 256;
};
template <class Op> struct MaxThreadsWant<Op, std::void_t<decltype(Op::MAXT)>> {
  static constexpr int v = Op::MAXT;
};
template <class Op> struct MaxThreads {
  static constexpr int G = whole_warp_rows(Op::L) * (Op::L / 8);
  static constexpr int W = MaxThreadsWant<Op>::v;
  static constexpr int v = W >= G ? W - W % G : G;
};

// ----------------------------------------------------------------------------
// Row (x) pass kernel
// ----------------------------------------------------------------------------
template <class Op> __device__ __forceinline__ void xpass_body(const KArgs<typename Op::R>& a) {
  using R = typename Op::R;
  using C = C2<R>;
  constexpr int L = Op::L, NF = Op::NF, NS = Op::NS;
  constexpr int NSR = NS > 0 ? NS : 1;
  constexpr int TPL = L / 8;
  constexpr int LP = row_len_padded<R, L>();
  if (!gate_open(a)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);
  LhyNode<R>* nodes = reinterpret_cast<LhyNode<R>*>(tw + L);
  C* buf = reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(nodes) + (Op::USES_LHY ? lhy_stage_bytes<R>(a.Q) : 0));
  RedSmem<NSR>* red = reinterpret_cast<RedSmem<NSR>*>(buf + NF * a.MX * LP);
  const int tid = threadIdx.x;
  const int mrow = tid / TPL, t = tid - mrow * TPL;
  for (int i = tid; i < L; i += blockDim.x) tw[i] = a.twx[i];
  if constexpr (Op::USES_LHY) {
    if constexpr (LhyTabOp<Op>::v) stage_lhy_nodes(nodes, a.xnodes, a.Qx);
    else stage_lhy_nodes(nodes, a.nodes, a.Q);
  }
  __syncthreads();
  typename Op::Uni u;
  Op::uniform(a, u);
  PAcc<R> acc[NSR];
  const int rows = a.ny * a.nz;
  const int ngroups = (rows + a.MX - 1) / a.MX;
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int row = grp * a.MX + mrow;
    const bool valid = row < rows;
    C v[NF][8];
    Op::load(a, u, row, valid, t, v, acc);
    fft_line<C, L, Op::INV, NF>(v, buf + mrow * LP, a.MX * LP, tw, t, RowIdx<PadShift<R>::v>{});
    if constexpr (StageOut<Op>::v) {
      // park the transform outputs in the (idle) exchange buffer: the FFT
      // registers are dead during the epilogue, which frees them for it
      C* sm = buf + mrow * LP;
      const RowIdx<PadShift<R>::v> si{};
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int e = 0; e < 8; ++e) sm[f * a.MX * LP + si(Plan<L>::exit_pos(Op::INV, t, e))] = v[f][e];
      Op::store_staged(a, u, row, valid, t, sm, a.MX * LP, acc, nodes);
      // the next row group's exchanges reuse the buffer (a warp's own rows when
      // the length is a power of two, else rows that may straddle warps)
      if constexpr (IsPow2<L>::v) __syncwarp();
      else __syncthreads();
    } else {
      Op::store(a, u, row, valid, t, v, acc, nodes);
    }
  }
  if constexpr (NS > 0) {
    if (reduce_blocks<NS>(acc, a.partials, a.counter, Op::out(a, u), *red)) {
      if (threadIdx.x == 0) Op::finish(a, u);
    }
  }
}

// Row-pass entry points.  A min-blocks bound is given only when the op asks for
// more than one resident block: an explicit 1 lets the compiler take far more
// registers than the default heuristic does.
template <class Op> __global__ void __launch_bounds__(MaxThreads<Op>::v) xpass_kernel(KArgs<typename Op::R> a) {
  xpass_body<Op>(a);
}
template <class Op>
__global__ void __launch_bounds__(MaxThreads<Op>::v, MinBlocks<Op>::v) xpass_kernel_mb(KArgs<typename Op::R> a) {
  xpass_body<Op>(a);
}
template <class Op>
__global__ void __launch_bounds__(MaxThreads<Op>::v) xpass_kernel_b(const __grid_constant__ KBatch<typename Op::R> kb) {
  xpass_body<Op>(kb.k[blockIdx.y]);
}
template <class Op>
__global__ void __launch_bounds__(MaxThreads<Op>::v, MinBlocks<Op>::v)
    xpass_kernel_bmb(const __grid_constant__ KBatch<typename Op::R> kb) {
  xpass_body<Op>(kb.k[blockIdx.y]);
}

#ifndef EGPE_COL_STAGES
#define EGPE_COL_STAGES 2
#endif
// Tiles in flight per block of a TMA-fed column pass (one transformed, the
// rest loading).
constexpr int kColStages = EGPE_COL_STAGES;

// Threads per block of a column pass.  The power-of-two lengths are bound to
// 512 threads (tile rows of 64 to 256 bytes, chosen at run time); the
// mixed-radix lengths keep 128-byte rows, max(128 B / element, whole warps)
// columns times L/8 threads, and give the compiler that exact bound.
template <class Op> struct ColMaxThreads {
  static constexpr int TPL = Op::L / 8;
  static constexpr int MC = (int)(128 / sizeof(C2<typename Op::R>));
  static constexpr int MW = whole_warp_rows(Op::L);
  static constexpr int exact = (MC > MW ? MC : MW) * TPL;
  static constexpr int v = IsPow2<Op::L>::v ? 512 : exact;
  static constexpr int minb = 1;
};

// Columns per tile at the default 128-byte tile rows (what the host picks for
// every grid while the column tile width is untuned): the kernels for this
// width take it as a compile-time constant.
template <class Op> struct ColDefaultM {
  static constexpr int TPL = Op::L / 8;
  static constexpr int MB = (int)(128 / sizeof(C2<typename Op::R>));
  static constexpr int M0 = IsPow2<Op::L>::v ? (MB < 512 / TPL ? MB : 512 / TPL) : MB;
  static constexpr int v = M0 > whole_warp_rows(Op::L) ? M0 : whole_warp_rows(Op::L);
};
// Launch bounds of a column kernel: the run-time width keeps ColMaxThreads; a
// compile-time width MC has exactly MC L/8 threads, and the FP32 plain y/z
// passes (the ColPlain op, small epilogue) of up to 256 threads ask for three
// resident blocks, as their run-time-width build reached without a bound.
template <class Op> struct ColMinB {
  static constexpr int v = 1;
};
template <class Op, int MC> struct ColBounds {
  static constexpr int threads = MC > 0 ? MC * (Op::L / 8) : ColMaxThreads<Op>::v;
  static constexpr int minb = MC > 0 && threads <= 256 ? ColMinB<Op>::v : ColMaxThreads<Op>::minb;
};

// ----------------------------------------------------------------------------
// Column (y or z) pass kernel
// ----------------------------------------------------------------------------
template <class Op, int MC> __device__ __forceinline__ void colpass_body(const KArgs<typename Op::R>& a) {
  using R = typename Op::R;
  using C = C2<R>;
  constexpr int L = Op::L, NS = Op::NS;
  constexpr int NSR = NS > 0 ? NS : 1;
  if (!gate_open(a)) return;
  const int M = MC > 0 ? MC : a.M;  // columns per tile
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);
  C* buf = tw + L;  // two exchange buffers of M lines each
  RedSmem<NSR>* red = reinterpret_cast<RedSmem<NSR>*>(buf + 2 * M * L);
  const int tid = threadIdx.x;
  const int m = tid % M, t = tid / M;
  const C* twsrc = (Op::AXIS == 1) ? a.twy : a.twz;
  for (int i = tid; i < L; i += blockDim.x) tw[i] = twsrc[i];
  __syncthreads();
  typename Op::Uni u;
  Op::uniform(a, u);
  PAcc<R> acc[NSR];
  const int xb_n = a.nx / M;
  const int other_n = (Op::AXIS == 1) ? a.nz : a.ny;
  const int tiles = xb_n * other_n * a.nf;
  const size_t lstride = (Op::AXIS == 1) ? (size_t)a.nx : (size_t)a.nx * a.ny;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int xb = tile % xb_n;
    const int rest = tile / xb_n;
    const int o = rest % other_n;
    const int f = a.f0 + rest / other_n;
    const int x = xb * M + m;
    const size_t base = (size_t)f * a.N + (Op::AXIS == 1 ? (size_t)o * a.nx * a.ny : (size_t)o * a.nx) + x;
    const C* src = Op::src(a);
    C v[1][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[0][e] = src[base + (size_t)Plan<L>::entry_pos(Op::FIRST_INV, t, e) * lstride];
    Op::process(a, u, f, x, o, base, lstride, t, v, buf + m, tw, ColIdxT<MC>{M, M * L}, acc);
    // the last exchange's reads end before the next tile's first writes
    if constexpr (IsPow2<L>::v) __syncthreads();
  }
  if constexpr (NS > 0) {
    if (reduce_blocks<NS>(acc, a.partials, a.counter, Op::out(a, u), *red)) {
      if (threadIdx.x == 0) Op::finish(a, u);
    }
  }
}
template <class Op, int MC = 0>
__global__ void __launch_bounds__(ColBounds<Op, MC>::threads, ColBounds<Op, MC>::minb)
    colpass_kernel(KArgs<typename Op::R> a) {
  colpass_body<Op, MC>(a);
}
template <class Op, int MC = 0>
__global__ void __launch_bounds__(ColBounds<Op, MC>::threads, ColBounds<Op, MC>::minb)
    colpass_kernel_b(const __grid_constant__ KBatch<typename Op::R> kb) {
  colpass_body<Op, MC>(kb.k[blockIdx.y]);
}

// ----------------------------------------------------------------------------
// Column (y or z) pass fed by TMA.  The tensor map describes the workspace as
// a 3D array (x in 8-byte elements, y, z x fields); one box is one tile, M
// columns by the whole line, landing in shared memory position-major exactly
// as the FFT's column layout expects.  While tile i is transformed, tile i+1
// is already loading into the other buffer.  Results go straight to global
// memory from registers.
// ----------------------------------------------------------------------------
template <class Op, int MC>
__device__ __forceinline__ void colpass_tma_body(const CUtensorMap* tm, const KArgs<typename Op::R>& a) {
  using R = typename Op::R;
  using C = C2<R>;
  constexpr int L = Op::L, NS = Op::NS;
  constexpr int NSR = NS > 0 ? NS : 1;
  constexpr int NST = kColStages;
  if (!gate_open(a)) return;
  const int M = MC > 0 ? MC : a.M;  // columns per tile
  extern __shared__ __align__(128) unsigned char smraw_tma[];
  const int tileC = M * L;
  C* tiles = reinterpret_cast<C*>(smraw_tma);  // NST tiles, then the second exchange buffer
  C* xbuf = tiles + NST * tileC;
  C* tw = xbuf + tileC;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tw + L);
  RedSmem<NSR>* red = reinterpret_cast<RedSmem<NSR>*>(bar + NST);
  const int tid = threadIdx.x;
  const int m = tid % M, t = tid / M;
  const C* twsrc = (Op::AXIS == 1) ? a.twy : a.twz;
  for (int i = tid; i < L; i += blockDim.x) tw[i] = twsrc[i];
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  typename Op::Uni u;
  Op::uniform(a, u);
  PAcc<R> acc[NSR];
  const int xb_n = a.nx / M;
  const int other_n = (Op::AXIS == 1) ? a.nz : a.ny;
  const int tiles_n = xb_n * other_n * a.nf;
  const size_t lstride = (Op::AXIS == 1) ? (size_t)a.nx : (size_t)a.nx * a.ny;
  const uint32_t bytes = (uint32_t)(tileC * sizeof(C));
  constexpr int ESZ = (int)(sizeof(C) / 8);  // 8-byte TMA elements per complex value
  auto issue = [&](int tile, int b) {
    const int xb = tile % xb_n;
    const int rest = tile / xb_n;
    const int o = rest % other_n;
    const int f = a.f0 + rest / other_n;
    const int c0 = xb * M * ESZ;
    const int c1 = (Op::AXIS == 1) ? 0 : o;
    const int c2 = (Op::AXIS == 1) ? f * a.nz + o : f * a.nz;
    fence_proxy_async();
    mbar_expect_tx(&bar[b], bytes);
    tma_load_3d(tiles + b * tileC, tm, c0, c1, c2, &bar[b]);
  };
  // iteration q of this block handles tile blockIdx.x + q gridDim.x in buffer q % NST;
  // the copies of the next NST - 1 iterations are in flight while one is transformed
  auto tile_of = [&](int q) { return (int)blockIdx.x + q * (int)gridDim.x; };
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NST - 1; ++q)
      if (tile_of(q) < tiles_n) issue(tile_of(q), q);
  }
  bool timed_out = false;
  int it = 0;
  for (int tile = blockIdx.x; tile < tiles_n; tile += gridDim.x, ++it) {
    const int b = it % NST;
    const int ahead = tile_of(it + NST - 1);
    // its buffer was last used by iteration it - 1, which ended with a barrier
    if (tid == 0 && ahead < tiles_n) issue(ahead, (it + NST - 1) % NST);
    const bool ok = mbar_wait(&bar[b], (uint32_t)((it / NST) & 1), a.wait_polls);
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    C* tb = tiles + b * tileC;
    C v[1][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[0][e] = tb[Plan<L>::entry_pos(Op::FIRST_INV, t, e) * M + m];
    // power-of-two lengths exchange through the second buffer first, and the
    // barrier of that exchange orders these reads before the tile's reuse;
    // the mixed-radix passes work in place in the tile
    if constexpr (!IsPow2<L>::v) __syncthreads();
    const int xb = tile % xb_n;
    const int rest = tile / xb_n;
    const int o = rest % other_n;
    const int f = a.f0 + rest / other_n;
    const int x = xb * M + m;
    const size_t base = (size_t)f * a.N + (Op::AXIS == 1 ? (size_t)o * a.nx * a.ny : (size_t)o * a.nx) + x;
    Op::process(a, u, f, x, o, base, lstride, t, v, tb + m, tw, ColIdxT<MC>{M, (int)(xbuf - tb)}, acc);
    __syncthreads();  // buffer b may be refilled, and the second buffer rewritten, from here on
  }
  if (timed_out) {
    // let every copy already issued land before exiting: these waits keep the
    // full budget whatever a.wait_polls says, so no copy can still write into
    // shared memory once the block has left
    for (int q = it; q < it + NST; ++q)
      if (tile_of(q) < tiles_n) mbar_wait(&bar[q % NST], (uint32_t)((q / NST) & 1), kTmaWaitPolls);
    if (tid == 0) {
      a.st->timeout = 1;  // sticky: every later controller step ends the run
      a.st->status = 7;   // EGPE_ERR_TIMEOUT
      a.st->phase = PH_DONE;
    }
  }
  if constexpr (NS > 0) {
    if (reduce_blocks<NS>(acc, a.partials, a.counter, Op::out(a, u), *red)) {
      if (threadIdx.x == 0) Op::finish(a, u);
    }
  }
}
template <class Op, int MC = 0>
__global__ void __launch_bounds__(ColBounds<Op, MC>::threads, ColBounds<Op, MC>::minb)
    colpass_tma_kernel(const __grid_constant__ CUtensorMap tm, KArgs<typename Op::R> a) {
  colpass_tma_body<Op, MC>(&tm, a);
}
template <class Op, int MC = 0>
__global__ void __launch_bounds__(ColBounds<Op, MC>::threads, ColBounds<Op, MC>::minb)
    colpass_tma_kernel_b(const __grid_constant__ KBatch<typename Op::R> kb) {
  colpass_tma_body<Op, MC>(&kb.tm[blockIdx.y], kb.k[blockIdx.y]);
}

struct NoUni {};

// ----------------------------------------------------------------------------
// Plain transforms (diagnostic entry point and the y passes of the pipelines)
// ----------------------------------------------------------------------------
template <class R_, int L_, bool INV_> struct XPlain {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "x-plain";
  static double alg_bytes(const KArgs<R>& a) { return 2.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 1, NS = 0;
  static constexpr bool INV = INV_, USES_LHY = false;
  using Uni = NoUni;
  static __device__ void uniform(const KArgs<R>&, Uni&) {}
  static __device__ void load(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[1][8], PAcc<R>*) {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      v[0][e] = valid ? a.gin[(size_t)row * a.nx + Plan<L>::entry_pos(INV, t, e)] : cmk<C>(0, 0);
  }
  static __device__ void store(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[1][8], PAcc<R>*,
                               const LhyNode<R>*) {
    if (!valid) return;
#pragma unroll
    for (int e = 0; e < 8; ++e) a.gout[(size_t)row * a.nx + Plan<L>::exit_pos(INV, t, e)] = v[0][e];
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_, int AXIS_, bool INV_> struct ColPlain {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = AXIS_ == 1 ? "y-pass" : "z-pass";
  static double alg_bytes(const KArgs<R>& a) { return 2.0 * a.nf * a.N * sizeof(C); }
  static constexpr int L = L_, NS = 0, AXIS = AXIS_;
  static constexpr bool INV = INV_;
  using Uni = NoUni;
  static __device__ void uniform(const KArgs<R>&, Uni&) {}
  static constexpr bool FIRST_INV = INV_;
  static __device__ const C* src(const KArgs<R>& a) { return a.gin; }
  template <class SI>
  static __device__ void process(const KArgs<R>& a, Uni&, int, int, int, size_t base, size_t ls, int t,
                                 C (&v)[1][8], C* sm, const C* tw, SI si, PAcc<R>*) {
    fft_line<C, L, INV, 1>(v, sm, 0, tw, t, si);
#pragma unroll
    for (int e = 0; e < 8; ++e) a.gout[base + (size_t)Plan<L>::exit_pos(INV, t, e) * ls] = v[0][e];
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};
template <int L_, int AXIS_, bool INV_> struct ColMinB<ColPlain<float, L_, AXIS_, INV_>> {
  static constexpr int v = 3;
};

// ----------------------------------------------------------------------------
// Energy / gradient pipeline (Eq. 1, coupled eGPE):
//   x fwd (psi or trial psi; packed dipolar source) -> y fwd -> z fused
//   (kinetic |k|^2/2, dipolar kernel, Parseval kinetic energy) -> y inv ->
//   x inv + H psi, LHY, energy sums.
// Workspace fields: 0, 1 = psi_1, psi_2; 2 = zeta = sum_j gdd_1j n_j + i sum_j gdd_2j n_j
// (both dipolar potentials from one complex transform: the kernel is real and
// even, so Phi_1 = Re and Phi_2 = Im of the inverse).
// ----------------------------------------------------------------------------
template <class R> struct EgUni {
  int cur, slot, nsel;
  R ca[2], cb[2];
};

// Controller step after an energy/gradient evaluation (last block, one thread):
// ctrl 1 = NCG (start point or trial), ctrl 2 = end of an imaginary-time step.
template <class R> __device__ __forceinline__ void eg_ctrl(const KArgs<R>& a) {
  if (a.ctrl == 2) {
    a.st->ffts += 20;  // two kinetic half steps (8) and two evaluations (12)
    ctrl_after_ite(a.st);
  } else if (a.ctrl) {
    a.st->ffts += 6;
    ctrl_after_eg(a.st, a.flag ? 1 : 0, a.trace);
  }
}

template <class R_, int L_> struct XFwdEG {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "x-fwd energy";
  static double alg_bytes(const KArgs<R>& a) { return (a.flag ? 9.0 : 5.0) * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 3, NS = 0;
  static constexpr bool INV = false, USES_LHY = false;
  using Uni = EgUni<R>;
  static __device__ void uniform(const KArgs<R>& a, Uni& u) {
    u.cur = __ldcg(&a.st->cur);
    u.slot = a.flag ? (u.cur ^ 1) : u.cur;
    u.nsel = __ldcg(&a.st->n) & 1;
    R c[4];
    load_uniforms<R, 4>({&a.st->coef_a[0], &a.st->coef_a[1], &a.st->coef_b[0], &a.st->coef_b[1]}, c);
    u.ca[0] = c[0];
    u.ca[1] = c[1];
    u.cb[0] = c[2];
    u.cb[1] = c[3];
  }
  static __device__ void load(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[3][8], PAcc<R>*) {
    const C* src = a.psi[u.cur];
    const C* pd = a.pb[u.nsel];
    C* dst = a.psi[u.slot];
    const size_t N = a.N;
    constexpr int CH = ChunkW<R>::v;
#pragma unroll
    for (int e0 = 0; e0 < 8; e0 += CH) {
      C p1[CH], p2[CH], q1[CH], q2[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const size_t idx = (size_t)row * a.nx + Plan<L>::entry_pos(false, t, e0 + j);
        p1[j] = valid ? src[idx] : cmk<C>(0, 0);
        p2[j] = valid ? src[N + idx] : cmk<C>(0, 0);
        if (a.flag) {
          q1[j] = valid ? pd[idx] : cmk<C>(0, 0);
          q2[j] = valid ? pd[N + idx] : cmk<C>(0, 0);
        }
      }
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int e = e0 + j;
        if (a.flag) {  // trial point on the geodesic (Sec. III), renormalised (Sec. V)
          p1[j] = cmk<C>(u.ca[0] * p1[j].x + u.cb[0] * q1[j].x, u.ca[0] * p1[j].y + u.cb[0] * q1[j].y);
          p2[j] = cmk<C>(u.ca[1] * p2[j].x + u.cb[1] * q2[j].x, u.ca[1] * p2[j].y + u.cb[1] * q2[j].y);
          if (valid) {
            const size_t idx = (size_t)row * a.nx + Plan<L>::entry_pos(false, t, e);
            dst[idx] = p1[j];
            dst[N + idx] = p2[j];
          }
        }
        const R n1 = cabs2(p1[j]), n2 = cabs2(p2[j]);
        v[0][e] = p1[j];
        v[1][e] = p2[j];
        v[2][e] = cmk<C>(a.d11 * n1 + a.d12 * n2, a.d21 * n1 + a.d22 * n2);
      }
    }
  }
  static __device__ void store(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[3][8], PAcc<R>*,
                               const LhyNode<R>*) {
    if (!valid) return;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = (size_t)row * a.nx + Plan<L>::exit_pos(false, t, e);
#pragma unroll
      for (int f = 0; f < 3; ++f) a.W[(size_t)f * a.N + idx] = v[f][e];
    }
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct ZEg {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "z fused energy";
  static double alg_bytes(const KArgs<R>& a) { return 6.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NS = 2, AXIS = 2;
  struct Uni {
    int slot;
  };
  static __device__ void uniform(const KArgs<R>& a, Uni& u) {
    const int cur = __ldcg(&a.st->cur);
    u.slot = a.flag ? (cur ^ 1) : cur;
  }
  static constexpr bool FIRST_INV = false;
  static __device__ const C* src(const KArgs<R>& a) { return a.W; }
  template <class SI>
  static __device__ void process(const KArgs<R>& a, Uni&, int f, int x, int y, size_t base, size_t ls, int t,
                                 C (&v)[1][8], C* sm, const C* tw, SI si, PAcc<R>* acc) {
    fft_line<C, L, false, 1>(v, sm, 0, tw, t, si);
    const R kx = wavenum<R>(x, a.nx, a.dkx), ky = wavenum<R>(y, a.ny, a.dky);
    const R kxy2 = kx * kx + ky * ky;
    R ekin = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const R kz = wavenum<R>(Plan<L>::exit_pos(false, t, e), a.nz, a.dkz);
      const R k2 = kxy2 + kz * kz;
      R mult;
      if (f < 2) {
        const R t2 = R(0.5) * k2;
        ekin += t2 * cabs2(v[0][e]);
        mult = t2 * a.invN;
      } else {
        mult = (k2 > R(0)) ? (R(3) * kz * kz / k2 - R(1)) * a.invN : R(0);
      }
      v[0][e] = cscale(v[0][e], mult);
    }
    if (f < 2) acc[f].add(ekin);
    col_after<L>(sm, si);
    fft_line<C, L, true, 1>(v, sm, 0, tw, t, si);
#pragma unroll
    for (int e = 0; e < 8; ++e) a.W[base + (size_t)Plan<L>::exit_pos(true, t, e) * ls] = v[0][e];
  }
  static __device__ double* out(const KArgs<R>& a, Uni& u) { return a.st->egz[u.slot]; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

// mu_LHY,i and the LHY energy density at NP points: the interpolation table
// plus the exactly evaluated nodes; F from Euler's identity for the degree-5/2
// density, F = (2/5)(n1 mu1 + n2 mu2).
template <class R, int NP>
__device__ __forceinline__ void lhy_terms(const KArgs<R>& a, const LhyNode<R>* nodes, const LhyCoef<R>& cf,
                                          const R (&n1)[NP], const R (&n2)[NP], R (&F)[NP], R (&m1)[NP],
                                          R (&m2)[NP]) {
#pragma unroll
  for (int j = 0; j < NP; ++j) m1[j] = m2[j] = R(0);
  if (a.Qx > 0) {
    // exact nodes two points at a time (few registers for a rarely long loop)
#pragma unroll
    for (int j = 0; j < NP; j += 2) {
      const R q1[2] = {n1[j], n1[j + 1]}, q2[2] = {n2[j], n2[j + 1]};
      R f[2], x1[2], x2[2];
      lhy_points<R, 2>(nodes, a.Qx, a.Qxm, cf, q1, q2, f, x1, x2);
      m1[j] = x1[0];
      m1[j + 1] = x1[1];
      m2[j] = x2[0];
      m2[j + 1] = x2[1];
    }
  }
  if (a.tab.ni > 0) {
    R t1[NP], t2[NP];
    lhy_tab_mu<R, NP>(a.tab, n1, n2, t1, t2);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      m1[j] += t1[j];
      m2[j] += t2[j];
    }
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) F[j] = R(0.4) * (n1[j] * m1[j] + n2[j] * m2[j]);
}

// n'^T (d^2 F/dn dn) n' at NP points: table plus exactly evaluated nodes.
template <class R, int NP>
__device__ __forceinline__ void lhy_second(const KArgs<R>& a, const LhyNode<R>* nodes, const LhyCoef<R>& cf,
                                           const R (&n1)[NP], const R (&n2)[NP], const R (&n1p)[NP],
                                           const R (&n2p)[NP], R (&H)[NP]) {
#pragma unroll
  for (int j = 0; j < NP; ++j) H[j] = R(0);
  if (a.Qx > 0) {
#pragma unroll
    for (int j = 0; j < NP; j += 2) {
      const R q1[2] = {n1[j], n1[j + 1]}, q2[2] = {n2[j], n2[j + 1]};
      const R p1[2] = {n1p[j], n1p[j + 1]}, p2[2] = {n2p[j], n2p[j + 1]};
      R hx[2];
      lhy_hess<R, 2>(nodes, a.Qx, a.Qxm, cf, q1, q2, p1, p2, hx);
      H[j] = hx[0];
      H[j + 1] = hx[1];
    }
  }
  if (a.tab.ni > 0) {
    R t[NP];
    lhy_tab_hess<R, NP>(a.tab, n1, n2, n1p, n2p, t);
#pragma unroll
    for (int j = 0; j < NP; ++j) H[j] += t[j];
  }
}

template <class R_, int L_> struct XInvEG {
  using R = R_;
  using C = C2<R>;
  static constexpr int MAXT = 128;
  static constexpr int MINB = sizeof(R_) == 4 ? EGPE_EG_MINB : 1;
  static constexpr const char* NAME = "x-inv energy+LHY";
  static double alg_bytes(const KArgs<R>& a) { return 9.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 3, NS = EG_NS;
  static constexpr bool INV = true, USES_LHY = true, LHY_TAB = true;
  using Uni = EgUni<R>;
  static __device__ void uniform(const KArgs<R>& a, Uni& u) { XFwdEG<R, L>::uniform(a, u); }
  static __device__ void load(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[3][8], PAcc<R>*) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = (size_t)row * a.nx + Plan<L>::entry_pos(true, t, e);
#pragma unroll
      for (int f = 0; f < 3; ++f) v[f][e] = valid ? a.W[(size_t)f * a.N + idx] : cmk<C>(0, 0);
    }
  }
  static constexpr int NP = LhyNP<R>::v;
  static constexpr bool STAGE_OUT = true;
  static __device__ void store_staged(const KArgs<R>& a, Uni& u, int row, bool valid, int t, const C* sm, int fs,
                                      PAcc<R>* acc, const LhyNode<R>* nodes) {
    const RowIdx<PadShift<R>::v> si{};
    if (!valid) return;
    const C* ps = a.psi[u.slot];
    C* hp = a.hp[u.slot];
    C* ax = a.ax[u.slot];
    const size_t N = a.N;
    const int y = row % a.ny, z = row / a.ny;
    const R Y = -a.Ly + (R)y * a.hy, Z = -a.Lz + (R)z * a.hz;
    const R vyz = a.vy * Y * Y + a.vz * Z * Z;
    const LhyCoef<R> cf = lhy_coef(a);
    R s[EG_NS];
#pragma unroll
    for (int k = 0; k < EG_NS; ++k) s[k] = 0;
#pragma unroll
    for (int e0 = 0; e0 < 8; e0 += NP) {
      C p1[NP], p2[NP];
      R n1[NP], n2[NP], F[NP], m1[NP], m2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const size_t idx = (size_t)row * a.nx + Plan<L>::exit_pos(true, t, e0 + j);
        p1[j] = ps[idx];
        p2[j] = ps[N + idx];
        n1[j] = cabs2(p1[j]);
        n2[j] = cabs2(p2[j]);
      }
      lhy_terms<R, NP>(a, nodes, cf, n1, n2, F, m1, m2);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const int e = e0 + j;
        const int x = Plan<L>::exit_pos(true, t, e);
        const size_t idx = (size_t)row * a.nx + x;
        const R X = -a.Lx + (R)x * a.hx;
        const R V = a.vx * X * X + vyz;
        const int o = si(x);
        const C T1 = sm[o], T2 = sm[fs + o], PH = sm[2 * fs + o];
        const R phi1 = PH.x, phi2 = PH.y;
        const R U1 = V + a.g11 * n1[j] + a.g12 * n2[j] + phi1 + m1[j];
        const R U2 = V + a.g21 * n1[j] + a.g22 * n2[j] + phi2 + m2[j];
        const C H1 = cmk<C>(T1.x + U1 * p1[j].x, T1.y + U1 * p1[j].y);
        const C H2 = cmk<C>(T2.x + U2 * p2[j].x, T2.y + U2 * p2[j].y);
        hp[idx] = H1;
        hp[N + idx] = H2;
        ax[idx] = cmk<C>(phi1, phi2);
        ax[N + idx] = cmk<C>(m1[j], m2[j]);
        s[EG_TRAP] += V * (n1[j] + n2[j]);
        s[EG_CONTACT] += R(0.5) * (a.g11 * n1[j] * n1[j] + (a.g12 + a.g21) * n1[j] * n2[j] + a.g22 * n2[j] * n2[j]);
        s[EG_DIPOLAR] += R(0.5) * (n1[j] * phi1 + n2[j] * phi2);
        s[EG_LHY] += F[j];
        s[EG_MU1] += cdot(p1[j], H1);
        s[EG_MU2] += cdot(p2[j], H2);
        s[EG_NPHI1] += n1[j] * phi1;
        s[EG_NPHI2] += n2[j] * phi2;
        s[EG_NMUL1] += n1[j] * m1[j];
        s[EG_NMUL2] += n2[j] * m2[j];
        s[EG_NORM1] += n1[j];
        s[EG_NORM2] += n2[j];
      }
    }
#pragma unroll
    for (int k = 0; k < EG_NS; ++k) acc[k].add(s[k]);
  }
  static __device__ double* out(const KArgs<R>& a, Uni& u) { return a.st->eg[u.slot]; }
  static __device__ void finish(const KArgs<R>& a, Uni&) { eg_ctrl(a); }
};

// ----------------------------------------------------------------------------
// Preconditioner pipeline (Sec. IV.B): r = H psi - mu psi, z = P^{-1} r with
// P^{-1} = P_Delta^{-1} P_V^{-1}; sums for HS+ beta, projection and descent.
// ----------------------------------------------------------------------------
template <class R> struct PcUni {
  int cur, nsel, rgiven;
  R mu[2], shift[2], floor_[2];
  R wv;  // weight of P_V in the blended preconditioner
};
template <class R> __device__ __forceinline__ void pc_uniform(const KArgs<R>& a, PcUni<R>& u) {
  u.cur = __ldcg(&a.st->cur);
  u.nsel = __ldcg(&a.st->n) & 1;
  u.rgiven = a.flag;
  if constexpr (sizeof(R) == sizeof(double)) {
    u.wv = __ldcg(&a.st->opt.pc_blend);
    const double fl = __ldcg(&a.st->opt.pv_floor);
    for (int i = 0; i < 2; ++i) {
      u.mu[i] = __ldcg(&a.st->mu[i]);
      u.shift[i] = __ldcg(&a.st->shift[i]);
      u.floor_[i] = fl * u.shift[i];
    }
  } else {
    R c[6];
    load_uniforms<R, 6>(
        {&a.st->opt.pc_blend, &a.st->opt.pv_floor, &a.st->mu[0], &a.st->mu[1], &a.st->shift[0], &a.st->shift[1]}, c);
    u.wv = c[0];
    for (int i = 0; i < 2; ++i) {
      u.mu[i] = c[2 + i];
      u.shift[i] = c[4 + i];
      u.floor_[i] = c[1] * c[4 + i];
    }
  }
}

// Inputs of the preconditioner prologue at one point.
template <class R> struct PcIn {
  C2<R> p1, p2, h1, h2, ml;
};
template <class R>
__device__ __forceinline__ void pc_load(const KArgs<R>& a, const PcUni<R>& u, size_t idx, PcIn<R>& in) {
  const size_t N = a.N;
  if (u.rgiven) {
    in.h1 = a.rb[u.nsel][idx];
    in.h2 = a.rb[u.nsel][N + idx];
  } else {
    in.h1 = a.hp[u.cur][idx];
    in.h2 = a.hp[u.cur][N + idx];
  }
  if (a.diag || !u.rgiven) {
    in.p1 = a.psi[u.cur][idx];
    in.p2 = a.psi[u.cur][N + idx];
  }
  if (a.diag) in.ml = a.ax[u.cur][N + idx];
}
// r_i = H_i psi_i - mu_i psi_i (stored unless given) and w_i = P_V^{-1} r_i when diag.
template <class R>
__device__ __forceinline__ void pc_apply(const KArgs<R>& a, const PcUni<R>& u, size_t idx, R V, const PcIn<R>& in,
                                         C2<R>& w1, C2<R>& w2) {
  using C = C2<R>;
  C r1, r2;
  if (u.rgiven) {
    r1 = in.h1;
    r2 = in.h2;
  } else {
    r1 = cmk<C>(in.h1.x - u.mu[0] * in.p1.x, in.h1.y - u.mu[0] * in.p1.y);
    r2 = cmk<C>(in.h2.x - u.mu[1] * in.p2.x, in.h2.y - u.mu[1] * in.p2.y);
    a.rb[u.nsel][idx] = r1;
    a.rb[u.nsel][(size_t)a.N + idx] = r2;
  }
  if (a.diag) {
    const R n1 = cabs2(in.p1), n2 = cabs2(in.p2);
    R P1 = u.shift[0] + V + a.g11 * n1 + a.g12 * n2 + in.ml.x;
    R P2 = u.shift[1] + V + a.g21 * n1 + a.g22 * n2 + in.ml.y;
    P1 = P1 > u.floor_[0] ? P1 : u.floor_[0];
    P2 = P2 > u.floor_[1] ? P2 : u.floor_[1];
    w1 = cscale(r1, R(1) / P1);
    w2 = cscale(r2, R(1) / P2);
  } else {
    w1 = r1;
    w2 = r2;
  }
}

// Inputs of the preconditioner sums at one point.
template <class R> struct PcSumIn {
  C2<R> r1, r2, q1, q2, d1, d2, p1, p2;
};
template <class R>
__device__ __forceinline__ void pc_sum_load(const KArgs<R>& a, const PcUni<R>& u, size_t idx, PcSumIn<R>& in) {
  const size_t N = a.N;
  in.r1 = a.rb[u.nsel][idx];
  in.r2 = a.rb[u.nsel][N + idx];
  in.q1 = a.rb[u.nsel ^ 1][idx];
  in.q2 = a.rb[u.nsel ^ 1][N + idx];
  in.d1 = a.pb[u.nsel ^ 1][idx];
  in.d2 = a.pb[u.nsel ^ 1][N + idx];
  in.p1 = a.psi[u.cur][idx];
  in.p2 = a.psi[u.cur][N + idx];
}
template <class R>
__device__ __forceinline__ void pc_sum_add(const PcSumIn<R>& in, C2<R> z1, C2<R> z2, R* s) {
  const C2<R> dr1 = csub(in.r1, in.q1), dr2 = csub(in.r2, in.q2);
  s[PC_SRZ] += cdot(dr1, z1) + cdot(dr2, z2);
  s[PC_SRP] += cdot(dr1, in.d1) + cdot(dr2, in.d2);
  s[PC_ZPSI1] += cdot(z1, in.p1);
  s[PC_ZPSI2] += cdot(z2, in.p2);
  s[PC_PPPSI1] += cdot(in.d1, in.p1);
  s[PC_PPPSI2] += cdot(in.d2, in.p2);
  s[PC_ZR1] += cdot(z1, in.r1);
  s[PC_ZR2] += cdot(z2, in.r2);
  s[PC_PPR1] += cdot(in.d1, in.r1);
  s[PC_PPR2] += cdot(in.d2, in.r2);
  s[PC_PSIR1] += cdot(in.p1, in.r1);
  s[PC_PSIR2] += cdot(in.p2, in.r2);
  s[PC_RR1] += cabs2(in.r1);
  s[PC_RR2] += cabs2(in.r2);
}

template <class R_, int L_> struct XFwdPC {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "x-fwd precond";
  static double alg_bytes(const KArgs<R>& a) { return (a.diag ? 9.0 : 8.0) * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 2, NS = 0;
  static constexpr bool INV = false, USES_LHY = false;
  using Uni = PcUni<R>;
  static __device__ void uniform(const KArgs<R>& a, Uni& u) { pc_uniform(a, u); }
  static __device__ void load(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[2][8], PAcc<R>*) {
    const int y = row % a.ny, z = row / a.ny;
    const R Y = -a.Ly + (R)y * a.hy, Z = -a.Lz + (R)z * a.hz;
    const R vyz = a.vy * Y * Y + a.vz * Z * Z;
    constexpr int CH = ChunkW<R>::v;
#pragma unroll
    for (int e0 = 0; e0 < 8; e0 += CH) {
      PcIn<R> in[CH];
      if (valid) {
#pragma unroll
        for (int j = 0; j < CH; ++j)
          pc_load<R>(a, u, (size_t)row * a.nx + Plan<L>::entry_pos(false, t, e0 + j), in[j]);
      }
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int e = e0 + j;
        v[0][e] = cmk<C>(0, 0);
        v[1][e] = cmk<C>(0, 0);
        if (valid) {
          const int x = Plan<L>::entry_pos(false, t, e);
          const R X = -a.Lx + (R)x * a.hx;
          pc_apply<R>(a, u, (size_t)row * a.nx + x, a.vx * X * X + vyz, in[j], v[0][e], v[1][e]);
        }
      }
    }
  }
  static __device__ void store(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[2][8], PAcc<R>*,
                               const LhyNode<R>*) {
    if (!valid) return;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = (size_t)row * a.nx + Plan<L>::exit_pos(false, t, e);
      a.W[idx] = v[0][e];
      a.W[(size_t)a.N + idx] = v[1][e];
    }
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct ZPc {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "z fused precond";
  static double alg_bytes(const KArgs<R>& a) { return 4.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NS = 0, AXIS = 2;
  struct Uni {
    R shift[2];
  };
  static __device__ void uniform(const KArgs<R>& a, Uni& u) {
    load_uniforms<R, 2>({&a.st->shift[0], &a.st->shift[1]}, u.shift);
  }
  static constexpr bool FIRST_INV = false;
  static __device__ const C* src(const KArgs<R>& a) { return a.W; }
  template <class SI>
  static __device__ void process(const KArgs<R>& a, Uni& u, int f, int x, int y, size_t base, size_t ls, int t,
                                 C (&v)[1][8], C* sm, const C* tw, SI si, PAcc<R>*) {
    fft_line<C, L, false, 1>(v, sm, 0, tw, t, si);
    const R kx = wavenum<R>(x, a.nx, a.dkx), ky = wavenum<R>(y, a.ny, a.dky);
    const R kxy2 = kx * kx + ky * ky;
    const R sh = f == 0 ? u.shift[0] : u.shift[1];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const R kz = wavenum<R>(Plan<L>::exit_pos(false, t, e), a.nz, a.dkz);
      v[0][e] = cscale(v[0][e], a.invN / (sh + R(0.5) * (kxy2 + kz * kz)));
    }
    col_after<L>(sm, si);
    fft_line<C, L, true, 1>(v, sm, 0, tw, t, si);
#pragma unroll
    for (int e = 0; e < 8; ++e) a.W[base + (size_t)Plan<L>::exit_pos(true, t, e) * ls] = v[0][e];
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct XInvPC {
  using R = R_;
  using C = C2<R>;
  static constexpr int MAXT = 128;  // heavy epilogue: smaller blocks, more of them per SM
  static constexpr int MINB = sizeof(R_) == 4 ? EGPE_PC_MINB : 1;
  static constexpr const char* NAME = "x-inv precond sums";
  static double alg_bytes(const KArgs<R>& a) { return 12.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 2, NS = PC_NS;
  static constexpr bool INV = true, USES_LHY = false;
  using Uni = PcUni<R>;
  static __device__ void uniform(const KArgs<R>& a, Uni& u) { pc_uniform(a, u); }
  static __device__ void load(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[2][8], PAcc<R>*) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = (size_t)row * a.nx + Plan<L>::entry_pos(true, t, e);
      v[0][e] = valid ? a.W[idx] : cmk<C>(0, 0);
      v[1][e] = valid ? a.W[(size_t)a.N + idx] : cmk<C>(0, 0);
    }
  }
  static __device__ void store(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[2][8], PAcc<R>* acc,
                               const LhyNode<R>*) {
    if (!valid) return;
    const int yy = row % a.ny, zz = row / a.ny;
    const R Yc = -a.Ly + (R)yy * a.hy, Zc = -a.Lz + (R)zz * a.hz;
    const R vyz = a.vy * Yc * Yc + a.vz * Zc * Zc;
    R s[PC_NS];
#pragma unroll
    for (int k = 0; k < PC_NS; ++k) s[k] = 0;
    constexpr int CH = ChunkW<R>::v;
#pragma unroll
    for (int e0 = 0; e0 < 8; e0 += CH) {
      PcSumIn<R> in[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) pc_sum_load<R>(a, u, (size_t)row * a.nx + Plan<L>::exit_pos(true, t, e0 + j), in[j]);
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int e = e0 + j;
        const int x = Plan<L>::exit_pos(true, t, e);
        const size_t idx = (size_t)row * a.nx + x;
        C z1 = v[0][e], z2 = v[1][e];
        if (a.blend) {  // z = (1 - w) P_Delta^{-1} r + w P_V^{-1} r
          const C ml = a.ax[u.cur][(size_t)a.N + idx];
          const R X = -a.Lx + (R)x * a.hx;
          const R V = a.vx * X * X + vyz;
          const R n1 = cabs2(in[j].p1), n2 = cabs2(in[j].p2);
          R P1 = u.shift[0] + V + a.g11 * n1 + a.g12 * n2 + ml.x;
          R P2 = u.shift[1] + V + a.g21 * n1 + a.g22 * n2 + ml.y;
          P1 = P1 > u.floor_[0] ? P1 : u.floor_[0];
          P2 = P2 > u.floor_[1] ? P2 : u.floor_[1];
          const R wd = R(1) - u.wv, w1 = u.wv / P1, w2 = u.wv / P2;
          z1 = cmk<C>(wd * z1.x + w1 * in[j].r1.x, wd * z1.y + w1 * in[j].r1.y);
          z2 = cmk<C>(wd * z2.x + w2 * in[j].r2.x, wd * z2.y + w2 * in[j].r2.y);
        }
        a.z[idx] = z1;
        a.z[(size_t)a.N + idx] = z2;
        pc_sum_add<R>(in[j], z1, z2, s);
      }
    }
#pragma unroll
    for (int k = 0; k < PC_NS; ++k) acc[k].add(s[k]);
  }
  static __device__ double* out(const KArgs<R>& a, Uni&) { return a.st->pc; }
  static __device__ void finish(const KArgs<R>& a, Uni&) {
    if (a.ctrl) {
      a.st->ffts += 4;
      ctrl_after_pc(a.st);
    }
  }
};

// Pointwise preconditioner (modes none and diagonal): one pass, no transform.
template <class R>
__device__ __forceinline__ void pc_point_body(const KArgs<R>& a) {
  using C = C2<R>;
  if (!gate_open(a)) return;
  __shared__ RedSmem<PC_NS> red;
  PcUni<R> u;
  pc_uniform(a, u);
  PAcc<R> acc[PC_NS];
  const size_t N = a.N;
  const size_t nxy = (size_t)a.nx * a.ny;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % a.nx);
    const int y = (int)((idx / a.nx) % a.ny);
    const int z = (int)(idx / nxy);
    const R X = -a.Lx + (R)x * a.hx, Y = -a.Ly + (R)y * a.hy, Z = -a.Lz + (R)z * a.hz;
    const R V = a.vx * X * X + a.vy * Y * Y + a.vz * Z * Z;
    C w1, w2;
    PcIn<R> in;
    pc_load<R>(a, u, idx, in);
    pc_apply<R>(a, u, idx, V, in, w1, w2);
    a.z[idx] = w1;
    a.z[N + idx] = w2;
    R s[PC_NS];
#pragma unroll
    for (int k = 0; k < PC_NS; ++k) s[k] = 0;
    PcSumIn<R> si;
    pc_sum_load<R>(a, u, idx, si);
    pc_sum_add<R>(si, w1, w2, s);
#pragma unroll
    for (int k = 0; k < PC_NS; ++k) acc[k].add(s[k]);
  }
  if (reduce_blocks<PC_NS>(acc, a.partials, a.counter, a.st->pc, red)) {
    if (threadIdx.x == 0 && a.ctrl) ctrl_after_pc(a.st);
  }
}
template <class R> __global__ void __launch_bounds__(256) pc_point_kernel(KArgs<R> a) { pc_point_body(a); }
template <class R> __global__ void __launch_bounds__(256) pc_point_kernel_b(const __grid_constant__ KBatch<R> kb) {
  pc_point_body(kb.k[blockIdx.y]);
}


// ----------------------------------------------------------------------------
// Line-search pipeline (Sec. V): p = -z + beta p_prev - c psi (projected
// direction), forward transforms of p (Parseval <p|T|p>), the packed dipolar
// transform of rho = Re(psi conj p), and the pointwise second-variation sums.
// ----------------------------------------------------------------------------
template <class R> struct LcUni {
  int cur, nsel, pgiven, fallback;
  R beta, c[2];
};
template <class R> __device__ __forceinline__ void lc_uniform(const KArgs<R>& a, LcUni<R>& u) {
  u.cur = __ldcg(&a.st->cur);
  u.nsel = __ldcg(&a.st->n) & 1;
  u.pgiven = a.flag;
  u.fallback = __ldcg(&a.st->fallback);
  R c[3];
  load_uniforms<R, 3>({&a.st->beta, &a.st->c[0], &a.st->c[1]}, c);
  u.beta = c[0];
  u.c[0] = c[1];
  u.c[1] = c[2];
}

template <class R_, int L_> struct XFwdLC {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "x-fwd line dir";
  static double alg_bytes(const KArgs<R>& a) { return 11.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 3, NS = 0;
  static constexpr bool INV = false, USES_LHY = false;
  using Uni = LcUni<R>;
  static __device__ void uniform(const KArgs<R>& a, Uni& u) { lc_uniform(a, u); }
  static __device__ void load(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[3][8], PAcc<R>*) {
    const size_t N = a.N;
    const C* ps = a.psi[u.cur];
    C* pd = a.pb[u.nsel];
    const C* pp = a.pb[u.nsel ^ 1];
    const C* wsrc = u.fallback ? a.rb[u.nsel] : a.z;
    const bool usepp = !u.pgiven && u.beta != R(0);
    constexpr int CH = ChunkW<R>::v;
#pragma unroll
    for (int e0 = 0; e0 < 8; e0 += CH) {
      C p1[CH], p2[CH], w1[CH], w2[CH], d1[CH], d2[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const size_t idx = (size_t)row * a.nx + Plan<L>::entry_pos(false, t, e0 + j);
        const size_t id = valid ? idx : 0;
        p1[j] = ps[id];
        p2[j] = ps[N + id];
        w1[j] = u.pgiven ? pd[id] : wsrc[id];
        w2[j] = u.pgiven ? pd[N + id] : wsrc[N + id];
        if (usepp) {
          d1[j] = pp[id];
          d2[j] = pp[N + id];
        }
      }
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int e = e0 + j;
        C q1 = cmk<C>(0, 0), q2 = cmk<C>(0, 0);
        R rho1 = 0, rho2 = 0;
        if (valid) {
          if (u.pgiven) {
            q1 = w1[j];
            q2 = w2[j];
          } else {
            q1 = cmk<C>(-w1[j].x - u.c[0] * p1[j].x, -w1[j].y - u.c[0] * p1[j].y);
            q2 = cmk<C>(-w2[j].x - u.c[1] * p2[j].x, -w2[j].y - u.c[1] * p2[j].y);
            if (usepp) {
              q1 = cmk<C>(q1.x + u.beta * d1[j].x, q1.y + u.beta * d1[j].y);
              q2 = cmk<C>(q2.x + u.beta * d2[j].x, q2.y + u.beta * d2[j].y);
            }
            const size_t idx = (size_t)row * a.nx + Plan<L>::entry_pos(false, t, e);
            pd[idx] = q1;
            pd[N + idx] = q2;
          }
          rho1 = cdot(p1[j], q1);
          rho2 = cdot(p2[j], q2);
        }
        v[0][e] = q1;
        v[1][e] = q2;
        v[2][e] = cmk<C>(a.d11 * rho1 + a.d12 * rho2, a.d21 * rho1 + a.d22 * rho2);
      }
    }
  }
  static __device__ void store(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[3][8], PAcc<R>*,
                               const LhyNode<R>*) {
    if (!valid) return;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = (size_t)row * a.nx + Plan<L>::exit_pos(false, t, e);
#pragma unroll
      for (int f = 0; f < 3; ++f) a.W[(size_t)f * a.N + idx] = v[f][e];
    }
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct ZLc {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "z line coeffs";
  static double alg_bytes(const KArgs<R>& a) { return 4.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NS = 2, AXIS = 2;
  using Uni = NoUni;
  static __device__ void uniform(const KArgs<R>&, Uni&) {}
  static constexpr bool FIRST_INV = false;
  static __device__ const C* src(const KArgs<R>& a) { return a.W; }
  template <class SI>
  static __device__ void process(const KArgs<R>& a, Uni&, int f, int x, int y, size_t base, size_t ls, int t,
                                 C (&v)[1][8], C* sm, const C* tw, SI si, PAcc<R>* acc) {
    fft_line<C, L, false, 1>(v, sm, 0, tw, t, si);
    const R kx = wavenum<R>(x, a.nx, a.dkx), ky = wavenum<R>(y, a.ny, a.dky);
    const R kxy2 = kx * kx + ky * ky;
    if (f < 2) {  // <p_f | T | p_f> by Parseval: forward transform only
      R tk = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const R kz = wavenum<R>(Plan<L>::exit_pos(false, t, e), a.nz, a.dkz);
        tk += R(0.5) * (kxy2 + kz * kz) * cabs2(v[0][e]);
      }
      acc[f].add(tk);
      return;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const R kz = wavenum<R>(Plan<L>::exit_pos(false, t, e), a.nz, a.dkz);
      const R k2 = kxy2 + kz * kz;
      const R mult = (k2 > R(0)) ? (R(3) * kz * kz / k2 - R(1)) * a.invN : R(0);
      v[0][e] = cscale(v[0][e], mult);
    }
    col_after<L>(sm, si);
    fft_line<C, L, true, 1>(v, sm, 0, tw, t, si);
#pragma unroll
    for (int e = 0; e < 8; ++e) a.W[base + (size_t)Plan<L>::exit_pos(true, t, e) * ls] = v[0][e];
  }
  static __device__ double* out(const KArgs<R>& a, Uni&) { return a.st->lcz; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct XInvLC {
  using R = R_;
  using C = C2<R>;
  static constexpr int MINB = sizeof(R_) == 4 ? EGPE_LC_MINB : 1;
  static constexpr const char* NAME = "x-inv line sums+LHY";
  static double alg_bytes(const KArgs<R>& a) { return 9.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 1, NS = LC_NS;
  static constexpr bool INV = true, USES_LHY = true, LHY_TAB = true;
  using Uni = LcUni<R>;
  static __device__ void uniform(const KArgs<R>& a, Uni& u) { lc_uniform(a, u); }
  static __device__ void load(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[1][8], PAcc<R>*) {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      v[0][e] = valid ? a.W[(size_t)2 * a.N + (size_t)row * a.nx + Plan<L>::entry_pos(true, t, e)] : cmk<C>(0, 0);
  }
  static constexpr int NP = LhyNP<R>::v;
  static __device__ void store(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[1][8], PAcc<R>* acc,
                               const LhyNode<R>* nodes) {
    if (!valid) return;
    const size_t N = a.N;
    const C* ps = a.psi[u.cur];
    const C* pd = a.pb[u.nsel];
    const C* hp = a.hp[u.cur];
    const C* ax = a.ax[u.cur];
    const int y = row % a.ny, z = row / a.ny;
    const R Y = -a.Ly + (R)y * a.hy, Z = -a.Lz + (R)z * a.hz;
    const R vyz = a.vy * Y * Y + a.vz * Z * Z;
    const LhyCoef<R> cf = lhy_coef(a);
    R s[LC_NS];
#pragma unroll
    for (int k = 0; k < LC_NS; ++k) s[k] = 0;
#pragma unroll
    for (int e0 = 0; e0 < 8; e0 += NP) {
      R n1[NP], n2[NP], n1p[NP], n2p[NP], Hh[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const int e = e0 + j;
        const int x = Plan<L>::exit_pos(true, t, e);
        const size_t idx = (size_t)row * a.nx + x;
        const C p1 = ps[idx], p2 = ps[N + idx];
        const C q1 = pd[idx], q2 = pd[N + idx];
        const C h1 = hp[idx], h2 = hp[N + idx];
        const C phi = ax[idx], ml = ax[N + idx];
        n1[j] = cabs2(p1);
        n2[j] = cabs2(p2);
        const R a1 = cabs2(q1), a2 = cabs2(q2);
        const R rho1 = cdot(p1, q1), rho2 = cdot(p2, q2);
        n1p[j] = R(2) * rho1;
        n2p[j] = R(2) * rho2;
        const R X = -a.Lx + (R)x * a.hx;
        const R V = a.vx * X * X + vyz;
        const R U1 = V + a.g11 * n1[j] + a.g12 * n2[j] + phi.x + ml.x;
        const R U2 = V + a.g21 * n1[j] + a.g22 * n2[j] + phi.y + ml.y;
        s[LC_P1] += a1;
        s[LC_P2] += a2;
        s[LC_PSIP1] += rho1;
        s[LC_PSIP2] += rho2;
        s[LC_PH1] += cdot(q1, h1);
        s[LC_PH2] += cdot(q2, h2);
        s[LC_UPP1] += U1 * a1;
        s[LC_UPP2] += U2 * a2;
        s[LC_SRHO] += rho1 * (a.g11 * rho1 + a.g12 * rho2 + v[0][e].x) + rho2 * (a.g21 * rho1 + a.g22 * rho2 + v[0][e].y);
      }
      lhy_second<R, NP>(a, nodes, cf, n1, n2, n1p, n2p, Hh);
#pragma unroll
      for (int j = 0; j < NP; ++j) s[LC_HLHY] += Hh[j];
    }
#pragma unroll
    for (int k = 0; k < LC_NS; ++k) acc[k].add(s[k]);
  }
  static __device__ double* out(const KArgs<R>& a, Uni&) { return a.st->lc; }
  static __device__ void finish(const KArgs<R>& a, Uni&) {
    if (a.ctrl) {
      a.st->ffts += 4;
      ctrl_after_lc(a.st);
    }
  }
};

// ----------------------------------------------------------------------------
// Imaginary-time evolution, the paper's baseline (Sec. I, Sec. VI.B): Strang
// steps psi <- e^{-dtau T/2} e^{-dtau U[psi_half]} e^{-dtau T/2} psi with per-
// component renormalisation.  A kinetic half step is an FFT pair with the
// separable multiplier e^{-dtau |k|^2/4} = ex(kx) ey(ky) ez(kz); the potential
// step is fused into the prologue of the second half step, with U_i = V +
// sum_j g_ij n_j + Phi_i + mu_LHY^(i) read from the aux fields that the
// energy/gradient pipeline wrote for the half-stepped state.
// ----------------------------------------------------------------------------
template <class R_, int L_> struct XFwdKin {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "x-fwd ITE half step";
  static double alg_bytes(const KArgs<R>& a) { return (a.flag ? 6.0 : 4.0) * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 2, NS = 0;
  static constexpr bool INV = false, USES_LHY = false;
  struct Uni {
    int cur;
    R dtau;
  };
  static __device__ void uniform(const KArgs<R>& a, Uni& u) {
    u.cur = __ldcg(&a.st->cur);
    u.dtau = a.kin_tab[a.nx + a.ny + a.nz];
  }
  static __device__ void load(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[2][8], PAcc<R>*) {
    const C* ps = a.psi[u.cur];
    const C* ax = a.ax[u.cur];
    const size_t N = a.N;
    const int y = row % a.ny, z = row / a.ny;
    const R Y = -a.Ly + (R)y * a.hy, Z = -a.Lz + (R)z * a.hz;
    const R vyz = a.vy * Y * Y + a.vz * Z * Z;
    constexpr int CH = ChunkW<R>::v;
#pragma unroll
    for (int e0 = 0; e0 < 8; e0 += CH) {
      C p1[CH], p2[CH], f0[CH], f1[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const size_t idx = (size_t)row * a.nx + Plan<L>::entry_pos(false, t, e0 + j);
        const size_t id = valid ? idx : 0;
        p1[j] = ps[id];
        p2[j] = ps[N + id];
        if (a.flag) {
          f0[j] = ax[id];
          f1[j] = ax[N + id];
        }
      }
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int e = e0 + j;
        C q1 = valid ? p1[j] : cmk<C>(0, 0), q2 = valid ? p2[j] : cmk<C>(0, 0);
        if (a.flag && valid) {
          const int x = Plan<L>::entry_pos(false, t, e);
          const R X = -a.Lx + (R)x * a.hx;
          const R V = a.vx * X * X + vyz;
          const R n1 = cabs2(q1), n2 = cabs2(q2);
          const R U1 = V + a.g11 * n1 + a.g12 * n2 + f0[j].x + f1[j].x;
          const R U2 = V + a.g21 * n1 + a.g22 * n2 + f0[j].y + f1[j].y;
          q1 = cscale(q1, exp(-u.dtau * U1));
          q2 = cscale(q2, exp(-u.dtau * U2));
        }
        v[0][e] = q1;
        v[1][e] = q2;
      }
    }
  }
  static __device__ void store(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[2][8], PAcc<R>*,
                               const LhyNode<R>*) {
    if (!valid) return;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = (size_t)row * a.nx + Plan<L>::exit_pos(false, t, e);
      a.W[idx] = v[0][e];
      a.W[(size_t)a.N + idx] = v[1][e];
    }
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct ZKin {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "z fused ITE half step";
  static double alg_bytes(const KArgs<R>& a) { return 4.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NS = 0, AXIS = 2;
  using Uni = NoUni;
  static __device__ void uniform(const KArgs<R>&, Uni&) {}
  static constexpr bool FIRST_INV = false;
  static __device__ const C* src(const KArgs<R>& a) { return a.W; }
  template <class SI>
  static __device__ void process(const KArgs<R>& a, Uni&, int, int x, int y, size_t base, size_t ls, int t,
                                 C (&v)[1][8], C* sm, const C* tw, SI si, PAcc<R>*) {
    fft_line<C, L, false, 1>(v, sm, 0, tw, t, si);
    const R exy = a.kin_tab[x] * a.kin_tab[a.nx + y] * a.invN;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int kz = Plan<L>::exit_pos(false, t, e);
      v[0][e] = cscale(v[0][e], exy * a.kin_tab[a.nx + a.ny + kz]);
    }
    col_after<L>(sm, si);
    fft_line<C, L, true, 1>(v, sm, 0, tw, t, si);
#pragma unroll
    for (int e = 0; e < 8; ++e) a.W[base + (size_t)Plan<L>::exit_pos(true, t, e) * ls] = v[0][e];
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct XInvKin {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "x-inv ITE half step";
  static double alg_bytes(const KArgs<R>& a) { return 4.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 2, NS = 2;
  static constexpr bool INV = true, USES_LHY = false;
  struct Uni {
    int cur;
  };
  static __device__ void uniform(const KArgs<R>& a, Uni& u) { u.cur = __ldcg(&a.st->cur); }
  static __device__ void load(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[2][8], PAcc<R>*) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = (size_t)row * a.nx + Plan<L>::entry_pos(true, t, e);
      v[0][e] = valid ? a.W[idx] : cmk<C>(0, 0);
      v[1][e] = valid ? a.W[(size_t)a.N + idx] : cmk<C>(0, 0);
    }
  }
  static __device__ void store(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[2][8], PAcc<R>* acc,
                               const LhyNode<R>*) {
    if (!valid) return;
    C* ps = a.psi[u.cur];
    R s0 = 0, s1 = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = (size_t)row * a.nx + Plan<L>::exit_pos(true, t, e);
      ps[idx] = v[0][e];
      ps[(size_t)a.N + idx] = v[1][e];
      s0 += cabs2(v[0][e]);
      s1 += cabs2(v[1][e]);
    }
    acc[0].add(s0);
    acc[1].add(s1);
  }
  static __device__ double* out(const KArgs<R>& a, Uni&) { return a.st->rt; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

// psi_i <- psi_i / ||psi_i|| with the norms the last half step reduced.
template <class R> __device__ __forceinline__ void ite_scale_body(const KArgs<R>& a) {
  if (!gate_open(a)) return;
  const int cur = __ldcg(&a.st->cur);
  const double dV = __ldcg(&a.st->dV);
  R s1, s2;
  if constexpr (sizeof(R) == sizeof(double)) {
    s1 = 1.0 / sqrt(__ldcg(&a.st->rt[0]) * dV);
    s2 = 1.0 / sqrt(__ldcg(&a.st->rt[1]) * dV);
  } else {  // FP32 fields: lane i forms ||psi_i||^2 in FP64, one conversion per warp
    const float q = (float)(__ldcg(&a.st->rt[threadIdx.x & 1]) * dV);
    const float sc = rsqrtf(q);
    s1 = __shfl_sync(0xffffffffu, sc, 0);
    s2 = __shfl_sync(0xffffffffu, sc, 1);
  }
  C2<R>* ps = a.psi[cur];
  const size_t N = a.N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (size_t)gridDim.x * blockDim.x) {
    ps[idx] = cscale(ps[idx], s1);
    ps[N + idx] = cscale(ps[N + idx], s2);
  }
}
template <class R> __global__ void __launch_bounds__(256) ite_scale_kernel(KArgs<R> a) { ite_scale_body(a); }
template <class R> __global__ void __launch_bounds__(256) ite_scale_kernel_b(const __grid_constant__ KBatch<R> kb) {
  ite_scale_body(kb.k[blockIdx.y]);
}


// ----------------------------------------------------------------------------
// Parameter derivatives at fixed psi (the adjoint pass of the energy with
// respect to its couplings, Eq. 1): x fwd of zeta = n1 + i n2 -> y -> z with the
// dipolar kernel K(k) -> y inv -> x inv: K*n1 = Re, K*n2 = Im (the kernel is real
// and even), then the contact, dipolar, trap and LHY (through eta) sums.
// ----------------------------------------------------------------------------
template <class R_, int L_> struct XFwdPG {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "x-fwd densities (param grad)";
  static double alg_bytes(const KArgs<R>& a) { return 3.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 1, NS = 0;
  static constexpr bool INV = false, USES_LHY = false;
  struct Uni {
    int cur;
  };
  static __device__ void uniform(const KArgs<R>& a, Uni& u) { u.cur = __ldcg(&a.st->cur); }
  static __device__ void load(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[1][8], PAcc<R>*) {
    const C* ps = a.psi[u.cur];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const size_t idx = valid ? (size_t)row * a.nx + Plan<L>::entry_pos(false, t, e) : 0;
      const C p1 = ps[idx], p2 = ps[(size_t)a.N + idx];
      v[0][e] = valid ? cmk<C>(cabs2(p1), cabs2(p2)) : cmk<C>(0, 0);
    }
  }
  static __device__ void store(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[1][8], PAcc<R>*,
                               const LhyNode<R>*) {
    if (!valid) return;
#pragma unroll
    for (int e = 0; e < 8; ++e) a.W[(size_t)row * a.nx + Plan<L>::exit_pos(false, t, e)] = v[0][e];
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct ZPg {
  using R = R_;
  using C = C2<R>;
  static constexpr const char* NAME = "z dipolar kernel (param grad)";
  static double alg_bytes(const KArgs<R>& a) { return 2.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NS = 0, AXIS = 2;
  using Uni = NoUni;
  static __device__ void uniform(const KArgs<R>&, Uni&) {}
  static constexpr bool FIRST_INV = false;
  static __device__ const C* src(const KArgs<R>& a) { return a.W; }
  template <class SI>
  static __device__ void process(const KArgs<R>& a, Uni&, int, int x, int y, size_t base, size_t ls, int t,
                                 C (&v)[1][8], C* sm, const C* tw, SI si, PAcc<R>*) {
    fft_line<C, L, false, 1>(v, sm, 0, tw, t, si);
    const R kx = wavenum<R>(x, a.nx, a.dkx), ky = wavenum<R>(y, a.ny, a.dky);
    const R kxy2 = kx * kx + ky * ky;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const R kz = wavenum<R>(Plan<L>::exit_pos(false, t, e), a.nz, a.dkz);
      const R k2 = kxy2 + kz * kz;
      v[0][e] = cscale(v[0][e], (k2 > R(0)) ? (R(3) * kz * kz / k2 - R(1)) * a.invN : R(0));
    }
    col_after<L>(sm, si);
    fft_line<C, L, true, 1>(v, sm, 0, tw, t, si);
#pragma unroll
    for (int e = 0; e < 8; ++e) a.W[base + (size_t)Plan<L>::exit_pos(true, t, e) * ls] = v[0][e];
  }
  static __device__ double* out(const KArgs<R>&, Uni&) { return nullptr; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

template <class R_, int L_> struct XInvPG {
  using R = R_;
  using C = C2<R>;
  static constexpr int MAXT = 128;
  static constexpr const char* NAME = "x-inv parameter sums";
  static double alg_bytes(const KArgs<R>& a) { return 3.0 * a.N * sizeof(C); }
  static constexpr int L = L_, NF = 1, NS = PG_NS;
  static constexpr bool INV = true, USES_LHY = true;
  struct Uni {
    int cur;
  };
  static __device__ void uniform(const KArgs<R>& a, Uni& u) { u.cur = __ldcg(&a.st->cur); }
  static __device__ void load(const KArgs<R>& a, Uni&, int row, bool valid, int t, C (&v)[1][8], PAcc<R>*) {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      v[0][e] = valid ? a.W[(size_t)row * a.nx + Plan<L>::entry_pos(true, t, e)] : cmk<C>(0, 0);
  }
  static __device__ void store(const KArgs<R>& a, Uni& u, int row, bool valid, int t, C (&v)[1][8], PAcc<R>* acc,
                               const LhyNode<R>* nodes) {
    if (!valid) return;
    const C* ps = a.psi[u.cur];
    const int y = row % a.ny, z = row / a.ny;
    const R Y = -a.Ly + (R)y * a.hy, Z = -a.Lz + (R)z * a.hz;
    const LhyCoef<R> cf = lhy_coef(a);
    R s[PG_NS];
#pragma unroll
    for (int k = 0; k < PG_NS; ++k) s[k] = R(0);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int x = Plan<L>::exit_pos(true, t, e);
      const size_t idx = (size_t)row * a.nx + x;
      const R n1 = cabs2(ps[idx]), n2 = cabs2(ps[(size_t)a.N + idx]);
      const R X = -a.Lx + (R)x * a.hx;
      const R nt = n1 + n2;
      R lh[7];
      lhy_eta_sums<R>(nodes, a.Q, cf, n1, n2, lh);
      s[PG_N11] += n1 * n1;
      s[PG_N12] += n1 * n2;
      s[PG_N22] += n2 * n2;
      s[PG_K11] += n1 * v[0][e].x;
      s[PG_K12] += n1 * v[0][e].y;
      s[PG_K22] += n2 * v[0][e].y;
      s[PG_X2] += X * X * nt;
      s[PG_Y2] += Y * Y * nt;
      s[PG_Z2] += Z * Z * nt;
      s[PG_F] += lh[0];
      s[PG_L11] += lh[1];
      s[PG_L22] += lh[2];
      s[PG_L12] += lh[3];
      s[PG_M11] += lh[4];
      s[PG_M22] += lh[5];
      s[PG_M12] += lh[6];
    }
#pragma unroll
    for (int k = 0; k < PG_NS; ++k) acc[k].add(s[k]);
  }
  static __device__ double* out(const KArgs<R>& a, Uni&) { return a.st->pg; }
  static __device__ void finish(const KArgs<R>&, Uni&) {}
};

// ----------------------------------------------------------------------------
// Small pointwise kernels: retraction sums and apply, residual norm, casts.
// ----------------------------------------------------------------------------
// sums over (psi = gin, p = gout-as-input) for the standalone retraction
template <class R> __global__ void __launch_bounds__(256) rt_sums_kernel(KArgs<R> a, const C2<R>* psi, const C2<R>* p) {
  __shared__ RedSmem<RT_NS> red;
  PAcc<R> acc[RT_NS];
  const size_t N = a.N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (size_t)gridDim.x * blockDim.x) {
    for (int i = 0; i < 2; ++i) {
      const C2<R> u = psi[i * N + idx], q = p[i * N + idx];
      acc[RT_P1 + i].add(cabs2(q));
      acc[RT_PSIP1 + i].add(cdot(u, q));
      acc[RT_PSI1 + i].add(cabs2(u));
    }
  }
  reduce_blocks<RT_NS>(acc, a.partials, a.counter, a.st->rt, red);
}

template <class R>
__global__ void __launch_bounds__(256) rt_apply_kernel(size_t N, const C2<R>* psi, const C2<R>* p, C2<R>* out, R a1,
                                                        R b1, R a2, R b2) {
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (size_t)gridDim.x * blockDim.x) {
    const C2<R> u1 = psi[idx], q1 = p[idx], u2 = psi[N + idx], q2 = p[N + idx];
    out[idx] = cmk<C2<R>>(a1 * u1.x + b1 * q1.x, a1 * u1.y + b1 * q1.y);
    out[N + idx] = cmk<C2<R>>(a2 * u2.x + b2 * q2.x, a2 * u2.y + b2 * q2.y);
  }
}

// ||r_i||^2 of the current point (final report of a solve).
template <class R> __global__ void __launch_bounds__(256) resnorm_kernel(KArgs<R> a) {
  __shared__ RedSmem<2> red;
  PAcc<R> acc[2];
  const int cur = __ldcg(&a.st->cur);
  R mu[2];
  load_uniforms<R, 2>({&a.st->mu[0], &a.st->mu[1]}, mu);
  const size_t N = a.N;
  const C2<R>* ps = a.psi[cur];
  const C2<R>* hp = a.hp[cur];
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (size_t)gridDim.x * blockDim.x) {
    for (int i = 0; i < 2; ++i) {
      const C2<R> u = ps[i * N + idx], h = hp[i * N + idx];
      const C2<R> r = cmk<C2<R>>(h.x - mu[i] * u.x, h.y - mu[i] * u.y);
      acc[i].add(cabs2(r));
    }
  }
  reduce_blocks<2>(acc, a.partials, a.counter, a.st->pca, red);
}

template <class A, class B> __global__ void cast_kernel(size_t n, const A* in, B* out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const A v = in[i];
    B w;
    w.x = (decltype(w.x))v.x;
    w.y = (decltype(w.y))v.y;
    out[i] = w;
  }
}

}  // namespace egpe
