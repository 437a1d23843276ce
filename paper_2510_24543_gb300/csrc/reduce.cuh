// Deterministic reductions: per-thread sums -> warp shuffle tree ->
// per-block partials -> the last block to finish sums the partials in a fixed
// order.  No floating-point atomics, so every run gives the same bits; the
// only atomic is an integer arrival counter (no waiting on it).
//
// FP64 fields reduce in FP64.  FP32 fields reduce in float-float (hi + lo)
// arithmetic on the FP32 pipe: GB300's FP64 pipe issues a warp instruction
// only every few dozen cycles per SM partition, so an FP64 shuffle tree of a
// dozen sums per warp costs as much pipe time as the points the warp handled.
// Float-float keeps about 44 bits, far below the FP32 fields' own rounding.
#pragma once
#include "common.cuh"

namespace egpe {

// Float-float value h + l.
struct FF {
  float h, l;
};
// Knuth's two-sum of the high parts (its error term is exact, so the result
// does not depend on the operand order), then the low parts, renormalised with
// Dekker's fast two-sum.  Plain additions only: nothing to contract into FMAs.
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.h + b.h, bp = s - a.h;
  const float e = (a.h - (s - bp)) + (b.h - bp);
  const float t = (a.l + b.l) + e;
  const float h = s + t;
  return FF{h, t - (h - s)};
}

// Per-thread partial sum.  FP64 fields accumulate in FP64; FP32 fields
// accumulate in FP32 with Kahan compensation, which keeps the per-thread
// partial as accurate as an FP64 accumulation of the same terms.
template <class R> struct PAcc {
  using Red = double;
  R v = R(0);
  __device__ __forceinline__ void add(R x) { v += x; }
  __device__ __forceinline__ double red() const { return (double)v; }
};
template <> struct PAcc<float> {
  using Red = FF;
  float hi = 0.f, lo = 0.f;  // sum = hi - lo
  __device__ __forceinline__ void add(float x) {
    const float y = x - lo;
    const float t = hi + y;
    lo = (t - hi) - y;
    hi = t;
  }
  __device__ __forceinline__ FF red() const { return FF{hi, -lo}; }
};

// The reduction's arithmetic on FP64 values and on float-float pairs.
template <class T> struct RedT;
template <> struct RedT<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double shfl(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
  static __device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
  static __device__ __forceinline__ double value(double v) { return v; }
};
template <> struct RedT<FF> {
  static __device__ __forceinline__ FF zero() { return FF{0.f, 0.f}; }
  static __device__ __forceinline__ FF add(FF a, FF b) { return ff_add(a, b); }
  static __device__ __forceinline__ FF shfl(FF v, int off) {
    return FF{__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
  }
  static __device__ __forceinline__ FF ldcg(const FF* p) {
    const float2 q = __ldcg(reinterpret_cast<const float2*>(p));
    return FF{q.x, q.y};
  }
  static __device__ __forceinline__ double value(FF v) { return (double)v.h + (double)v.l; }
};

__host__ __device__ constexpr int pow2_ceil(int n) { return n <= 1 ? 1 : 2 * pow2_ceil((n + 1) / 2); }
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// Warp reduce-scatter of P = 2^k sums: at each exchange distance the lane
// keeps half of the slots it still holds and sends the other half, so a lane
// adds P/2 + P/4 + ... + 1 values instead of P per level; once it holds one
// slot the remaining levels are a plain butterfly.  Afterwards lane j holds
// slot j >> (5 - k), complete over the warp.
template <class T, int OFF, int HELD, int P>
__device__ __forceinline__ void warp_reduce_scatter(T (&v)[P], int lane) {
  if constexpr (OFF > 0) {
    if constexpr (HELD > 1) {
      constexpr int H = HELD / 2;
      const bool up = (lane & OFF) != 0;
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const T keep = up ? v[k + H] : v[k];
        const T send = up ? v[k] : v[k + H];
        v[k] = RedT<T>::add(keep, RedT<T>::shfl(send, OFF));
      }
      warp_reduce_scatter<T, OFF / 2, H, P>(v, lane);
    } else {
      v[0] = RedT<T>::add(v[0], RedT<T>::shfl(v[0], OFF));
      warp_reduce_scatter<T, OFF / 2, 1, P>(v, lane);
    }
  }
}

// Shared scratch for NS values per warp (32 warps max); holds FP64 values or
// float-float pairs (both 8 bytes).
template <int NS> struct RedSmem {
  double w[32][NS];
  int last;
};
static_assert(sizeof(FF) == sizeof(double), "float-float slots share the FP64 scratch");

// Block-wide sum of v[0..NS) (v[NS..P) are zero); the result is valid in
// thread s for slot s (s < NS).  Warps are summed in warp order.
template <class T, int NS>
__device__ __forceinline__ T block_sum_to_thread(T (&v)[pow2_ceil(NS)], RedSmem<NS>& sm) {
  constexpr int P = pow2_ceil(NS), SH = 5 - ilog2(P);
  static_assert(P <= 32, "at most 32 slots");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  warp_reduce_scatter<T, 16, P, P>(v, lane);
  T* w = reinterpret_cast<T*>(&sm.w[0][0]);
  const int s = lane >> SH;
  if ((lane & ((1 << SH) - 1)) == 0 && s < NS) w[warp * NS + s] = v[0];
  __syncthreads();
  T r = RedT<T>::zero();
  if (threadIdx.x < NS) {
    r = w[threadIdx.x];
    for (int k = 1; k < nw; ++k) r = RedT<T>::add(r, w[k * NS + threadIdx.x]);
  }
  __syncthreads();
  return r;
}

// Writes this block's partial sums; the last block to arrive reduces all
// partials in block order and writes out[0..NS) in FP64.  Returns true in the
// last block (all its threads), after out[] is written and visible to the block.
template <int NS, class T>
__device__ __forceinline__ bool reduce_grid(T (&v)[pow2_ceil(NS)], double* __restrict__ partials, unsigned* counter,
                                            double* out, RedSmem<NS>& sm) {
  constexpr int P = pow2_ceil(NS);
  T* part = reinterpret_cast<T*>(partials);
  const T r = block_sum_to_thread<T, NS>(v, sm);
  if (threadIdx.x < NS) {
    part[(size_t)blockIdx.x * NS + threadIdx.x] = r;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    sm.last = (prev == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!sm.last) return false;
  __threadfence();
  T acc[P];
#pragma unroll
  for (int s = 0; s < P; ++s) acc[s] = RedT<T>::zero();
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = RedT<T>::add(acc[s], RedT<T>::ldcg(&part[(size_t)b * NS + s]));
  }
  const T tot = block_sum_to_thread<T, NS>(acc, sm);
  if (threadIdx.x < NS) out[threadIdx.x] = RedT<T>::value(tot);
  if (threadIdx.x == 0) *counter = 0u;
  __threadfence();
  __syncthreads();
  return true;
}

// Grid reduction of per-thread accumulators (FP64 or compensated FP32).
template <int NS, class R>
__device__ __forceinline__ bool reduce_blocks(const PAcc<R> (&acc)[NS], double* __restrict__ partials,
                                              unsigned* counter, double* out, RedSmem<NS>& sm) {
  using T = typename PAcc<R>::Red;
  T v[pow2_ceil(NS)];
#pragma unroll
  for (int s = 0; s < pow2_ceil(NS); ++s) v[s] = s < NS ? acc[s].red() : RedT<T>::zero();
  return reduce_grid<NS, T>(v, partials, counter, out, sm);
}

// Converts K FP64 scalars of the device state to R.  For FP32, lane k loads
// and converts scalar k and shuffles broadcast the results: one conversion
// instruction per warp instead of K on the narrow FP64 pipe.
template <class R, int K>
__device__ __forceinline__ void load_uniforms(const double* const (&src)[K], R (&dst)[K]) {
  static_assert(K <= 32, "one scalar per lane");
  if constexpr (sizeof(R) == sizeof(double)) {
#pragma unroll
    for (int k = 0; k < K; ++k) dst[k] = (R)__ldcg(src[k]);
  } else {
    const int lane = threadIdx.x & 31;
    const double* p = src[0];
#pragma unroll
    for (int k = 1; k < K; ++k) p = lane == k ? src[k] : p;
    const R mine = (R)__ldcg(p);
#pragma unroll
    for (int k = 0; k < K; ++k) dst[k] = __shfl_sync(0xffffffffu, mine, k);
  }
}

}  // namespace egpe
