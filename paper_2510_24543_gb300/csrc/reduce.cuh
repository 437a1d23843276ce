// Deterministic FP64 reductions: per-thread sums -> warp shuffle tree ->
// per-block partials -> the last block to finish sums the partials in a fixed
// order.  No floating-point atomics, so every run gives the same bits; the
// only atomic is an integer arrival counter (no waiting on it).
#pragma once
#include "common.cuh"

namespace egpe {

// Per-thread partial sum.  FP64 fields accumulate in FP64; FP32 fields
// accumulate in FP32 with Kahan compensation (GB300's FP64 pipe is narrow, so
// one conversion per thread instead of one FP64 add per tile), which keeps the
// per-thread partial as accurate as an FP64 accumulation of the same terms.
template <class R> struct PAcc {
  R v = R(0);
  __device__ __forceinline__ void add(R x) { v += x; }
  __device__ __forceinline__ double get() const { return (double)v; }
};
template <> struct PAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - lo;
    const float t = hi + y;
    lo = (t - hi) - y;
    hi = t;
  }
  __device__ __forceinline__ double get() const { return (double)hi - (double)lo; }
};

// Shared scratch for NS values per warp (32 warps max).
template <int NS> struct RedSmem {
  double w[32][NS];
  int last;
};

template <int NS> __device__ __forceinline__ void warp_sum(double (&a)[NS]) {
#pragma unroll
  for (int s = 0; s < NS; ++s) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a[s] += __shfl_down_sync(0xffffffffu, a[s], off);
  }
}

// Block-wide sum of a[NS]; the result is valid in thread s for value s (s < NS).
template <int NS> __device__ __forceinline__ double block_sum_to_thread(double (&a)[NS], RedSmem<NS>& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  warp_sum<NS>(a);
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) sm.w[warp][s] = a[s];
  }
  __syncthreads();
  double v = 0.0;
  if (threadIdx.x < NS) {
    for (int k = 0; k < nw; ++k) v += sm.w[k][threadIdx.x];
  }
  __syncthreads();
  return v;
}

// Writes this block's partial sums; the last block to arrive reduces all
// partials in block order and writes out[0..NS).  Returns true in the last
// block (all its threads), after out[] is written and visible to the block.
template <int NS>
__device__ __forceinline__ bool reduce_blocks(double (&a)[NS], double* __restrict__ partials,
                                              unsigned* counter, double* out, RedSmem<NS>& sm) {
  double v = block_sum_to_thread<NS>(a, sm);
  if (threadIdx.x < NS) {
    partials[(size_t)blockIdx.x * NS + threadIdx.x] = v;
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
  double acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] += __ldcg(&partials[(size_t)b * NS + s]);
  }
  double tot = block_sum_to_thread<NS>(acc, sm);
  if (threadIdx.x < NS) out[threadIdx.x] = tot;
  if (threadIdx.x == 0) *counter = 0u;
  __threadfence();
  __syncthreads();
  return true;
}

}  // namespace egpe
