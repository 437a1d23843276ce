// Batched Stockham (self-sorting) FFT of one line per group of L/8 threads.
//
// Each thread owns 8 complex values of its line.  A length-L transform is a
// sequence of radix passes (radix 8, then one radix-2 or radix-4 pass when
// log2 L is not a multiple of 3); the inverse plan runs the radices in reverse
// order so that the forward transform's last-pass register layout is exactly
// the inverse transform's first-pass layout.  That is what lets the z pass
// fuse forward FFT -> k-space multiply -> inverse FFT without touching shared
// memory at the turn.  Between passes values go through shared memory; the
// first-pass inputs and last-pass outputs stay in registers, so prologue and
// epilogue code reads and writes global memory directly in natural order.
//
// Pass p (radix r, Ns = product of earlier radices), butterfly j, element q:
//   input position  j + q L/r
//   twiddle         W_{Ns r}^{q (j mod Ns)}   (table entry q (j mod Ns) L/(Ns r))
//   output position (j div Ns) Ns r + (j mod Ns) + q Ns
// Thread t of a line owns butterflies j = t + b L/8 (b < 8/r).
//
// Lengths 48, 80 and 96 (a power of two times 3 or 5) use the same register
// interface with a mixed-radix plan (radix 8, then 3/5 and 2/4 passes in
// shared memory) and natural entry/exit layouts; see fft_mixed.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace egpe {

template <int L> struct IsPow2 {
  static constexpr bool v = L > 0 && (L & (L - 1)) == 0;
};

// Radix sequence of the mixed-radix lengths (a multiple of 8 times 3 or 5):
// radix 8 first, then the remaining factors.
template <int L> struct MixedPlan {
  static constexpr int TPL = L / 8;
  static constexpr int P = (L == 48) ? 3 : (L == 80) ? 3 : (L == 96) ? 3 : -1;
  static_assert(P > 0, "unsupported FFT length");
  __host__ __device__ static constexpr int rad(int p) {
    return p == 0 ? 8 : (L == 48 ? (p == 1 ? 3 : 2) : L == 80 ? (p == 1 ? 5 : 2) : (p == 1 ? 4 : 3));
  }
  __host__ __device__ static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * rad(p - 1); }
  // natural layout on entry and exit, in both directions
  __device__ static __forceinline__ int entry_pos(bool, int t, int e) { return t + e * TPL; }
  __device__ static __forceinline__ int exit_pos(bool, int t, int e) { return t + e * TPL; }
};

template <int L, bool POW2 = IsPow2<L>::v> struct Plan;
template <int L> struct Plan<L, false> : MixedPlan<L> {};

template <int L> struct Plan<L, true> {
  static constexpr int TPL = L / 8;
  static constexpr int LOG2 = (L == 8) ? 3 : (L == 16) ? 4 : (L == 32) ? 5 : (L == 64) ? 6
                            : (L == 128) ? 7 : (L == 256) ? 8 : -1;
  static_assert(LOG2 > 0, "unsupported FFT length");
  static constexpr int P = (LOG2 + 2) / 3;
  static constexpr int LAST = L >> (3 * (P - 1));  // radix of the forward plan's last pass
  __host__ __device__ static constexpr int rad(bool inv, int p) {
    return inv ? (p == 0 ? LAST : 8) : (p == P - 1 ? LAST : 8);
  }
  __host__ __device__ static constexpr int ns(bool inv, int p) {
    return p == 0 ? 1 : ns(inv, p - 1) * rad(inv, p - 1);
  }
  // position of register e of thread t on entry to / exit from the transform
  __device__ static __forceinline__ int entry_pos(bool inv, int t, int e) {
    const int r = rad(inv, 0);
    return t + (e / r) * TPL + (e % r) * (L / r);
  }
  __device__ static __forceinline__ int exit_pos(bool inv, int t, int e) {
    const int r = rad(inv, P - 1);
    return t + (e / r) * TPL + (e % r) * (L / r);
  }
};

template <int MC> struct ColIdxT;
template <class SI> struct IsColIdx {
  static constexpr bool v = false;
};
template <int MC> struct IsColIdx<ColIdxT<MC>> {
  static constexpr bool v = true;
};
// Synchronisation of one transform's exchange buffer.  A row line's L/8
// threads are consecutive and, for the power-of-two lengths (L/8 <= 32
// dividing 32), inside one warp with a buffer of their own: a warp barrier
// suffices.  Column lines spread over the block and need the block barrier.
template <class SI> __device__ __forceinline__ void line_sync() {
  if constexpr (IsColIdx<SI>::v) __syncthreads();
  else __syncwarp();
}
// Column lines (power-of-two lengths) exchange through two buffers in turn,
// so one block barrier per exchange suffices: a buffer is written again only
// after the barrier of the exchange that used the other one, which every
// thread reaches after its reads of the first.  Row lines reuse one buffer
// with two warp barriers per exchange.
template <class SI> struct PingPong {
  static constexpr bool v = IsColIdx<SI>::v;
};

template <class C> __device__ __forceinline__ C mul_i(C a) { return cmk<C>(-a.y, a.x); }
template <class C> __device__ __forceinline__ C mul_mi(C a) { return cmk<C>(a.y, -a.x); }

template <bool INV, class C> __device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV, class C> __device__ __forceinline__ void dft4v(C& a0, C& a1, C& a2, C& a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
  t3 = INV ? mul_i(t3) : mul_mi(t3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <bool INV, class C> __device__ __forceinline__ void dft4(C* v) { dft4v<INV>(v[0], v[1], v[2], v[3]); }

template <bool INV, class C> __device__ __forceinline__ void dft8(C* v) {
  using R = decltype(C::x);
  const R h = R(0.70710678118654752440084436210485);
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4v<INV>(e0, e1, e2, e3);
  dft4v<INV>(o0, o1, o2, o3);
  // odd outputs times W8^k (forward W8 = exp(-i pi/4); inverse its conjugate)
  if (INV) {
    o1 = cmk<C>((o1.x - o1.y) * h, (o1.x + o1.y) * h);
    o2 = mul_i(o2);
    o3 = cmk<C>((-o3.x - o3.y) * h, (o3.x - o3.y) * h);
  } else {
    o1 = cmk<C>((o1.x + o1.y) * h, (o1.y - o1.x) * h);
    o2 = mul_mi(o2);
    o3 = cmk<C>((o3.y - o3.x) * h, -(o3.x + o3.y) * h);
  }
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

// y_k = sum_q a_q W_3^{qk}: with c = cos(2 pi/3) = -1/2 and s = sin(2 pi/3),
// y_{1,2} = a0 + c (a1 + a2) -/+ i s (a1 - a2) (signs swapped for the inverse).
template <bool INV, class C> __device__ __forceinline__ void dft3(C* v) {
  using R = decltype(C::x);
  const R s = R(0.86602540378443864676372317075294);
  const C a0 = v[0], t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
  const C b = cmk<C>(a0.x - R(0.5) * t1.x, a0.y - R(0.5) * t1.y);
  const C d = cscale(INV ? mul_i(t2) : mul_mi(t2), s);
  v[0] = cadd(a0, t1);
  v[1] = cadd(b, d);
  v[2] = csub(b, d);
}

// Five-point DFT from the real and imaginary parts of W_5^k:
// c1 = cos(2 pi/5), c2 = cos(4 pi/5), s1 = sin(2 pi/5), s2 = sin(4 pi/5).
template <bool INV, class C> __device__ __forceinline__ void dft5(C* v) {
  using R = decltype(C::x);
  const R c1 = R(0.30901699437494742410229341718282), c2 = R(-0.80901699437494742410229341718282);
  const R s1 = R(0.95105651629515357211643933337938), s2 = R(0.58778525229247312916870595463907);
  const C a0 = v[0];
  const C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  const C b1 = cmk<C>(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
  const C b2 = cmk<C>(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
  const C e1 = cmk<C>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
  const C e2 = cmk<C>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
  const C d1 = INV ? mul_i(e1) : mul_mi(e1), d2 = INV ? mul_i(e2) : mul_mi(e2);
  v[0] = cadd(a0, cadd(t1, t2));
  v[1] = cadd(b1, d1);
  v[4] = csub(b1, d1);
  v[2] = cadd(b2, d2);
  v[3] = csub(b2, d2);
}

template <int R_, bool INV, class C> __device__ __forceinline__ void dft_r(C* v) {
  if constexpr (R_ == 8) dft8<INV>(v);
  else if constexpr (R_ == 5) dft5<INV>(v);
  else if constexpr (R_ == 4) dft4<INV>(v);
  else if constexpr (R_ == 3) dft3<INV>(v);
  else dft2<INV>(v);
}

// Runs passes p..P-1 of the (forward or inverse) plan on NF lines at once.
// v[f][8]: this thread's registers for field f; sm + f*fstride: the shared
// line buffer of field f for this thread's line; si(pos): offset of line
// position pos inside that buffer; tw: shared table W_L^m, m < L.
template <class C, int L, bool INV, int NF, int p, class SI>
__device__ __forceinline__ void fft_passes(C (&v)[NF][8], C* sm, int fstride, const C* __restrict__ tw,
                                           int t, const SI& si) {
  using PL = Plan<L>;
  constexpr int r = PL::rad(INV, p);
  constexpr int Ns = PL::ns(INV, p);
  constexpr int NB = 8 / r;
  constexpr int TPL = PL::TPL;
  constexpr int STW = L / (Ns * r);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = t + b * TPL;
    if constexpr (Ns > 1) {
      const int k = j % Ns;
#pragma unroll
      for (int q = 1; q < r; ++q) {
        const C w = tw[q * k * STW];
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f][b * r + q] = INV ? cmulc(v[f][b * r + q], w) : cmul(v[f][b * r + q], w);
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) dft_r<r, INV>(&v[f][b * r]);
  }
  if constexpr (p + 1 < PL::P) {
    // exchange p goes through the second buffer when p is even (column lines)
    C* xb = sm;
    if constexpr (PingPong<SI>::v) {
      if constexpr ((p & 1) == 0) xb = sm + si.alt;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + b * TPL;
      const int base = (j / Ns) * Ns * r + (j % Ns);
#pragma unroll
      for (int q = 0; q < r; ++q) {
        const int o = si(base + q * Ns);
#pragma unroll
        for (int f = 0; f < NF; ++f) xb[f * fstride + o] = v[f][b * r + q];
      }
    }
    line_sync<SI>();
    constexpr int r2 = PL::rad(INV, p + 1);
    constexpr int NB2 = 8 / r2;
#pragma unroll
    for (int b = 0; b < NB2; ++b) {
      const int j = t + b * TPL;
#pragma unroll
      for (int q = 0; q < r2; ++q) {
        const int o = si(j + q * (L / r2));
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f][b * r2 + q] = xb[f * fstride + o];
      }
    }
    if constexpr (!PingPong<SI>::v) line_sync<SI>();
    fft_passes<C, L, INV, NF, p + 1, SI>(v, sm, fstride, tw, t, si);
  }
}

// Mixed-radix passes p >= 1 through shared memory: the L/r butterflies of a
// pass are spread over the line's L/8 threads (some threads idle when they do
// not divide evenly); each thread reads all inputs of its butterflies before
// the block synchronises and the outputs overwrite them in place.
template <class C, int L, bool INV, int NF, int p, class SI>
__device__ __forceinline__ void fft_mixed_passes(C* sm, int fstride, const C* __restrict__ tw, int t, const SI& si) {
  using PL = MixedPlan<L>;
  constexpr int r = PL::rad(p);
  constexpr int Ns = PL::ns(p);
  constexpr int NBF = L / r;                       // butterflies in this pass
  constexpr int NB = (NBF + PL::TPL - 1) / PL::TPL;  // per thread (upper bound)
  constexpr int STW = L / (Ns * r);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    C w[NB][r];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + b * PL::TPL;
      if (j < NBF) {
#pragma unroll
        for (int q = 0; q < r; ++q) w[b][q] = sm[f * fstride + si(j + q * NBF)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + b * PL::TPL;
      if (j < NBF) {
        const int k = j % Ns;
#pragma unroll
        for (int q = 1; q < r; ++q) {
          const C tq = tw[q * k * STW];
          w[b][q] = INV ? cmulc(w[b][q], tq) : cmul(w[b][q], tq);
        }
        dft_r<r, INV>(w[b]);
        const int base = (j / Ns) * Ns * r + k;
#pragma unroll
        for (int q = 0; q < r; ++q) sm[f * fstride + si(base + q * Ns)] = w[b][q];
      }
    }
    __syncthreads();
  }
  if constexpr (p + 1 < PL::P) fft_mixed_passes<C, L, INV, NF, p + 1, SI>(sm, fstride, tw, t, si);
}

// Mixed-radix line transform with natural entry and exit layouts (register e
// of thread t holds position t + e L/8): the radix-8 first pass runs on the
// registers as loaded, the later passes in shared memory, and the result is
// read back in the same layout.
template <class C, int L, bool INV, int NF, class SI>
__device__ __forceinline__ void fft_mixed(C (&v)[NF][8], C* sm, int fstride, const C* __restrict__ tw, int t,
                                          const SI& si) {
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    dft8<INV>(v[f]);
#pragma unroll
    for (int q = 0; q < 8; ++q) sm[f * fstride + si(8 * t + q)] = v[f][q];
  }
  __syncthreads();
  fft_mixed_passes<C, L, INV, NF, 1, SI>(sm, fstride, tw, t, si);
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int e = 0; e < 8; ++e) v[f][e] = sm[f * fstride + si(t + e * MixedPlan<L>::TPL)];
  __syncthreads();  // callers may reuse the buffer
}

template <class C, int L, bool INV, int NF, class SI>
__device__ __forceinline__ void fft_line(C (&v)[NF][8], C* sm, int fstride, const C* __restrict__ tw, int t,
                                         const SI& si) {
  if constexpr (IsPow2<L>::v) fft_passes<C, L, INV, NF, 0, SI>(v, sm, fstride, tw, t, si);
  else fft_mixed<C, L, INV, NF, SI>(v, sm, fstride, tw, t, si);
}

// Shared-memory index maps.  Row tiles (lines contiguous in global memory):
// one padded line per row, one pad element per 128 bytes to break the
// power-of-two strides of the Stockham writes.  Column tiles (lines strided
// in global memory, M adjacent lines per tile): position-major, so each
// quarter/half warp touches one 128-byte row of the tile.
template <int PADSHIFT> struct RowIdx {
  __device__ __forceinline__ int operator()(int pos) const { return pos + (pos >> PADSHIFT); }
};
// MC > 0: the tile width M is the compile-time constant MC (the default tile
// rows), so the exchange offsets fold into the shared-memory instructions;
// MC = 0: M at run time (the other tile widths).
template <int MC> struct ColIdxT {
  int M;
  int alt;  // offset (elements) of the second exchange buffer from the first
  __device__ __forceinline__ int operator()(int pos) const { return pos * (MC > 0 ? MC : M); }
};
using ColIdx = ColIdxT<0>;
// A column transform of power-of-two length L makes P - 1 exchanges, the first
// through the second buffer.  When that count is odd the transform ends having
// written the second buffer last, so a following transform of the same line
// starts with the roles of the buffers swapped (its first exchange then writes
// the buffer whose last reads preceded the earlier barrier).
template <int L, class C, class SI> __device__ __forceinline__ void col_after(C*& sm, SI& si) {
  if constexpr (IsPow2<L>::v) {
    if constexpr (((Plan<L>::P - 1) & 1) != 0) {
      sm += si.alt;
      si.alt = -si.alt;
    }
  }
}
template <class R> struct PadShift;
template <> struct PadShift<double> { static constexpr int v = 3; };  // 8 x 16 B
template <> struct PadShift<float> { static constexpr int v = 4; };   // 16 x 8 B
template <class R, int L> __host__ __device__ constexpr int row_len_padded() {
  return L + (L >> PadShift<R>::v);
}

}  // namespace egpe
