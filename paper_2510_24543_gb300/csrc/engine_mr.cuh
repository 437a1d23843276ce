// Launch dispatch of the mixed-radix line lengths 48, 80 and 96 (transform
// plans in fft.cuh).  Included only by engine_mr_f64.cu and engine_mr_f32.cu,
// which instantiate it for every pipeline op.
#pragma once
#include "engine_impl.cuh"

namespace egpe {

template <class R> template <template <class, int> class OpT>
egpe_status Engine<R>::dispatch_x_mr(int L, const KArgs<R>& a) {
  switch (L) {
    case 48: return launch_x<OpT<R, 48>>(a);
    case 80: return launch_x<OpT<R, 80>>(a);
    case 96: return launch_x<OpT<R, 96>>(a);
  }
  return EGPE_ERR_UNSUPPORTED;
}

template <class R> template <template <class, int> class OpT>
egpe_status Engine<R>::dispatch_col_mr(int L, const KArgs<R>& a, const CUtensorMap* tm) {
  switch (L) {
    case 48: return launch_col<OpT<R, 48>>(a, tm);
    case 80: return launch_col<OpT<R, 80>>(a, tm);
    case 96: return launch_col<OpT<R, 96>>(a, tm);
  }
  return EGPE_ERR_UNSUPPORTED;
}

template <class R> egpe_status Engine<R>::plain_x_mr(int inverse, const KArgs<R>& a) {
#define EGPE_PX(LL) \
  case LL: return inverse ? launch_x<XPlain<R, LL, true>>(a) : launch_x<XPlain<R, LL, false>>(a);
  switch (nx) {
    EGPE_PX(48) EGPE_PX(80) EGPE_PX(96)
  }
#undef EGPE_PX
  return EGPE_ERR_UNSUPPORTED;
}

template <class R>
egpe_status Engine<R>::plain_col_mr(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm) {
  const int L = axis == 1 ? ny : nz;
#define EGPE_PC(LL)                                                                                        \
  case LL:                                                                                                 \
    if (axis == 1)                                                                                         \
      return inverse ? launch_col<ColPlain<R, LL, 1, true>>(a, tm) : launch_col<ColPlain<R, LL, 1, false>>(a, tm); \
    return inverse ? launch_col<ColPlain<R, LL, 2, true>>(a, tm) : launch_col<ColPlain<R, LL, 2, false>>(a, tm);
  switch (L) {
    EGPE_PC(48) EGPE_PC(80) EGPE_PC(96)
  }
#undef EGPE_PC
  return EGPE_ERR_UNSUPPORTED;
}

}  // namespace egpe

// Explicit instantiations for one field precision R.
#define EGPE_MR_INSTANTIATE(R)                                                                           \
  namespace egpe {                                                                                       \
  template egpe_status Engine<R>::dispatch_x_mr<XFwdEG>(int, const KArgs<R>&);                           \
  template egpe_status Engine<R>::dispatch_x_mr<XInvEG>(int, const KArgs<R>&);                           \
  template egpe_status Engine<R>::dispatch_x_mr<XInvW3>(int, const KArgs<R>&);                           \
  template egpe_status Engine<R>::dispatch_x_mr<XFwdPC>(int, const KArgs<R>&);                           \
  template egpe_status Engine<R>::dispatch_x_mr<XInvPC>(int, const KArgs<R>&);                           \
  template egpe_status Engine<R>::dispatch_x_mr<XFwdLC>(int, const KArgs<R>&);                           \
  template egpe_status Engine<R>::dispatch_x_mr<XInvLC>(int, const KArgs<R>&);                           \
  template egpe_status Engine<R>::dispatch_x_mr<XInvW1F2>(int, const KArgs<R>&);                         \
  template egpe_status Engine<R>::dispatch_x_mr<XFwdKin>(int, const KArgs<R>&);                          \
  template egpe_status Engine<R>::dispatch_x_mr<XInvKin>(int, const KArgs<R>&);                          \
  template egpe_status Engine<R>::dispatch_col_mr<ZEg>(int, const KArgs<R>&, const CUtensorMap*);        \
  template egpe_status Engine<R>::dispatch_col_mr<ZPc>(int, const KArgs<R>&, const CUtensorMap*);        \
  template egpe_status Engine<R>::dispatch_col_mr<ZLc>(int, const KArgs<R>&, const CUtensorMap*);        \
  template egpe_status Engine<R>::dispatch_col_mr<ZKin>(int, const KArgs<R>&, const CUtensorMap*);       \
  template egpe_status Engine<R>::plain_x_mr(int, const KArgs<R>&);                                      \
  template egpe_status Engine<R>::plain_col_mr(int, int, const KArgs<R>&, const CUtensorMap*);           \
  }
