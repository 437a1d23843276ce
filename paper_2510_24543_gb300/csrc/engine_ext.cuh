// Launch dispatch for the line lengths compiled in translation units of their
// own: 48 and 96 (suffix mr), 80 (mr5) and 128, 256 (big).  Each
// unit defines one suffix with EGPE_EXT_DEFINE and instantiates it for one
// field precision with EGPE_EXT_INSTANTIATE.
#pragma once
#include "engine_impl.cuh"

#define EGPE_EXT_DEFINE(SFX, ...)                                                                          \
  namespace egpe {                                                                                         \
  template <class R> template <template <class, int> class OpT>                                            \
  egpe_status Engine<R>::dispatch_x_##SFX(int L, const KArgs<R>& a) {                                      \
    return dispatch_x_in<OpT, __VA_ARGS__>(L, a);                                                          \
  }                                                                                                        \
  template <class R> template <template <class, int> class OpT>                                            \
  egpe_status Engine<R>::dispatch_col_##SFX(int L, const KArgs<R>& a, const CUtensorMap* tm) {             \
    return dispatch_col_in<OpT, __VA_ARGS__>(L, a, tm);                                                    \
  }                                                                                                        \
  template <class R> egpe_status Engine<R>::plain_x_##SFX(int inverse, const KArgs<R>& a) {                \
    return plain_x_in<__VA_ARGS__>(inverse, a);                                                            \
  }                                                                                                        \
  template <class R>                                                                                       \
  egpe_status Engine<R>::plain_col_##SFX(int axis, int inverse, const KArgs<R>& a, const CUtensorMap* tm) { \
    return plain_col_in<__VA_ARGS__>(axis, inverse, a, tm);                                                \
  }                                                                                                        \
  }

#define EGPE_EXT_INSTANTIATE(R, SFX)                                                                     \
  namespace egpe {                                                                                       \
  template egpe_status Engine<R>::dispatch_x_##SFX<XFwdEG>(int, const KArgs<R>&);                        \
  template egpe_status Engine<R>::dispatch_x_##SFX<XInvEG>(int, const KArgs<R>&);                        \
  template egpe_status Engine<R>::dispatch_x_##SFX<XFwdPC>(int, const KArgs<R>&);                        \
  template egpe_status Engine<R>::dispatch_x_##SFX<XInvPC>(int, const KArgs<R>&);                        \
  template egpe_status Engine<R>::dispatch_x_##SFX<XFwdLC>(int, const KArgs<R>&);                        \
  template egpe_status Engine<R>::dispatch_x_##SFX<XInvLC>(int, const KArgs<R>&);                        \
  template egpe_status Engine<R>::dispatch_x_##SFX<XFwdKin>(int, const KArgs<R>&);                       \
  template egpe_status Engine<R>::dispatch_x_##SFX<XInvKin>(int, const KArgs<R>&);                       \
  template egpe_status Engine<R>::dispatch_x_##SFX<XFwdPG>(int, const KArgs<R>&);                        \
  template egpe_status Engine<R>::dispatch_x_##SFX<XInvPG>(int, const KArgs<R>&);                        \
  template egpe_status Engine<R>::dispatch_col_##SFX<ZEg>(int, const KArgs<R>&, const CUtensorMap*);     \
  template egpe_status Engine<R>::dispatch_col_##SFX<ZPc>(int, const KArgs<R>&, const CUtensorMap*);     \
  template egpe_status Engine<R>::dispatch_col_##SFX<ZLc>(int, const KArgs<R>&, const CUtensorMap*);     \
  template egpe_status Engine<R>::dispatch_col_##SFX<ZKin>(int, const KArgs<R>&, const CUtensorMap*);    \
  template egpe_status Engine<R>::dispatch_col_##SFX<ZPg>(int, const KArgs<R>&, const CUtensorMap*);     \
  template egpe_status Engine<R>::plain_x_##SFX(int, const KArgs<R>&);                                   \
  template egpe_status Engine<R>::plain_col_##SFX(int, int, const KArgs<R>&, const CUtensorMap*);        \
  }
