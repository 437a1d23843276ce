// Engine<float>: FP32 fields and transforms with FP64 reductions and controller.
#include "engine_impl.cuh"
template class egpe::Engine<float>;
