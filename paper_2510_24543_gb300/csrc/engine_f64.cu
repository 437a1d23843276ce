// Engine<double>: the FP64 path.
#include "engine_impl.cuh"
template class egpe::Engine<double>;
