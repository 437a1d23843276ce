// Mixed-radix lengths 48 and 96 of Engine<float>.
#include "engine_ext.cuh"
EGPE_EXT_DEFINE(mr, 48, 96)
EGPE_EXT_INSTANTIATE(float, mr)
