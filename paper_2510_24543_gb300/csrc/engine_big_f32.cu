// Lengths 128 and 256 of Engine<float>.
#include "engine_ext.cuh"
EGPE_EXT_DEFINE(big, 128, 256)
EGPE_EXT_INSTANTIATE(float, big)
