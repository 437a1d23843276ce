// Mixed-radix (48, 80, 96) launches of Engine<float>.
#include "engine_mr.cuh"
EGPE_MR_INSTANTIATE(float)
