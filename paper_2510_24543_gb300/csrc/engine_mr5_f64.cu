// Mixed-radix length 80 of Engine<double>.
#include "engine_ext.cuh"
EGPE_EXT_DEFINE(mr5, 80)
EGPE_EXT_INSTANTIATE(double, mr5)
