// Engine<float>: FP32 fields and transforms; sums reduced deterministically
// (float-float) to FP64 values for the FP64 controller.
#include "batch.cuh"
template class egpe::Engine<float>;
template egpe_status egpe::batch_solve<float>(const std::vector<egpe::Engine<float>*>&, cudaStream_t,
                                             const egpe_solve_opts&, int, int, double, double,
                                             std::vector<egpe::SolveRun>&, egpe_trace_entry*, int, int*);
