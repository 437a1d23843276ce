// Engine<float>: FP32 fields and transforms with FP64 reductions and controller.
#include "batch.cuh"
template class egpe::Engine<float>;
template egpe_status egpe::batch_solve<float>(const std::vector<egpe::Engine<float>*>&, cudaStream_t,
                                             const egpe_solve_opts&, int, int, double, double,
                                             std::vector<egpe::SolveRun>&, egpe_trace_entry*, int, int*);
