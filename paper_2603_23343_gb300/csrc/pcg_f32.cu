// Solver kernels and graph construction for FP32 iteration vectors
// (one translation unit per storage type, compiled in parallel).
#include "solver.cuh"

namespace gb {
template int solve_launch<float>(const SolveCall &, bool, cudaStream_t);
template int batched_capture<float>(const SolveCall *, const int *, int, cudaGraph_t *);
template int solve_profiled<float>(const SolveCall &, bool, gbpcg_result *, cudaStream_t);
template int solve_host_loop<float>(const SolveCall &, bool, cudaStream_t);
}  // namespace gb
