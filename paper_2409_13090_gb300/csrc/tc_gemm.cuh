// Tensor-core (tcgen05, TF32) product tiles for SC_TF32. Placeholder until the
// tcgen05 kernel lands: no task is routed here, so SC_TF32 runs the SIMT FP32 path.
#pragma once
#include "kernels.cuh"

namespace sc {
inline bool tc_gemm_init() { return true; }
inline bool tc_eligible(const Task &) { return false; }
inline void tc_tiles_of(const Task &, int32_t, std::vector<GemmTile> &) {}
template <typename T>
inline bool launch_tc_gemm(T *, T *, const Task *, const GemmTile *, int32_t, cudaStream_t) { return false; }
}  // namespace sc
