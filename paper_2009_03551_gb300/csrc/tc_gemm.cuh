// Tensor-core (tcgen05) numeric phase: declarations shared with the driver.
#pragma once

#include "rdm_internal.cuh"

namespace rdm {

// work buffers of the tensor-core path (tile lists, per-tile step lists)
struct TcWork {
    DevBuf<int> tiles;        // per tile: descriptor ints
    DevBuf<int> steps;        // per tile step: operand block indices
    DevBuf<int> counters;
    DevBuf<int64_t> step_off;
    DevBuf<int> scan32;
    DevBuf<int64_t> scan64;
};

// Convert the FP64 master values of `in` into the operand planes of
// arithmetic `ar` (hi/lo halves in the shared-memory layout of the MMA).
void prepare_operands(MatSet &in, Arith ar, cudaStream_t st);

// Numeric phase on the tensor cores; same contract as launch_numeric_simt.
// Returns the number of flops issued to the tensor cores.
double launch_numeric_tc(const NumArgs &a, const MatSet &in, Arith ar, TcWork &w, int NB,
                         cudaStream_t st);

}  // namespace rdm
