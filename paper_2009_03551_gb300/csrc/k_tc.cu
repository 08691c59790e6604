// Tensor-core numeric phase (tcgen05, sm_103a).
#include "tc_gemm.cuh"

namespace rdm {

void prepare_operands(MatSet &in, Arith ar, cudaStream_t st) {
    (void)in; (void)ar; (void)st;
    throw Error{-1, "tensor-core arithmetic is not available in this build"};
}

double launch_numeric_tc(const NumArgs &a, const MatSet &in, Arith ar, TcWork &w, int NB,
                         cudaStream_t st) {
    (void)a; (void)in; (void)ar; (void)w; (void)NB; (void)st;
    throw Error{-1, "tensor-core arithmetic is not available in this build"};
}

}  // namespace rdm
