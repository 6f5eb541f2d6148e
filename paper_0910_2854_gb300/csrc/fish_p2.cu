// fish_p2.cu -- the two-column sweep kernels: FP32 pencils advanced in pairs
// with the packed FP32x2 instructions of sm_100+ (compiled with the FP32
// flags of fish_f32.cu).
#include "fish_col_impl.cuh"

namespace fish {
template cudaError_t col_fluid<P2>(const ColFluidArgs<float> &, bool, bool, cudaStream_t);
template cudaError_t col_ct<P2>(const ColCTArgs<float> &, bool, cudaStream_t);
}
