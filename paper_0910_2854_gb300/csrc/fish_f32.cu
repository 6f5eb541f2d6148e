// fish_f32.cu -- FP32 instantiation of the launchers and of the one-column
// (scalar FP32) sweep kernels (FMA contraction allowed); the pressure
// recovery keeps its compensated final subtraction and the CFL and
// conserved-total reductions accumulate in FP64.
#include "fish_col_impl.cuh"
#include "fish_launch.cuh"

namespace fish {
// the two-column kernels are instantiated in fish_p2.cu
extern template cudaError_t col_fluid<P2>(const ColFluidArgs<float> &, bool, bool, cudaStream_t);
extern template cudaError_t col_ct<P2>(const ColCTArgs<float> &, bool, cudaStream_t);
template struct Launch<float>;
template cudaError_t col_fluid<float>(const ColFluidArgs<float> &, bool, bool, cudaStream_t);
template cudaError_t col_ct<float>(const ColCTArgs<float> &, bool, cudaStream_t);
}
