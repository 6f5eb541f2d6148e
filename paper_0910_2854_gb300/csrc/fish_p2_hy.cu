// fish_p2_hy.cu -- the two-column L_d kernels with the hybrid limiter (see fish_p2.cu).
#include "fish_col_impl.cuh"

namespace fish {
template cudaError_t col_fluid_launch<P2, false, 0, LIM_HYBRID, true, false>(const ColFluidArgs<float> &, cudaStream_t);
template cudaError_t col_fluid_launch<P2, false, 1, LIM_HYBRID, true, false>(const ColFluidArgs<float> &, cudaStream_t);
template cudaError_t col_fluid_launch<P2, false, 2, LIM_HYBRID, true, false>(const ColFluidArgs<float> &, cudaStream_t);
}
