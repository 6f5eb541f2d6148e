// fish_p2_mm.cu -- the two-column L_d kernels with the minmod limiter (see fish_p2.cu).
#include "fish_col_impl.cuh"

namespace fish {
template cudaError_t col_fluid_launch<P2, false, false, LIM_MINMOD, true, false>(const ColFluidArgs<float> &, cudaStream_t);
template cudaError_t col_fluid_launch<P2, false, true, LIM_MINMOD, true, false>(const ColFluidArgs<float> &, cudaStream_t);
}
