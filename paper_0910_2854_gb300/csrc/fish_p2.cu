// fish_p2.cu -- the two-column sweep kernels: FP32 pencils advanced in pairs
// with the packed FP32x2 instructions of sm_100+ (compiled with the FP32
// flags of fish_f32.cu).  This unit holds the dispatcher and the Van Leer
// kernels; fish_p2_mm.cu and fish_p2_hy.cu the minmod and hybrid ones, so
// the three compile in parallel.
#include "fish_col_impl.cuh"

namespace fish {
#define FISH_P2_OTHER(LIMV)                                                                                     \
    extern template cudaError_t col_fluid_launch<P2, false, 0, LIMV, true, false>(const ColFluidArgs<float> &,  \
                                                                                 cudaStream_t);                \
    extern template cudaError_t col_fluid_launch<P2, false, 1, LIMV, true, false>(const ColFluidArgs<float> &,  \
                                                                                 cudaStream_t);                \
    extern template cudaError_t col_fluid_launch<P2, false, 2, LIMV, true, false>(const ColFluidArgs<float> &,  \
                                                                                 cudaStream_t);
FISH_P2_OTHER(LIM_MINMOD)
FISH_P2_OTHER(LIM_HYBRID)
#undef FISH_P2_OTHER
template cudaError_t col_fluid<P2>(const ColFluidArgs<float> &, bool, bool, cudaStream_t);
#ifdef FISH_CT_PAIRS
template cudaError_t col_ct<P2>(const ColCTArgs<float> &, bool, cudaStream_t);
#endif
}
