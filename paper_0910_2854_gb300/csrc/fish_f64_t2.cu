// fish_f64_t2.cu -- the FP64 sweep kernels whose fast transverse axis is t2
// (FT1 = false), compiled in parallel with fish_f64.cu and with the same
// flags (-fmad=false).
#include "fish_col_impl.cuh"

namespace fish {
#define FISH_F64_T2(HSE, GRAV, NU) \
    template cudaError_t col_fluid_launch<double, HSE, GRAV, -1, false, NU>(const ColFluidArgs<double> &, cudaStream_t);
FISH_F64_T2(false, 0, false)
FISH_F64_T2(false, 0, true)
FISH_F64_T2(false, 1, false)
FISH_F64_T2(false, 1, true)
FISH_F64_T2(true, 0, false)
FISH_F64_T2(true, 0, true)
FISH_F64_T2(true, 1, false)
FISH_F64_T2(true, 1, true)
FISH_F64_T2(false, 2, false)
#undef FISH_F64_T2
template cudaError_t col_fluid_launch<double, false, 0, LIM_VANLEER, false, false>(const ColFluidArgs<double> &,
                                                                                 cudaStream_t);
template cudaError_t col_ct_launch<double, LIM_VANLEER, false, false>(const ColCTArgs<double> &, cudaStream_t);
template cudaError_t col_ct_launch<double, -1, false, false>(const ColCTArgs<double> &, cudaStream_t);
template cudaError_t col_ct_launch<double, -1, false, true>(const ColCTArgs<double> &, cudaStream_t);
}
