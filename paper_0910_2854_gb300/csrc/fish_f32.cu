// fish_f32.cu -- FP32 instantiation of the sweep kernels (FMA contraction
// allowed); the pressure recovery keeps its compensated final subtraction and
// the CFL and conserved-total reductions accumulate in FP64.
#include "fish_launch.cuh"

namespace fish {
template struct Launch<float>;
}
