// fish_f64.cu -- FP64 instantiation of the sweep kernels.  Compiled without
// FMA contraction (-fmad=false) so that every operation rounds like a plain
// IEEE double evaluation of the paper's formulas, in the order written.
#include "fish_col_impl.cuh"
#include "fish_launch.cuh"

namespace fish {
template struct Launch<double>;
template cudaError_t col_fluid<double>(const ColFluidArgs<double> &, bool, bool, cudaStream_t);
template cudaError_t col_ct<double>(const ColCTArgs<double> &, bool, cudaStream_t);
}

namespace fish {
cudaError_t launch_cfl_finish(unsigned long long *minbits, double k, double *dt, double *dt_copy,
                              cudaStream_t s)
{
    cfl_finish_kernel<<<1, 1, 0, s>>>(minbits, k, dt, dt_copy);
    return cudaGetLastError();
}

static __global__ void reset_min_kernel(unsigned long long *p) { *p = 0x7FF0000000000000ull; }

cudaError_t launch_reset_min(unsigned long long *minbits, cudaStream_t s)
{
    reset_min_kernel<<<1, 1, 0, s>>>(minbits);
    return cudaGetLastError();
}

cudaError_t launch_set_scalar(double *p, double v, cudaStream_t s)
{
    set_scalar_kernel<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}
}  // namespace fish
