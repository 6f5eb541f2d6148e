// fish_f64.cu -- FP64 instantiation of the sweep kernels.  Compiled without
// FMA contraction (-fmad=false) so that every operation rounds like a plain
// IEEE double evaluation of the paper's formulas, in the order written.
#include "fish_col_impl.cuh"
#include "fish_launch.cuh"

namespace fish {
// the sweeps whose fast axis is t2 (FT1 = false) compile in fish_f64_t2.cu
#define FISH_F64_T2(HSE, GRAV, NU)                                                                                \
    extern template cudaError_t col_fluid_launch<double, HSE, GRAV, -1, false, NU>(const ColFluidArgs<double> &,  \
                                                                                   cudaStream_t);
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
extern template cudaError_t col_fluid_launch<double, false, 0, LIM_VANLEER, false, false>(const ColFluidArgs<double> &,
                                                                                        cudaStream_t);
extern template cudaError_t col_ct_launch<double, LIM_VANLEER, false, false>(const ColCTArgs<double> &, cudaStream_t);
extern template cudaError_t col_ct_launch<double, -1, false, false>(const ColCTArgs<double> &, cudaStream_t);
extern template cudaError_t col_ct_launch<double, -1, false, true>(const ColCTArgs<double> &, cudaStream_t);
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

// FP64 pipe throughput probe: every thread runs eight independent chains of
// fused multiply-adds (x <- x a + b, |a| < 1, so the chains stay bounded) and
// writes its sum, so nothing is optimised away.  The FP64 sweeps are
// compared against this rate (their DADD, DMUL and DFMA each take one issue
// of the FP64 pipe).
static __global__ void __launch_bounds__(256) dfma_probe_kernel(double *out, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __fma_rn(x[k], a, b);
    }
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += x[k];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

cudaError_t launch_dfma_probe(double *out, int blocks, int iters, cudaStream_t s)
{
    dfma_probe_kernel<<<blocks, 256, 0, s>>>(out, iters, 0.9999999, 1e-7);
    return cudaGetLastError();
}
}  // namespace fish

