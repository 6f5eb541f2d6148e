// fish_ring.cu -- ring-fed FP32 sweep kernels (compiled with the FP32 flags
// of fish_f32.cu) and their launchers.
#include "fish_ring.cuh"

namespace fish {

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bool ring_fluid_applies(const ColFluidArgs<float> &A)
{
    if (A.phi || A.wd || A.sg) return false;
    if (A.nf < 4 || A.nf % 4 != 0) return false;
    if (A.lim != LIM_VANLEER && A.lim != LIM_MINMOD && A.lim != LIM_HYBRID) return false;
    // every bulk copy starts on a 16-byte boundary: aligned field bases and
    // element offsets / strides that are multiples of four floats
    for (int k = 0; k < 5; ++k)
        if (!aligned16(A.u[k])) return false;
    if (!aligned16(A.bd) || !aligned16(A.bt1) || !aligned16(A.bt2)) return false;
    if (A.off % 4 != 0 || A.so % 4 != 0 || A.sd % 4 != 0) return false;
    return true;
}

template <int LIM, bool CFLF> static cudaError_t ring_fluid_launch(const ColFluidArgs<float> &A, cudaStream_t s)
{
    // the shared-memory size attribute is per device: set it once per device
    static unsigned char done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[dev]) {
        e = cudaFuncSetAttribute(fluid_ring_kernel<LIM, CFLF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ring_fluid_smem());
        if (e != cudaSuccess) return e;
        done[dev] = 1;
    }
    const long long blocks = (long long)((A.nf + RF_COLS - 1) / RF_COLS) * A.no;
    fluid_ring_kernel<LIM, CFLF><<<(unsigned)blocks, RF_THREADS, ring_fluid_smem(), s>>>(A);
    return cudaGetLastError();
}

cudaError_t ring_fluid(const ColFluidArgs<float> &A, cudaStream_t s)
{
    if (!ring_fluid_applies(A)) return cudaErrorNotSupported;
    const bool c = A.cfl_min != nullptr;
    switch (A.lim) {
    case LIM_VANLEER: return c ? ring_fluid_launch<LIM_VANLEER, true>(A, s) : ring_fluid_launch<LIM_VANLEER, false>(A, s);
    case LIM_MINMOD: return c ? ring_fluid_launch<LIM_MINMOD, true>(A, s) : ring_fluid_launch<LIM_MINMOD, false>(A, s);
    case LIM_HYBRID: return c ? ring_fluid_launch<LIM_HYBRID, true>(A, s) : ring_fluid_launch<LIM_HYBRID, false>(A, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace fish
