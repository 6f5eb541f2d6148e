// fish_math.cuh -- per-cell and per-interface arithmetic of FISH's sweep
// (Kaeppeli et al., arXiv:0910.2854, Sec. 2), templated on the real type.
//
// Everything here is written in the evaluation order of the paper's
// formulas so that the FP64 build (compiled without FMA contraction) rounds
// exactly like a plain IEEE evaluation of them.  The FP32 build adds one
// compensated island: the final subtraction of the pressure recovery
// (E minus kinetic minus magnetic energy) is done with an error-free
// two-sum, so that cancellation there costs no more than the rounding of
// the inputs.
//
// Frame: component 0 is along the sweep direction d, components 1 and 2
// along t1 = d+1 and t2 = d+2 (cyclic); u = (rho, m_n, m_t1, m_t2, E),
// bb = cell-centred field (b_n, b_t1, b_t2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fish_types.h"

namespace fish {


template <class T> struct Real;
template <> struct Real<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
    static __device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }
};
template <> struct Real<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
    static __device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
};

// Reciprocal and quotient: IEEE in FP64 (the oracle's rounding), the fast
// hardware approximations (about 1-2 ulp) in FP32.
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
__device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }

// ---------------------------------------------------------------------------
// pressure recovery, eq0050 with E = rho e + rho v^2/2 + b^2/2
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T gas_pressure(T gm1, T E, T kin, T mag);

template <> __device__ __forceinline__ double gas_pressure<double>(double gm1, double E, double kin, double mag)
{
    return gm1 * (E - kin - mag);
}

// FP32: internal energy E - (kin + mag) with the error of kin + mag carried
// by a two-sum (Knuth), so the cancellation against E is exact when
// E and kin + mag are within a factor two (Sterbenz).
template <> __device__ __forceinline__ float gas_pressure<float>(float gm1, float E, float kin, float mag)
{
    float s = __fadd_rn(kin, mag);
    float bp = __fsub_rn(s, kin);
    float es = __fadd_rn(__fsub_rn(kin, __fsub_rn(s, bp)), __fsub_rn(mag, bp));
    float e = __fsub_rn(__fsub_rn(E, s), es);
    return gm1 * e;
}

// ---------------------------------------------------------------------------
// signal speed of one cell (CFL)
// ---------------------------------------------------------------------------
// |v_n| + c_F along the frame's first axis only (CFL, eq0084), in the
// operations and order of the sweeps' cell evaluation for those two
// quantities.
template <class T>
__device__ __forceinline__ T signal_speed(const T u[5], const T bb[3], T gamma, T gm1, unsigned &flags)
{
    const T rho = u[0];
    T v0, a2, bn2, bt2, p, kin;
    const T mag = T(0.5) * (bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
    if constexpr (sizeof(T) == 8) {
        v0 = u[1] / rho;
        const T v1 = u[2] / rho, v2 = u[3] / rho;
        kin = T(0.5) * (u[1] * v0 + u[2] * v1 + u[3] * v2);
        p = gas_pressure<T>(gm1, u[4], kin, mag);
        a2 = gamma * p / rho;
        bn2 = bb[0] * bb[0] / rho;
        bt2 = (bb[1] * bb[1] + bb[2] * bb[2]) / rho;
    } else {
        const T ri = rcp_(rho);
        v0 = u[1] * ri;
        const T v1 = u[2] * ri, v2 = u[3] * ri;
        kin = T(0.5) * (u[1] * v0 + u[2] * v1 + u[3] * v2);
        p = gas_pressure<T>(gm1, u[4], kin, mag);
        a2 = gamma * p * ri;
        bn2 = bb[0] * bb[0] * ri;
        bt2 = (bb[1] * bb[1] + bb[2] * bb[2]) * ri;
    }
    const T B2 = bn2 + bt2;
    const T disc = (a2 - B2) * (a2 - B2) + T(4) * a2 * bt2;
    const T cf = Real<T>::sqrt_(T(0.5) * (a2 + B2 + Real<T>::sqrt_(disc)));
    if (!(rho > T(0))) flags |= FLAG_RHO;
    if (!(p > T(0))) flags |= FLAG_P;
    if (rho != rho || p != p || cf != cf) flags |= FLAG_NAN;
    return Real<T>::abs_(v0) + cf;
}

// ---------------------------------------------------------------------------
// index helpers: ghost map (periodic wrap or outflow clamp)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int gmap(int s, int n, int bc)
{
    if (bc == BC_PERIODIC) {
        int r = s % n;
        return r < 0 ? r + n : r;
    }
    return s < 0 ? 0 : (s >= n ? n - 1 : s);
}

}  // namespace fish
