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
// limiters, eq0190 (minmod) and eq0200 (Van Leer); sign(0) = 0
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T sgn(T a)
{
    return a > T(0) ? T(1) : (a < T(0) ? T(-1) : T(0));
}

template <class T> __device__ __forceinline__ T limit(int lim, T a, T b)
{
    if (lim == LIM_VANLEER) {
        if (a * b > T(0)) return div_(T(2) * a * b, a + b);
        return T(0);
    }
    if (lim == LIM_MINMOD)
        return T(0.5) * (sgn(a) + sgn(b)) * Real<T>::min_(Real<T>::abs_(a), Real<T>::abs_(b));
    return T(0);
}

template <class T> __device__ __forceinline__ T minmod(T a, T b)
{
    return T(0.5) * (sgn(a) + sgn(b)) * Real<T>::min_(Real<T>::abs_(a), Real<T>::abs_(b));
}

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
// one cell: primitives, flux vector (eq0100), freezing speed (label 0111)
// ---------------------------------------------------------------------------
template <class T> struct Cell {
    T u[5];
    T F[5];
    T p, cs, cf, vn, d;
};

template <class T>
__device__ __forceinline__ void cell_eval(const T u[5], const T bb[3], T gamma, T gm1, Cell<T> &c,
                                          unsigned &flags)
{
    const T rho = u[0];
#pragma unroll
    for (int k = 0; k < 5; ++k) c.u[k] = u[k];
    T v0, v1, v2, a2, bn2, bt2, p, kin;
    const T mag = T(0.5) * (bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
    if constexpr (sizeof(T) == 8) {
        v0 = u[1] / rho;
        v1 = u[2] / rho;
        v2 = u[3] / rho;
        kin = T(0.5) * (u[1] * v0 + u[2] * v1 + u[3] * v2);
        p = gas_pressure<T>(gm1, u[4], kin, mag);
        a2 = gamma * p / rho;
        bn2 = bb[0] * bb[0] / rho;
        bt2 = (bb[1] * bb[1] + bb[2] * bb[2]) / rho;
    } else {
        const T ri = rcp_(rho);
        v0 = u[1] * ri;
        v1 = u[2] * ri;
        v2 = u[3] * ri;
        kin = T(0.5) * (u[1] * v0 + u[2] * v1 + u[3] * v2);
        p = gas_pressure<T>(gm1, u[4], kin, mag);
        a2 = gamma * p * ri;
        bn2 = bb[0] * bb[0] * ri;
        bt2 = (bb[1] * bb[1] + bb[2] * bb[2]) * ri;
    }
    const T ptot = p + mag;
    const T B2 = bn2 + bt2;
    // fast speed along the sweep; discriminant as a sum of squares
    const T disc = (a2 - B2) * (a2 - B2) + T(4) * a2 * bt2;
    c.cf = Real<T>::sqrt_(T(0.5) * (a2 + B2 + Real<T>::sqrt_(disc)));
    c.cs = Real<T>::sqrt_(a2);
    c.p = p;
    c.vn = v0;
    c.d = Real<T>::abs_(v0) + c.cf;
    const T bv = bb[0] * v0 + bb[1] * v1 + bb[2] * v2;
    c.F[0] = u[1];
    c.F[1] = u[1] * v0 + ptot - bb[0] * bb[0];
    c.F[2] = u[2] * v0 - bb[0] * bb[1];
    c.F[3] = u[3] * v0 - bb[0] * bb[2];
    c.F[4] = (u[4] + ptot) * v0 - bb[0] * bv;
    if (!(rho > T(0))) flags |= FLAG_RHO;
    if (!(p > T(0))) flags |= FLAG_P;
    if (rho != rho || p != p || c.cf != c.cf) flags |= FLAG_NAN;
}

// |v_n| + c_F along the frame's first axis only (CFL, eq0084); same
// operations and order as cell_eval for those two quantities.
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

// hydrostatic estimate g (eq0321) and HSE-corrected difference (eq0323)
template <class T>
__device__ __forceinline__ void hse_delta(const Cell<T> &a, const Cell<T> &b, T phia, T phib, T du[5], T ddu[5])
{
    T xa[5], xb[5];
    xa[0] = -a.u[0]; xa[1] = -a.u[1]; xa[2] = -a.u[2]; xa[3] = -a.u[3];
    xa[4] = -(a.u[4] + a.p);
    xb[0] = -b.u[0]; xb[1] = -b.u[1]; xb[2] = -b.u[2]; xb[3] = -b.u[3];
    xb[4] = -(b.u[4] + b.p);
    const T fac = div_(phib - phia, a.cs * b.cs);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const T gk = T(0.5) * (xb[k] + xa[k]) * fac;
        du[k] = b.u[k] - a.u[k];
        ddu[k] = minmod(du[k] - gk, du[k]);
    }
}

// first-order interface flux: eq0140 with D = alpha max(d_a, d_b) (eq0150),
// or with the HSE correction eq0324 (D_adv, D_ac scaled by alpha)
template <class T, bool HSE>
__device__ __forceinline__ void flux1(const Cell<T> &a, const Cell<T> &b, T phia, T phib, T alpha, T F[5])
{
    if (!HSE) {
        const T D = alpha * Real<T>::max_(a.d, b.d);
#pragma unroll
        for (int k = 0; k < 5; ++k) F[k] = T(0.5) * (a.F[k] + b.F[k]) - T(0.5) * D * (b.u[k] - a.u[k]);
    } else {
        T du[5], ddu[5];
        const T Dadv = alpha * Real<T>::max_(Real<T>::abs_(a.vn), Real<T>::abs_(b.vn));
        const T Dac = alpha * Real<T>::max_(a.cf, b.cf);
        hse_delta(a, b, phia, phib, du, ddu);
#pragma unroll
        for (int k = 0; k < 5; ++k)
            F[k] = T(0.5) * (a.F[k] + b.F[k]) - T(0.5) * Dadv * du[k] - T(0.5) * Dac * ddu[k];
    }
}

// second-order TVD flux at the interface c1|c2 from predicted cells c0..c3
// (eq0160-eq0230; one freezing speed per interface, reading C-2; HSE form
// of the slope differences, reading C-19)
template <class T, bool HSE>
__device__ __forceinline__ void flux2(int lim, const Cell<T> &c0, const Cell<T> &c1, const Cell<T> &c2,
                                      const Cell<T> &c3, T ph0, T ph1, T ph2, T ph3, T F[5])
{
    if (!HSE && sizeof(T) == 4) {
        // FP32: the same flux written with differences of F and u, so each
        // split-flux slope costs one multiply-add:
        //   F+_{j+1} - F+_j = (dF_j + D du_j)/2,  F-_{j+1} - F-_j = (dF_j - D du_j)/2
        //   F = (F_e + F_{e+1})/2 - D du_e/2 + [phi(+) - phi(-)]/2
        const T D = Real<T>::max_(c1.d, c2.d);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const T df0 = c1.F[k] - c0.F[k], du0 = c1.u[k] - c0.u[k];
            const T df1 = c2.F[k] - c1.F[k], du1 = c2.u[k] - c1.u[k];
            const T df2 = c3.F[k] - c2.F[k], du2 = c3.u[k] - c2.u[k];
            const T slp = limit(lim, df0 + D * du0, df1 + D * du1);
            const T slm = limit(lim, df1 - D * du1, df2 - D * du2);
            F[k] = T(0.5) * (c1.F[k] + c2.F[k]) - T(0.5) * D * du1 + T(0.25) * (slp - slm);
        }
    } else if (!HSE) {
        const T D = Real<T>::max_(c1.d, c2.d);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const T fp0 = T(0.5) * (c0.F[k] + D * c0.u[k]);
            const T fp1 = T(0.5) * (c1.F[k] + D * c1.u[k]);
            const T fp2 = T(0.5) * (c2.F[k] + D * c2.u[k]);
            const T fm1 = T(0.5) * (c1.F[k] - D * c1.u[k]);
            const T fm2 = T(0.5) * (c2.F[k] - D * c2.u[k]);
            const T fm3 = T(0.5) * (c3.F[k] - D * c3.u[k]);
            const T slp = limit(lim, fp1 - fp0, fp2 - fp1);
            const T slm = limit(lim, fm2 - fm1, fm3 - fm2);
            F[k] = fp1 + fm2 + T(0.5) * (slp - slm);
        }
    } else {
        const T Dadv = Real<T>::max_(Real<T>::abs_(c1.vn), Real<T>::abs_(c2.vn));
        const T Dac = Real<T>::max_(c1.cf, c2.cf);
        T du0[5], dd0[5], du1[5], dd1[5], du2[5], dd2[5];
        hse_delta(c0, c1, ph0, ph1, du0, dd0);
        hse_delta(c1, c2, ph1, ph2, du1, dd1);
        hse_delta(c2, c3, ph2, ph3, du2, dd2);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const T q0 = Dadv * du0[k] + Dac * dd0[k];
            const T q1 = Dadv * du1[k] + Dac * dd1[k];
            const T q2 = Dadv * du2[k] + Dac * dd2[k];
            const T fp_l = T(0.5) * ((c1.F[k] - c0.F[k]) + q0);
            const T fp_r = T(0.5) * ((c2.F[k] - c1.F[k]) + q1);
            const T fm_l = T(0.5) * ((c2.F[k] - c1.F[k]) - q1);
            const T fm_r = T(0.5) * ((c3.F[k] - c2.F[k]) - q2);
            const T slp = limit(lim, fp_l, fp_r);
            const T slm = limit(lim, fm_l, fm_r);
            F[k] = T(0.5) * (c1.F[k] + c2.F[k]) - T(0.5) * q1 + T(0.5) * (slp - slm);
        }
    }
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
