// fish_vec.cuh -- lane-vector arithmetic for the column-march sweep kernels.
//
// A thread of the column kernels advances W pencils at once: W = 1 with
// V = double (FP64 path) or V = float, W = 2 with V = P2, two FP32 pencils
// that sit next to each other along the fastest memory axis.  P2 arithmetic
// maps onto the packed FP32x2 instructions of sm_100+ (one FADD2 / FMUL2 /
// FFMA2 issues two single-precision operations), and its loads and stores
// are single 64-bit accesses.  Comparisons, selections, reciprocals and
// square roots act on each component.
//
// The FP64 instantiation is compiled without FMA contraction and every
// formula keeps the operation order of the plain IEEE evaluation, so that
// the double path rounds like a straightforward implementation of the
// paper's formulas.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fish {

struct P2 {
    float2 v;
};

template <class V> struct VT;
template <> struct VT<double> {
    using S = double;
    static constexpr int W = 1;
    static constexpr bool F64 = true;
};
template <> struct VT<float> {
    using S = float;
    static constexpr int W = 1;
    static constexpr bool F64 = false;
};
template <> struct VT<P2> {
    using S = float;
    static constexpr int W = 2;
    static constexpr bool F64 = false;
};

// ---- P2 arithmetic -------------------------------------------------------
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return {__fmul2_rn(a.v, b.v)}; }
// a - b as one FFMA2: b * (-1) is exact, so the single rounding is that of a - b
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ P2 operator-(P2 a) { return {make_float2(-a.v.x, -a.v.y)}; }

// ---- construction and fused multiply-add ---------------------------------
template <class V> __device__ __forceinline__ V vb(typename VT<V>::S s);  // broadcast
template <> __device__ __forceinline__ double vb<double>(double s) { return s; }
template <> __device__ __forceinline__ float vb<float>(float s) { return s; }
template <> __device__ __forceinline__ P2 vb<P2>(float s) { return {make_float2(s, s)}; }

// a*b + c: unfused in FP64 (the IEEE order of the plain formula), fused in FP32
__device__ __forceinline__ double vfma(double a, double b, double c) { return a * b + c; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ P2 vfma(P2 a, P2 b, P2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }

// ---- component-wise functions ---------------------------------------------
__device__ __forceinline__ double vsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float vsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ P2 vsqrt(P2 a) { return {make_float2(sqrtf(a.v.x), sqrtf(a.v.y))}; }

__device__ __forceinline__ double vabs(double a) { return fabs(a); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ P2 vabs(P2 a) { return {make_float2(fabsf(a.v.x), fabsf(a.v.y))}; }

__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ P2 vmax(P2 a, P2 b) { return {make_float2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y))}; }

__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ P2 vmin(P2 a, P2 b) { return {make_float2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y))}; }

// reciprocal: IEEE in FP64, the fast hardware reciprocal (about 1 ulp) in FP32
__device__ __forceinline__ double vrcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float vrcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ P2 vrcp(P2 a) { return {make_float2(__fdividef(1.0f, a.v.x), __fdividef(1.0f, a.v.y))}; }

// quotient: IEEE in FP64, a * rcp(b) in FP32
__device__ __forceinline__ double vdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float vdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ P2 vdiv(P2 a, P2 b) { return a * vrcp(b); }

// select: c > 0 ? a : b, per component
__device__ __forceinline__ double vsel_pos(double c, double a, double b) { return c > 0.0 ? a : b; }
__device__ __forceinline__ float vsel_pos(float c, float a, float b) { return c > 0.0f ? a : b; }
__device__ __forceinline__ P2 vsel_pos(P2 c, P2 a, P2 b)
{
    return {make_float2(c.v.x > 0.0f ? a.v.x : b.v.x, c.v.y > 0.0f ? a.v.y : b.v.y)};
}

// component access (for the rare per-lane work)
__device__ __forceinline__ double vget(double a, int) { return a; }
__device__ __forceinline__ float vget(float a, int) { return a; }
__device__ __forceinline__ float vget(P2 a, int i) { return i ? a.v.y : a.v.x; }

// ---- limiters (eq0190 minmod, eq0200 Van Leer; sign(0) = 0, reading C-8) --
template <class S> __device__ __forceinline__ S ssgn(S a) { return a > S(0) ? S(1) : (a < S(0) ? S(-1) : S(0)); }

__device__ __forceinline__ double vminmod(double a, double b)
{
    return 0.5 * (ssgn(a) + ssgn(b)) * fmin(fabs(a), fabs(b));
}
__device__ __forceinline__ float sminmod_f(float a, float b)
{
    // same value as 0.5 (sgn a + sgn b) min(|a|, |b|) without the sign products
    return a * b > 0.0f ? copysignf(fminf(fabsf(a), fabsf(b)), a) : 0.0f;
}
__device__ __forceinline__ float vminmod(float a, float b) { return sminmod_f(a, b); }
__device__ __forceinline__ P2 vminmod(P2 a, P2 b)
{
    return {make_float2(sminmod_f(a.v.x, b.v.x), sminmod_f(a.v.y, b.v.y))};
}

__device__ __forceinline__ double vvanleer(double a, double b)
{
    if (a * b > 0.0) return 2.0 * a * b / (a + b);
    return 0.0;
}
__device__ __forceinline__ float vvanleer(float a, float b)
{
    const float ab = a * b;
    return ab > 0.0f ? __fdividef(ab + ab, a + b) : 0.0f;
}
__device__ __forceinline__ P2 vvanleer(P2 a, P2 b)
{
    const P2 ab = a * b;
    const P2 q = (ab + ab) * vrcp(a + b);
    return {make_float2(ab.v.x > 0.0f ? q.v.x : 0.0f, ab.v.y > 0.0f ? q.v.y : 0.0f)};
}

// limiter: 0 Van Leer, 1 minmod, 2 none (first order); LIM < 0 selects at
// run time from lim
template <int LIM, class V> __device__ __forceinline__ V vlimit(V a, V b, int lim)
{
    if constexpr (LIM == 0) return vvanleer(a, b);
    else if constexpr (LIM == 1) return vminmod(a, b);
    else if constexpr (LIM == 2) return vb<V>(0);
    else return lim == 0 ? vvanleer(a, b) : (lim == 1 ? vminmod(a, b) : vb<V>(0));
}

// ---- memory access -----------------------------------------------------------
// Loads of W consecutive values at element offset i of a field.
template <class V> __device__ __forceinline__ V vload(const typename VT<V>::S *p, long long i);
template <> __device__ __forceinline__ double vload<double>(const double *p, long long i) { return __ldg(p + i); }
template <> __device__ __forceinline__ float vload<float>(const float *p, long long i) { return __ldg(p + i); }
template <> __device__ __forceinline__ P2 vload<P2>(const float *p, long long i)
{
    return {__ldg(reinterpret_cast<const float2 *>(p + i))};
}

// Hint that the line holding p will be read soon: fetch it into L2 (no
// register is written and nothing waits for it).
__device__ __forceinline__ void pf_l2(const void *p) { asm volatile("prefetch.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ void vstore(double *p, long long i, double a) { p[i] = a; }
__device__ __forceinline__ void vstore(float *p, long long i, float a) { p[i] = a; }
__device__ __forceinline__ void vstore(float *p, long long i, P2 a) { *reinterpret_cast<float2 *>(p + i) = a.v; }

// The pair shifted down by one along the fast axis: (lo, a.x) for a = (a.x, a.y).
__device__ __forceinline__ double vshift_lo(double lo, double) { return lo; }
__device__ __forceinline__ float vshift_lo(float lo, float) { return lo; }
__device__ __forceinline__ P2 vshift_lo(float lo, P2 a) { return {make_float2(lo, a.v.x)}; }
// The pair shifted up by one: (a.y, hi).
__device__ __forceinline__ double vshift_hi(double, double hi) { return hi; }
__device__ __forceinline__ float vshift_hi(float, float hi) { return hi; }
__device__ __forceinline__ P2 vshift_hi(P2 a, float hi) { return {make_float2(a.v.y, hi)}; }

}  // namespace fish
