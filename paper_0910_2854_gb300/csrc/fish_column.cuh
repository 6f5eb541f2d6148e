// fish_column.cuh -- column-march kernels of FISH's fluid operator L_d and
// magnetic operator B_d (Kaeppeli et al., arXiv:0910.2854, Sec. 2-3).
//
// Geometry.  A sweep runs along axis d with element stride sd.  The two
// transverse axes are the "fast" axis (element stride 1, the fastest memory
// axis of the current layout) and the "other" axis (stride so).  A thread
// owns W adjacent columns along the fast axis (V = P2: two FP32 columns
// advanced together with packed FP32x2 arithmetic and 64-bit accesses;
// V = float or double: one column) and marches them along d, so every global
// access of a warp is coalesced.  In the x-fastest layout this serves the y
// and z sweeps; the x sweeps run on the y-fastest copy of the state.
//
// The march is the paper's pipelined loop (Sec. 3) held in registers: raw
// cell r enters, predicted cell r-1 is formed, corrected cell r-3 leaves.
// Windows are indexed by r mod 4 (unrolled by four) so they rotate without
// moves; the steady-state loop over interior cells carries no boundary tests,
// ghost cells (periodic wrap or zeroth-order extrapolation, no ghost storage)
// are handled by a short prologue and a guarded tail.
//
// Both operators read the current buffers and write the other ones.
#pragma once

#include <type_traits>

#include "fish_math.cuh"
#include "fish_types.h"
#include "fish_vec.cuh"

namespace fish {

// ---------------------------------------------------------------------------
// arguments
// ---------------------------------------------------------------------------
template <class S> struct ColFluidArgs {
    const S *u[5];          // rho, m_d, m_t1, m_t2, E of the current buffer (sweep frame)
    const S *bd, *bt1, *bt2;  // face fields b_d, b_t1, b_t2 (sweep frame)
    S *uo[5];               // outputs, sweep frame
    const S *phi;           // potential or nullptr; FP32: phi(next cell along d) - phi(cell), from FP64
    const double *dt;
    long long off;          // element offset of the box in the field arrays (batches; else 0)
    long long sd, so;       // strides along the sweep and the other transverse axis
    int n, nf, no;          // cells along the sweep, the fast and the other axis
    int bc;
    int lim;                // limiter (kernels with LIM < 0 read it at run time)
    S gamma, gm1, alpha;
    double h;               // cell width along d
    unsigned *flags;
    // CFL of the updated state (kernels built with CFLF): the maximum over the
    // output cells of (|v_a| + c_F,a) / h_a over the three axes a in the frame
    // order (d, t1, t2) goes to *cfl_min as the order-preserving bits of its
    // reciprocal (atomic minimum)
    unsigned long long *cfl_min;
    S rh[3];
    const S *wd = nullptr;  // irregular mesh (kernels built with NU): the n cell widths along d
    int sg = 0;             // 1: phi drives operator-split kicks G_d(dt/2) around the sweep, not source terms
};

template <class S> struct ColCTArgs {
    const S *rho, *md;      // density and momentum along d (unchanged by B_d)
    const S *bd, *bf, *bo;  // b_d and the face fields of the fast and other transverse axes
    S *bdo, *bfo, *boo;     // outputs (other buffer)
    const double *dt;
    long long off;          // element offset of the box in the field arrays (batches; else 0)
    long long sd, so;
    int n, nf, no;
    int bc;
    int lim;
    double h, hf, ho;       // cell widths along d, the fast and the other axis
    // irregular mesh (kernels built with NU): cell widths along d, fast, other
    const S *wd = nullptr, *wf = nullptr, *wo = nullptr;
};

// ---------------------------------------------------------------------------
// per-cell arithmetic (frame: component 0 along d)
// ---------------------------------------------------------------------------
template <class V> struct CCell {
    V u[5];
    V F[5];
    V d;                 // freezing speed |v_d| + c_F (label 0111)
    V p, cs, cf, vn;     // used by the hydrostatic correction only
};

// running checks for reading C-16: min rho, min p, and a sum of c_F that
// turns NaN if any evaluated cell produced one
template <class V> struct Checks {
    V mn_rho, mn_p, nsum;
};

template <class V> __device__ __forceinline__ void checks_init(Checks<V> &k)
{
    k.mn_rho = vb<V>(3.0e38f);
    k.mn_p = vb<V>(3.0e38f);
    k.nsum = vb<V>(0.0f);
}

template <class V> __device__ __forceinline__ unsigned checks_flags(const Checks<V> &k)
{
    unsigned f = 0;
#pragma unroll
    for (int i = 0; i < VT<V>::W; ++i) {
        const auto r = vget(k.mn_rho, i), p = vget(k.mn_p, i), s = vget(k.nsum, i);
        if (!(r > 0)) f |= FLAG_RHO;
        if (!(p > 0)) f |= FLAG_P;
        if (s != s) f |= FLAG_NAN;
    }
    return f;
}

// E - (kin + mag) with the rounding error of kin + mag carried by an
// error-free two-sum (Knuth), so the cancellation against E costs no more
// than the rounding of its inputs (the FP32 compensated island).
__device__ __forceinline__ float eint_comp(float E, float kin, float mag)
{
    const float s = __fadd_rn(kin, mag);
    const float bp = __fsub_rn(s, kin);
    const float es = __fadd_rn(__fsub_rn(kin, __fsub_rn(s, bp)), __fsub_rn(mag, bp));
    return __fsub_rn(__fsub_rn(E, s), es);
}
__device__ __forceinline__ P2 eint_comp(P2 E, P2 kin, P2 mag)
{
    const P2 s = kin + mag;
    const P2 bp = s - kin;
    const P2 es = (kin - (s - bp)) + (mag - bp);
    return (E - s) - es;
}

// Primitives, flux vector (eq0100) and freezing speed (label 0111) of a cell
// with conserved state u and cell-centred field bb (reading C-1 for c_F).
template <class V>
__device__ __forceinline__ void ceval(const V u[5], const V bb[3], V gamma, V gm1, CCell<V> &c, Checks<V> &k)
{
    const V rho = u[0];
#pragma unroll
    for (int i = 0; i < 5; ++i) c.u[i] = u[i];
    V v0, v1, v2, p, a2, bn2, bt2, mag;
    if constexpr (VT<V>::F64) {
        v0 = u[1] / rho;
        v1 = u[2] / rho;
        v2 = u[3] / rho;
        const V kin = 0.5 * (u[1] * v0 + u[2] * v1 + u[3] * v2);
        mag = 0.5 * (bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
        p = gm1 * (u[4] - kin - mag);
        a2 = gamma * p / rho;
        bn2 = bb[0] * bb[0] / rho;
        bt2 = (bb[1] * bb[1] + bb[2] * bb[2]) / rho;
    } else {
        const V half = vb<V>(0.5f);
        const V ri = vrcp(rho);
        v0 = u[1] * ri;
        v1 = u[2] * ri;
        v2 = u[3] * ri;
        const V kin = half * vfma(u[3], v2, vfma(u[2], v1, u[1] * v0));
        const V bb2 = bb[2] * bb[2];
        const V bt = vfma(bb[1], bb[1], bb2);
        const V bn = bb[0] * bb[0];
        mag = half * (bn + bt);
        p = gm1 * eint_comp(u[4], kin, mag);
        a2 = gamma * p * ri;
        bn2 = bn * ri;
        bt2 = bt * ri;
    }
    const V ptot = p + mag;
    const V B2 = bn2 + bt2;
    V disc;
    if constexpr (VT<V>::F64) disc = (a2 - B2) * (a2 - B2) + 4.0 * a2 * bt2;
    else disc = vfma(a2 - B2, a2 - B2, vb<V>(4.0f) * a2 * bt2);
    c.cf = vsqrt(vb<V>(0.5f) * (a2 + B2 + vsqrt(disc)));
    c.cs = vsqrt(a2);
    c.p = p;
    c.vn = v0;
    c.d = vabs(v0) + c.cf;
    if constexpr (VT<V>::F64) {
        const V bv = bb[0] * v0 + bb[1] * v1 + bb[2] * v2;
        c.F[0] = u[1];
        c.F[1] = u[1] * v0 + ptot - bb[0] * bb[0];
        c.F[2] = u[2] * v0 - bb[0] * bb[1];
        c.F[3] = u[3] * v0 - bb[0] * bb[2];
        c.F[4] = (u[4] + ptot) * v0 - bb[0] * bv;
    } else {
        const V bv = vfma(bb[2], v2, vfma(bb[1], v1, bb[0] * v0));
        const V nb0 = -bb[0];
        c.F[0] = u[1];
        c.F[1] = vfma(nb0, bb[0], vfma(u[1], v0, ptot));
        c.F[2] = vfma(nb0, bb[1], u[2] * v0);
        c.F[3] = vfma(nb0, bb[2], u[3] * v0);
        c.F[4] = vfma(nb0, bv, (u[4] + ptot) * v0);
    }
    k.mn_rho = vmin(k.mn_rho, rho);
    k.mn_p = vmin(k.mn_p, p);
    k.nsum = k.nsum + c.cf;
}

// Potential difference phi_b - phi_a across the interface a|b.  FP64 takes
// the difference of the cell potentials; the FP32 kernels read, per cell,
// the difference to the next cell along the sweep (formed in FP64 when the
// potential is set), so phia already holds phi_b - phi_a.
template <class V> __device__ __forceinline__ V pdiff(V phia, V phib)
{
    if constexpr (VT<V>::F64) return phib - phia;
    else return phia;
}

// hydrostatic estimate g (eq0321) and the HSE-corrected difference (eq0323).
// FP32 island: g = s * fac is split into its rounded value and the exact
// rounding error (TwoProduct with an FMA), both subtracted from du, so the
// cancellation du - g near equilibrium adds no product rounding.
template <class V>
__device__ __forceinline__ void chse(const CCell<V> &a, const CCell<V> &b, V phia, V phib, V du[5], V ddu[5])
{
    V xa[5], xb[5];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        xa[i] = -a.u[i];
        xb[i] = -b.u[i];
    }
    xa[4] = -(a.u[4] + a.p);
    xb[4] = -(b.u[4] + b.p);
    const V fac = vdiv(pdiff(phia, phib), a.cs * b.cs);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        du[i] = b.u[i] - a.u[i];
        if constexpr (VT<V>::F64) {
            const V g = 0.5 * (xb[i] + xa[i]) * fac;
            ddu[i] = vminmod(du[i] - g, du[i]);
        } else {
            const V sx = vb<V>(0.5f) * (xb[i] + xa[i]);
            const V ghi = sx * fac;
            const V glo = vfma(sx, fac, -ghi);
            ddu[i] = vminmod((du[i] - ghi) - glo, du[i]);
        }
    }
}

// first-order interface flux: eq0140 with D = alpha max(d_a, d_b) (eq0150),
// or the HSE-corrected form eq0324 (reading C-3)
template <class V, bool HSE>
__device__ __forceinline__ void cflux1(const CCell<V> &a, const CCell<V> &b, V phia, V phib, V alpha, V F[5])
{
    if constexpr (!HSE) {
        const V D = alpha * vmax(a.d, b.d);
        if constexpr (VT<V>::F64) {
#pragma unroll
            for (int i = 0; i < 5; ++i) F[i] = 0.5 * (a.F[i] + b.F[i]) - 0.5 * D * (b.u[i] - a.u[i]);
        } else {
            const V half = vb<V>(0.5f);
#pragma unroll
            for (int i = 0; i < 5; ++i) F[i] = half * vfma(-D, b.u[i] - a.u[i], a.F[i] + b.F[i]);
        }
    } else {
        V du[5], ddu[5];
        const V Dadv = alpha * vmax(vabs(a.vn), vabs(b.vn));
        const V Dac = alpha * vmax(a.cf, b.cf);
        chse(a, b, phia, phib, du, ddu);
        const V half = vb<V>(0.5f);
#pragma unroll
        for (int i = 0; i < 5; ++i)
            F[i] = half * (a.F[i] + b.F[i]) - half * Dadv * du[i] - half * Dac * ddu[i];
    }
}

// second-order TVD flux at the interface c1|c2 from predicted cells c0..c3
// (eq0160-eq0230; one freezing speed per interface, reading C-2; HSE form of
// the slope differences, reading C-19).  The hybrid limiter is taken only by
// the one-column kernels with the limiter read at run time.
// NU (irregular mesh, reading C-25): each one-sided difference is divided
// by the distance of the centres it joins and the limited slope carried
// over half the width of its own cell (w1 for F+, w2 for F-).
template <class V, bool HSE, int LIM, bool NU = false>
__device__ __forceinline__ void cflux2(const CCell<V> &c0, const CCell<V> &c1, const CCell<V> &c2, const CCell<V> &c3,
                                       V ph0, V ph1, V ph2, V ph3, V F[5], int lim, V w0 = V(), V w1 = V(),
                                       V w2 = V(), V w3 = V())
{
    V gl = w0, gc = w1, gr = w2;
    if constexpr (NU) {
        const V half = vb<V>(0.5f);
        gl = half * (w0 + w1);
        gc = half * (w1 + w2);
        gr = half * (w2 + w3);
    }
    if constexpr (LIM < 0 && VT<V>::W == 1) {
        // hybrid limiter (Sec. 2.2): minmod where either cell of the
        // interface moves faster than its sound speed, else Van Leer (reading C-21)
        if (lim == LIM_HYBRID)
            lim = (vabs(c1.vn) > c1.cs || vabs(c2.vn) > c2.cs) ? LIM_MINMOD : LIM_VANLEER;
    }
    // compile-time hybrid (LIM = LIM_HYBRID, packed kernels): per lane,
    // sup > 0 where either cell is supersonic (|v| - c_S > 0 iff |v| > c_S)
    V sup = vb<V>(0.0f);
    if constexpr (LIM == LIM_HYBRID) sup = vmax(vabs(c1.vn) - c1.cs, vabs(c2.vn) - c2.cs);
    if constexpr (!HSE && !VT<V>::F64) {
        // FP32: F = (F_e + F_{e+1})/2 - D du_e/2 + [phi(+) - phi(-)]/4 with the
        // split-flux slopes written as dF +- D du (each one multiply-add)
        const V D = vmax(c1.d, c2.d);
        const V nD = -D;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const V df0 = c1.F[i] - c0.F[i], du0 = c1.u[i] - c0.u[i];
            const V df1 = c2.F[i] - c1.F[i], du1 = c2.u[i] - c1.u[i];
            const V df2 = c3.F[i] - c2.F[i], du2 = c3.u[i] - c2.u[i];
            V slp, slm;
            if constexpr (NU) {
                slp = w1 * vlimit<LIM>(vdiv(vfma(D, du0, df0), gl), vdiv(vfma(D, du1, df1), gc), lim);
                slm = w2 * vlimit<LIM>(vdiv(vfma(nD, du1, df1), gc), vdiv(vfma(nD, du2, df2), gr), lim);
            } else if constexpr (LIM == LIM_HYBRID) {
                const V ap = vfma(D, du0, df0), bp = vfma(D, du1, df1);
                const V am = vfma(nD, du1, df1), bm = vfma(nD, du2, df2);
                slp = vsel_pos(sup, vminmod(ap, bp), vvanleer(ap, bp));
                slm = vsel_pos(sup, vminmod(am, bm), vvanleer(am, bm));
            } else {
                slp = vlimit<LIM>(vfma(D, du0, df0), vfma(D, du1, df1), lim);
                slm = vlimit<LIM>(vfma(nD, du1, df1), vfma(nD, du2, df2), lim);
            }
            F[i] = vfma(vb<V>(0.5f), vfma(nD, du1, c1.F[i] + c2.F[i]), vb<V>(0.25f) * (slp - slm));
        }
    } else if constexpr (!HSE) {
        const V D = vmax(c1.d, c2.d);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const V fp0 = 0.5 * (c0.F[i] + D * c0.u[i]);
            const V fp1 = 0.5 * (c1.F[i] + D * c1.u[i]);
            const V fp2 = 0.5 * (c2.F[i] + D * c2.u[i]);
            const V fm1 = 0.5 * (c1.F[i] - D * c1.u[i]);
            const V fm2 = 0.5 * (c2.F[i] - D * c2.u[i]);
            const V fm3 = 0.5 * (c3.F[i] - D * c3.u[i]);
            V slp, slm;
            if constexpr (NU) {
                slp = w1 * vlimit<LIM>((fp1 - fp0) / gl, (fp2 - fp1) / gc, lim);
                slm = w2 * vlimit<LIM>((fm2 - fm1) / gc, (fm3 - fm2) / gr, lim);
            } else {
                slp = vlimit<LIM>(fp1 - fp0, fp2 - fp1, lim);
                slm = vlimit<LIM>(fm2 - fm1, fm3 - fm2, lim);
            }
            F[i] = fp1 + fm2 + 0.5 * (slp - slm);
        }
    } else {
        const V half = vb<V>(0.5f);
        const V Dadv = vmax(vabs(c1.vn), vabs(c2.vn));
        const V Dac = vmax(c1.cf, c2.cf);
        V du0[5], dd0[5], du1[5], dd1[5], du2[5], dd2[5];
        chse(c0, c1, ph0, ph1, du0, dd0);
        chse(c1, c2, ph1, ph2, du1, dd1);
        chse(c2, c3, ph2, ph3, du2, dd2);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const V q0 = Dadv * du0[i] + Dac * dd0[i];
            const V q1 = Dadv * du1[i] + Dac * dd1[i];
            const V q2 = Dadv * du2[i] + Dac * dd2[i];
            const V fp_l = half * ((c1.F[i] - c0.F[i]) + q0);
            const V fp_r = half * ((c2.F[i] - c1.F[i]) + q1);
            const V fm_l = half * ((c2.F[i] - c1.F[i]) - q1);
            const V fm_r = half * ((c3.F[i] - c2.F[i]) - q2);
            V slp, slm;
            if constexpr (NU) {
                slp = w1 * vlimit<LIM>(vdiv(fp_l, gl), vdiv(fp_r, gc), lim);
                slm = w2 * vlimit<LIM>(vdiv(fm_l, gc), vdiv(fm_r, gr), lim);
            } else {
                slp = vlimit<LIM>(fp_l, fp_r, lim);
                slm = vlimit<LIM>(fm_l, fm_r, lim);
            }
            F[i] = half * (c1.F[i] + c2.F[i]) - half * q1 + half * (slp - slm);
        }
    }
}

// Largest (|v_a| + c_F,a) / h_a over the three axes of the frame (eq0083-
// eq0084, reading C-15) for a cell with conserved state u and cell-centred
// field b; the primitives are shared between the axes (FP32 path).
template <class V>
__device__ __forceinline__ V cfl_rate3(const V u[5], const V b[3], V gamma, V gm1, const V rh[3])
{
    const V half = vb<V>(0.5f);
    const V ri = vrcp(u[0]);
    const V v0 = u[1] * ri, v1 = u[2] * ri, v2 = u[3] * ri;
    const V kin = half * vfma(u[3], v2, vfma(u[2], v1, u[1] * v0));
    const V q0 = b[0] * b[0], q1 = b[1] * b[1], q2 = b[2] * b[2];
    const V mag = half * (q0 + q1 + q2);
    const V p = gm1 * eint_comp(u[4], kin, mag);
    const V a2 = gamma * p * ri;
    const V B2 = (q0 + q1 + q2) * ri;
    const V am = a2 - B2;
    const V c0 = am * am;
    const V aB = a2 + B2;
    const V f4a2 = vb<V>(4.0f) * a2;
    const V r0 = (vabs(v0) + vsqrt(half * (aB + vsqrt(vfma(f4a2, (q1 + q2) * ri, c0))))) * rh[0];
    const V r1 = (vabs(v1) + vsqrt(half * (aB + vsqrt(vfma(f4a2, (q0 + q2) * ri, c0))))) * rh[1];
    const V r2 = (vabs(v2) + vsqrt(half * (aB + vsqrt(vfma(f4a2, (q0 + q1) * ri, c0))))) * rh[2];
    return vmax(vmax(r0, r1), r2);
}

// ---------------------------------------------------------------------------
// L_d: fluid column march
// ---------------------------------------------------------------------------
template <class V> struct FRaw {
    V u[5];
    V bd;      // b_d at the cell's own (upper) face
    V bdm;     // b_d at the lower face
    V bf;      // fast-axis transverse face field at the cell's own faces
    V bo, bom; // other-axis transverse face field at own / lower face
    V phi;
    typename VT<V>::S bfm;  // fast-axis field at the face below the first column
    typename VT<V>::S w;    // cell width along d (irregular mesh; the same for all columns of a group)
};

template <class V> struct FMarch {
    FRaw<V> R;           // raw input of the next cell (prefetched)
    CCell<V> C[2];       // evaluated raw cells r-1, r (slot r & 1)
    V bb[2][3];          // their cell-centred field
    V ph[2];             // their potential
    V F1[2][5];          // predictor fluxes at (r-2, r-1), (r-1, r)
    CCell<V> P[4];       // predicted cells (slot index mod 4)
    V q[4];              // their potential
    V F2[2][5];          // corrector fluxes
    V phm2;              // potential of raw cell r-2
    Checks<V> chk;
    V cflr;              // largest CFL rate of the output cells (CFLF)
    typename VT<V>::S w0, w1, w2, w3, w4;  // irregular mesh: widths of raw cells r, r-1, .. r-4
    V dprev;             // split gravity: potential (FP64) or its difference (FP32) of raw cell r-1
};

// IX: element index type (int where every index of the launch fits, else
// long long): a load then costs one wide multiply-add for its address.
template <class S, class IX = long long> struct FCtx {
    IX base;             // offset of cell 0 of the first column
    IX ofm;              // offset of the fast-axis face below the first column
    IX oom;              // offset of the other-axis face below (mapped)
};

// L2 prefetch of one cell of a warp's march with a single instruction: lane
// l takes field row l / 2 (u0..u4, b_d, b_f, b_o, b_o of the row below, the
// potential) and the (l % 2)-th 128-byte line of the warp's span of it in
// cell 0, shifted by whole cells along the sweep (when the stride along the
// sweep is not a multiple of a line the lines drift by less than one line:
// it is a hint).
#ifndef FISH_FL_PF_WARP
#define FISH_FL_PF_WARP 1
#endif
template <class S, class IX> struct FPf {
    const S *p;   // the lane's line in cell 0 (nullptr: lane idle); cell c: p + c * sd
};

template <class S, class IX>
__device__ __forceinline__ void fpf_setup(const ColFluidArgs<S> &A, const S *bfp, const S *bop, IX base0, IX oom0,
                                          int span, bool grav, int lane, FPf<S, IX> &P)
{
    P.p = nullptr;
    const int r = lane >> 1;
    if (r >= (grav ? 10 : 9)) return;
    const S *f = r < 5 ? A.u[r] : (r == 5 ? A.bd : (r == 6 ? bfp : (r == 9 ? A.phi : bop)));
    const IX r0 = base0 + (r == 8 ? oom0 : (IX)0);
    const IX line = (r0 & ~(IX)31) + (IX)(32 * (lane & 1));
    if (line <= r0 + (IX)(span - 1)) P.p = f + line;
}

template <class S, class IX>
__device__ __forceinline__ void fpf_step(const ColFluidArgs<S> &A, const FPf<S, IX> &P, int c)
{
    if (P.p) pf_l2(P.p + (IX)c * (IX)A.sd);
}

// load raw cell s (any s): every index through the boundary map; a ghost
// cell copies the mapped cell as a whole, its lower b_d face included
template <class V, bool GRAV, bool FT1, class IX = long long>
__device__ __forceinline__ void fload_mapped(const ColFluidArgs<typename VT<V>::S> &A,
                                             const FCtx<typename VT<V>::S, IX> &X, int s, FRaw<V> &R)
{
    const int cc = gmap(s, A.n, A.bc);
    const IX i = X.base + (IX)cc * (IX)A.sd;
    const IX im = X.base + (IX)gmap(cc - 1, A.n, A.bc) * (IX)A.sd;
    const auto *bfp = FT1 ? A.bt1 : A.bt2;
    const auto *bop = FT1 ? A.bt2 : A.bt1;
#pragma unroll
    for (int k = 0; k < 5; ++k) R.u[k] = vload<V>(A.u[k], i);
    R.bd = vload<V>(A.bd, i);
    R.bdm = vload<V>(A.bd, im);
    R.bf = vload<V>(bfp, i);
    R.bfm = __ldg(bfp + i + X.ofm);
    R.bo = vload<V>(bop, i);
    R.bom = vload<V>(bop, i + X.oom);
    if (GRAV) {
        // FP32 reads the difference to the next cell: zero between the copies
        // of an outflow boundary cell (and across its face)
        R.phi = vload<V>(A.phi, i);
        if constexpr (!VT<V>::F64)
            if (A.bc == BC_OUTFLOW && (s < 0 || s >= A.n)) R.phi = vb<V>(0.0f);
    }
    // a ghost has the width of the cell it copies (reading C-23)
    if (A.wd) R.w = A.wd[cc];
}

// load interior cell at element offset i (no map; its lower b_d face is the
// upper face of the previous cell, set by the caller)
template <class V, bool GRAV, bool FT1, class IX = long long>
__device__ __forceinline__ void fload_direct(const ColFluidArgs<typename VT<V>::S> &A,
                                             const FCtx<typename VT<V>::S, IX> &X, IX i, FRaw<V> &R)
{
    const auto *bfp = FT1 ? A.bt1 : A.bt2;
    const auto *bop = FT1 ? A.bt2 : A.bt1;
#pragma unroll
    for (int k = 0; k < 5; ++k) R.u[k] = vload<V>(A.u[k], i);
    R.bd = vload<V>(A.bd, i);
    R.bf = vload<V>(bfp, i);
    R.bfm = __ldg(bfp + i + X.ofm);
    R.bo = vload<V>(bop, i);
    R.bom = vload<V>(bop, i + X.oom);
    if (GRAV) R.phi = vload<V>(A.phi, i);
}

// L2 prefetch distance of the steady-state loops (cells ahead of the load)
#ifndef FISH_PF_DIST
#define FISH_PF_DIST 2
#endif

#ifndef FISH_FL_PF_NEIGH
#define FISH_FL_PF_NEIGH 1   // also the lower other-axis face (a neighbour row)
#endif
// prefetch into L2 the fields the fluid march will load for interior cell i
template <class V, bool GRAV, bool FT1, class IX = long long>
__device__ __forceinline__ void fprefetch(const ColFluidArgs<typename VT<V>::S> &A,
                                          const FCtx<typename VT<V>::S, IX> &X, IX i)
{
    const auto *bfp = FT1 ? A.bt1 : A.bt2;
    const auto *bop = FT1 ? A.bt2 : A.bt1;
#pragma unroll
    for (int k = 0; k < 5; ++k) pf_l2(A.u[k] + i);
    pf_l2(A.bd + i);
    pf_l2(bfp + i);
    pf_l2(bop + i);
#if FISH_FL_PF_NEIGH
    pf_l2(bop + i + X.oom);
#endif
    if (GRAV) pf_l2(A.phi + i);
}

// Stage flags of one march step.
enum : int { ST_F1 = 1, ST_PRED = 2, ST_F2 = 4, ST_OUT = 8 };
// Load kinds: none, interior (direct), mapped.
enum : int { LD_NONE = 0, LD_DIRECT = 1, LD_MAPPED = 2, LD_DIRECT_PF = 3 };

// One step of the march for raw cell r (K = r mod 4).  The raw data of cell
// r is in M.R on entry (loaded by the previous step); the step loads raw
// cell r+1 (kind LD) into M.R.  FT1: the fast axis is t1 (else t2).  NU:
// irregular mesh along d (eq037): the cells' own widths replace h (the
// widths of raw cells r .. r-4 ride along in M.w0 .. M.w4).
// Operator-split gravity kick G_d(tau) of one cell (eq02512, reading C-22):
// m_d -= tau rho dphi, E changes by the kinetic energy change; FP64 in the
// oracle's operation order.
template <class V> __device__ __forceinline__ void sg_kick(V u[5], V dk, V tau)
{
    if constexpr (VT<V>::F64) {
        const V mo = u[1];
        const V mn = mo - tau * u[0] * dk;
        u[1] = mn;
        u[4] = u[4] + 0.5 * (mn * mn - mo * mo) / u[0];
    } else {
        const V mo = u[1];
        const V dm = -(tau * u[0]) * dk;
        u[1] = mo + dm;
        u[4] = u[4] + vdiv(dm * vfma(vb<V>(0.5f), dm, mo), u[0]);
    }
}

// Centred potential difference (eq02513) of the image cell of ghost r (its
// copy along d): FP64 from the potential, FP32 from the stored differences
// D_c = phi_{c+1} - phi_c (D_{-1} = 0 at an outflow boundary).
template <class V, class IX = long long>
__device__ __forceinline__ V sg_image_dk(const ColFluidArgs<typename VT<V>::S> &A,
                                         const FCtx<typename VT<V>::S, IX> &X, int r, V rtwoh)
{
    const int cc = gmap(r, A.n, A.bc);
    if constexpr (VT<V>::F64) {
        const V pp = vload<V>(A.phi, X.base + (IX)gmap(cc + 1, A.n, A.bc) * (IX)A.sd);
        const V pm = vload<V>(A.phi, X.base + (IX)gmap(cc - 1, A.n, A.bc) * (IX)A.sd);
        return (pp - pm) / (2.0 * A.h);
    } else {
        const V dc = vload<V>(A.phi, X.base + (IX)cc * (IX)A.sd);
        V dl = vb<V>(0.0f);
        if (cc > 0 || A.bc == BC_PERIODIC) dl = vload<V>(A.phi, X.base + (IX)gmap(cc - 1, A.n, A.bc) * (IX)A.sd);
        return (dc + dl) * rtwoh;
    }
}

// GM: gravity mode, 0 none, 1 unsplit source terms (eq0253-eq0255), 2
// operator-split kicks G_d(dt/2) folded into the march (eq025111): the raw
// cell is kicked as it is consumed, the output cell's old state before its
// update and the result after it (reading C-22 for the kick).
#ifndef FISH_CFL_SMEM
#define FISH_CFL_SMEM 1   // CFL epilogue: cell-centred field from a shared-memory ring
#endif
// The ring of the packed kernels with the CFL epilogue (blocks of 128
// threads): the cell-centred fields of a thread's raw cells r .. r-3, slot
// r mod 4, component k at [(slot * 3 + k) * 128 + thread]; only the kernels
// that use it allocate it.
static __shared__ float2 cfl_bb_ring[4 * 3 * 128];

template <class V, bool HSE, int GM, int LIM, bool FT1, bool CFLF, bool NU, int K, int ST, int LD, class IX = long long,
          bool PFW = FISH_FL_PF_WARP != 0>
__device__ __forceinline__ void fstep(const ColFluidArgs<typename VT<V>::S> &A, const FCtx<typename VT<V>::S, IX> &X,
                                      FMarch<V> &M, int r, V lam, V lamh, V hdt, V dt, V rtwoh,
                                      const FPf<typename VT<V>::S, IX> &PF)
{
    constexpr bool GRAV = GM == 1, SG = GM == 2, PHI = GM != 0;
    constexpr int k2 = K & 1, p2 = (K + 1) & 1;
    const V half = vb<V>(0.5f);
    // consume the raw input of cell r
    V bbr[3];
    V ur[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) ur[k] = M.R.u[k];
    bbr[0] = half * (M.R.bdm + M.R.bd);
    const V bd_r = M.R.bd;
    const V bfc = half * (vshift_lo(M.R.bfm, M.R.bf) + M.R.bf);
    const V boc = half * (M.R.bom + M.R.bo);
    if constexpr (FT1) {
        bbr[1] = bfc;
        bbr[2] = boc;
    } else {
        bbr[1] = boc;
        bbr[2] = bfc;
    }
    const V phr = PHI ? M.R.phi : vb<V>(0.0f);  // no potential: phi = 0
    if constexpr (CFLF && FISH_CFL_SMEM) {
        // keep the cell-centred field of raw cell r for the CFL rate of its
        // update three steps later (b is unchanged by L_d)
        static_assert(VT<V>::W == 2, "the CFL epilogue is built for the packed kernels");
        const int t = threadIdx.x & 127;
#pragma unroll
        for (int k = 0; k < 3; ++k) cfl_bb_ring[((K & 3) * 3 + k) * 128 + t] = bbr[k].v;
    }
    if constexpr (NU) {
        M.w4 = M.w3;
        M.w3 = M.w2;
        M.w2 = M.w1;
        M.w1 = M.w0;
        M.w0 = M.R.w;
    }
    // prefetch raw cell r+1
    if constexpr (LD == LD_DIRECT || LD == LD_DIRECT_PF) {
        fload_direct<V, PHI, FT1, IX>(A, X, X.base + (IX)(r + 1) * (IX)A.sd, M.R);
        if constexpr (NU) M.R.w = A.wd[r + 1];
        M.R.bdm = bd_r;
        if constexpr (LD == LD_DIRECT_PF) {
            const int pf = min(r + 1 + FISH_PF_DIST, A.n - 1);
            if constexpr (PFW) fpf_step(A, PF, pf);
            else fprefetch<V, PHI, FT1, IX>(A, X, X.base + (IX)pf * (IX)A.sd);
        }
    } else if constexpr (LD == LD_MAPPED) {
        fload_mapped<V, PHI, FT1, IX>(A, X, r + 1, M.R);
    }
    // old state of the output cell o = r-3
    const int o = r - 3;
    const IX io = X.base + (IX)o * (IX)A.sd;
    V un[5];
    if constexpr ((ST & ST_OUT) != 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) un[k] = vload<V>(A.u[k], io);
    }
    if constexpr (SG) {
        // kick of raw cell r with its centred potential difference (a ghost
        // takes its image cell's), and of the output cell's old state
        V dk;
        if (r < 0 || r >= A.n) {
            dk = sg_image_dk<V, IX>(A, X, r, rtwoh);
        } else if constexpr (VT<V>::F64) {
            dk = (M.R.phi - M.dprev) / (2.0 * A.h);  // phi_{r+1} - phi_{r-1}
        } else {
            dk = (phr + M.dprev) * rtwoh;            // D_r + D_{r-1}
        }
        M.dprev = phr;
        sg_kick<V>(ur, dk, hdt);
        M.ph[k2] = dk;
        if constexpr ((ST & ST_OUT) != 0) sg_kick<V>(un, M.q[(K + 1) & 3], hdt);
    }
    ceval<V>(ur, bbr, vb<V>(A.gamma), vb<V>(A.gm1), M.C[k2], M.chk);
#pragma unroll
    for (int k = 0; k < 3; ++k) M.bb[k2][k] = bbr[k];
    if (!SG && (GRAV || HSE)) M.ph[k2] = phr;
    if constexpr ((ST & ST_F1) != 0) {
        // predictor flux at (r-1, r) (eq0140 / eq0324)
        cflux1<V, HSE>(M.C[p2], M.C[k2], M.ph[p2], phr, vb<V>(A.alpha), M.F1[k2]);
    }
    if constexpr ((ST & ST_PRED) != 0) {
        // predicted half step of cell r-1 (eq0253; source eq0254, reading C-6)
        const CCell<V> &cp = M.C[p2];
        V up[5];
        V lh = lamh;
        if constexpr (NU) {
            if constexpr (VT<V>::F64) lh = dt / (2.0 * M.w1);
            else lh = vdiv(hdt, vb<V>(M.w1));
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if constexpr (VT<V>::F64) up[k] = cp.u[k] - lh * (M.F1[k2][k] - M.F1[p2][k]);
            else up[k] = vfma(-lh, M.F1[k2][k] - M.F1[p2][k], cp.u[k]);
        }
        if (GRAV) {
            // centred difference phi_r - phi_{r-2} (eq02513; NU: over the
            // centre span, reading C-26)
            V dphi;
            if constexpr (NU) {
                const V span = vb<V>(0.5f) * vb<V>(M.w2) + vb<V>(M.w1) + vb<V>(0.5f) * vb<V>(M.w0);
                if constexpr (VT<V>::F64) dphi = (phr - M.phm2) / span;
                else dphi = vdiv(M.ph[p2] + M.phm2, span);
            } else if constexpr (VT<V>::F64) {
                dphi = (phr - M.phm2) / (2.0 * A.h);
            } else {
                dphi = (M.ph[p2] + M.phm2) * rtwoh;
            }
            up[1] = up[1] - hdt * cp.u[0] * dphi;
            up[4] = up[4] - hdt * cp.u[1] * dphi;
        }
        constexpr int s3 = (K + 3) & 3;  // slot of cell r-1
        ceval<V>(up, M.bb[p2], vb<V>(A.gamma), vb<V>(A.gm1), M.P[s3], M.chk);
        if (PHI || HSE) M.q[s3] = M.ph[p2];
        if constexpr ((ST & ST_F2) != 0) {
            // corrector flux at (r-3, r-2) from predicted cells r-4 .. r-1 (eq0230)
            constexpr int s0 = K & 3, s1 = (K + 1) & 3, s2 = (K + 2) & 3;
            cflux2<V, HSE, LIM, NU>(M.P[s0], M.P[s1], M.P[s2], M.P[s3], M.q[s0], M.q[s1], M.q[s2], M.q[s3],
                                    M.F2[k2], A.lim, vb<V>(M.w4), vb<V>(M.w3), vb<V>(M.w2), vb<V>(M.w1));
            if constexpr ((ST & ST_OUT) != 0) {
                V lo = lam;
                if constexpr (NU) {
                    if constexpr (VT<V>::F64) lo = dt / M.w3;
                    else lo = vdiv(dt, vb<V>(M.w3));
                }
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    if constexpr (VT<V>::F64) un[k] = un[k] - lo * (M.F2[k2][k] - M.F2[p2][k]);
                    else un[k] = vfma(-lo, M.F2[k2][k] - M.F2[p2][k], un[k]);
                }
                if (GRAV) {
                    // corrector source from the predicted state (eq0255)
                    V dphi;
                    if constexpr (NU) {
                        const V span = vb<V>(0.5f) * vb<V>(M.w4) + vb<V>(M.w3) + vb<V>(0.5f) * vb<V>(M.w2);
                        if constexpr (VT<V>::F64) dphi = (M.q[s2] - M.q[s0]) / span;
                        else dphi = vdiv(M.q[s0] + M.q[s1], span);
                    } else if constexpr (VT<V>::F64) {
                        dphi = (M.q[s2] - M.q[s0]) / (2.0 * A.h);
                    } else {
                        dphi = (M.q[s0] + M.q[s1]) * rtwoh;
                    }
                    un[1] = un[1] - dt * M.P[s1].u[0] * dphi;
                    un[4] = un[4] - dt * M.P[s1].u[1] * dphi;
                }
                if constexpr (SG) sg_kick<V>(un, M.q[s1], hdt);  // output cell: second half kick
#pragma unroll
                for (int k = 0; k < 5; ++k) vstore(A.uo[k], io, un[k]);
                if constexpr (CFLF) {
                    // CFL rate of the updated cell with its cell-centred field,
                    // formed when the cell entered as raw cell o = r-3 (slot
                    // (r-3) mod 4 of the ring)
                    V bc[3];
                    if constexpr (FISH_CFL_SMEM) {
                        const int t = threadIdx.x & 127;
#pragma unroll
                        for (int k = 0; k < 3; ++k) bc[k].v = cfl_bb_ring[(((K + 1) & 3) * 3 + k) * 128 + t];
                    } else {
                        const auto *bfp = FT1 ? A.bt1 : A.bt2;
                        const auto *bop = FT1 ? A.bt2 : A.bt1;
                        const IX iom = X.base + (IX)(o > 0 ? o - 1 : gmap(-1, A.n, A.bc)) * (IX)A.sd;
                        bc[0] = half * (vload<V>(A.bd, iom) + vload<V>(A.bd, io));
                        const V bfv = vload<V>(bfp, io);
                        const V bfc = half * (vshift_lo(__ldg(bfp + io + X.ofm), bfv) + bfv);
                        const V boc = half * (vload<V>(bop, io + X.oom) + vload<V>(bop, io));
                        bc[FT1 ? 1 : 2] = bfc;
                        bc[FT1 ? 2 : 1] = boc;
                    }
                    const V rh[3] = {vb<V>(A.rh[0]), vb<V>(A.rh[1]), vb<V>(A.rh[2])};
                    M.cflr = vmax(M.cflr, cfl_rate3<V>(un, bc, vb<V>(A.gamma), vb<V>(A.gm1), rh));
                }
            }
        }
    }
    if (GRAV) M.phm2 = M.ph[p2];
}

#ifndef FISH_COL_MINB
#define FISH_COL_MINB 2
#endif
#ifndef FISH_COL_MINB1
#define FISH_COL_MINB1 3   // one-column FP32 kernels
#endif

// L_d over all columns.  The prologue runs raw cells -3 .. 2 (K = 1, 2, 3,
// 0, 1, 2); boxes with n < 8 load everything through the map.
template <class V, bool HSE, int GRAV, int LIM, bool FT1, bool CFLF, bool NU, int PLD, class IX = long long,
          bool PFW = FISH_FL_PF_WARP != 0>
__device__ __forceinline__ void fprologue(const ColFluidArgs<typename VT<V>::S> &A,
                                          const FCtx<typename VT<V>::S, IX> &X, FMarch<V> &M, V lam, V lamh, V hdt,
                                          V dt, V rtwoh, const FPf<typename VT<V>::S, IX> &PF)
{
    fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 1, 0, LD_MAPPED, IX, PFW>(A, X, M, -3, lam, lamh, hdt, dt, rtwoh, PF);
    fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 2, ST_F1, LD_MAPPED, IX, PFW>(A, X, M, -2, lam, lamh, hdt, dt, rtwoh, PF);
    fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 3, ST_F1 | ST_PRED, PLD, IX, PFW>(A, X, M, -1, lam, lamh, hdt, dt, rtwoh, PF);
    fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 0, ST_F1 | ST_PRED, PLD, IX, PFW>(A, X, M, 0, lam, lamh, hdt, dt, rtwoh, PF);
    fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 1, ST_F1 | ST_PRED, PLD, IX, PFW>(A, X, M, 1, lam, lamh, hdt, dt, rtwoh, PF);
    fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 2, ST_F1 | ST_PRED | ST_F2, PLD, IX, PFW>(A, X, M, 2, lam, lamh, hdt, dt, rtwoh, PF);
}

#ifndef FISH_COL_MINB
#define FISH_COL_MINB 2
#endif
#ifndef FISH_COL_MINB1
#define FISH_COL_MINB1 3   // one-column FP32 kernels
#endif

// The march of thread cid (column group cid of the box described by A).
// PFW: L2 prefetch of the next cells by one instruction per warp over the
// warp's span of its first row (the single-box sweeps, whose rows hold a
// multiple of 32 column groups), or per lane and field (the batch, whose
// short rows leave warps that straddle two rows)
template <class V, bool HSE, int GRAV, int LIM, bool FT1, bool CFLF, bool NU = false, class IX = long long,
          bool PFW = FISH_FL_PF_WARP != 0>
__device__ __forceinline__ void fluid_columns(const ColFluidArgs<typename VT<V>::S> &A, long long cid)
{
    using S = typename VT<V>::S;
    constexpr int W = VT<V>::W;
    const int cols = A.nf / W;
    if (cid >= (long long)cols * A.no) return;
    const int fp = (int)(cid % cols), ob = (int)(cid / cols);
    const int f0 = fp * W;
    FCtx<S, IX> X;
    X.base = (IX)A.off + (IX)f0 + (IX)ob * (IX)A.so;
    X.ofm = (IX)(gmap(f0 - 1, A.nf, A.bc) - f0);
    X.oom = (IX)(gmap(ob - 1, A.no, A.bc) - ob) * (IX)A.so;
    // per-warp L2 prefetch over the span of the warp's first lane (32 groups
    // of W columns; a warp that crosses a row end prefetches its first row)
    FPf<S, IX> PF;
    PF.p = nullptr;
    if constexpr (PFW) {
        const unsigned am = __activemask();
        const int l0 = __ffs(am) - 1;
        const IX b0 = __shfl_sync(am, X.base, l0);
        const IX m0 = __shfl_sync(am, X.oom, l0);
        const int span = min(32 * W, A.nf - (int)(b0 - (IX)A.off) % A.nf);
        fpf_setup(A, FT1 ? A.bt1 : A.bt2, FT1 ? A.bt2 : A.bt1, b0, m0, span, GRAV != 0, (int)(threadIdx.x & 31), PF);
    }
    const double dtd = *A.dt;
    const V dt = vb<V>(S(dtd));
    const V lam = vb<V>(S(dtd / A.h));
    const V lamh = vb<V>(S(dtd / (2.0 * A.h)));
    const V hdt = vb<V>(S(0.5 * dtd));
    const V rtwoh = vb<V>(S(1.0 / (2.0 * A.h)));
    const int n = A.n;

    FMarch<V> M;
    checks_init(M.chk);
    M.cflr = vb<V>(0.0f);
    M.phm2 = vb<V>(0.0f);
    M.ph[0] = M.ph[1] = vb<V>(0.0f);
    M.w0 = M.w1 = M.w2 = M.w3 = M.w4 = typename VT<V>::S(1);
    M.dprev = vb<V>(0.0f);
    fload_mapped<V, GRAV != 0, FT1, IX>(A, X, -3, M.R);
    constexpr int ALL = ST_F1 | ST_PRED | ST_F2 | ST_OUT;
    int r = 3;
    if (n >= 8) {
        fprologue<V, HSE, GRAV, LIM, FT1, CFLF, NU, LD_DIRECT, IX, PFW>(A, X, M, lam, lamh, hdt, dt, rtwoh, PF);
        // steady state: the four steps r .. r+3 prefetch interior cells
#pragma unroll 1
        for (; r + 4 <= n - 1; r += 4) {
            fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 3, ALL, LD_DIRECT_PF, IX, PFW>(A, X, M, r, lam, lamh, hdt, dt, rtwoh, PF);
            fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 0, ALL, LD_DIRECT_PF, IX, PFW>(A, X, M, r + 1, lam, lamh, hdt, dt, rtwoh, PF);
            fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 1, ALL, LD_DIRECT_PF, IX, PFW>(A, X, M, r + 2, lam, lamh, hdt, dt, rtwoh, PF);
            fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 2, ALL, LD_DIRECT_PF, IX, PFW>(A, X, M, r + 3, lam, lamh, hdt, dt, rtwoh, PF);
        }
    } else {
        fprologue<V, HSE, GRAV, LIM, FT1, CFLF, NU, LD_MAPPED, IX, PFW>(A, X, M, lam, lamh, hdt, dt, rtwoh, PF);
    }
    // tail: raw cells r .. n+2 (r = 3 mod 4, at most seven), loads through
    // the map (harmless beyond n+2)
    if (r <= n + 2) fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 3, ALL, LD_MAPPED, IX, PFW>(A, X, M, r, lam, lamh, hdt, dt, rtwoh, PF);
    if (r + 1 <= n + 2) fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 0, ALL, LD_MAPPED, IX, PFW>(A, X, M, r + 1, lam, lamh, hdt, dt, rtwoh, PF);
    if (r + 2 <= n + 2) fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 1, ALL, LD_MAPPED, IX, PFW>(A, X, M, r + 2, lam, lamh, hdt, dt, rtwoh, PF);
    if (r + 3 <= n + 2) fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 2, ALL, LD_MAPPED, IX, PFW>(A, X, M, r + 3, lam, lamh, hdt, dt, rtwoh, PF);
    if (r + 4 <= n + 2) fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 3, ALL, LD_MAPPED, IX, PFW>(A, X, M, r + 4, lam, lamh, hdt, dt, rtwoh, PF);
    if (r + 5 <= n + 2) fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 0, ALL, LD_MAPPED, IX, PFW>(A, X, M, r + 5, lam, lamh, hdt, dt, rtwoh, PF);
    if (r + 6 <= n + 2) fstep<V, HSE, GRAV, LIM, FT1, CFLF, NU, 1, ALL, LD_NONE, IX, PFW>(A, X, M, r + 6, lam, lamh, hdt, dt, rtwoh, PF);
    const unsigned fl = checks_flags(M.chk);
    if (fl) atomicOr(A.flags, fl);
    if constexpr (CFLF) {
        // warp maximum of the rates (order-preserving bits of non-negative
        // floats), then one atomic minimum of 1/rate per warp
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < VT<V>::W; ++i) m = fmaxf(m, (float)vget(M.cflr, i));
        const unsigned mask = __activemask();
        const unsigned wm = __reduce_max_sync(mask, __float_as_uint(m));
        if ((threadIdx.x & 31) == __ffs(mask) - 1) {
            const float mx = __uint_as_float(wm);
            if (mx > 0.0f && mx == mx) {
                atomicMin(A.cfl_min, (unsigned long long)__double_as_longlong(1.0 / (double)mx));
            } else {
                atomicOr(A.flags, FLAG_NAN);
            }
        }
    }
}

template <class V, bool HSE, int GRAV, int LIM, bool FT1, bool CFLF = false, bool NU = false, class IX = long long>
__global__ void __launch_bounds__(128, VT<V>::F64 ? 1 : (VT<V>::W == 2 || HSE ? FISH_COL_MINB : FISH_COL_MINB1))
    fluid_col_kernel(const ColFluidArgs<typename VT<V>::S> A)
{
    fluid_columns<V, HSE, GRAV, LIM, FT1, CFLF, NU, IX>(A, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// B_d: constrained transport column march (eq0330-eq0364, signs of C-5)
// ---------------------------------------------------------------------------
// Rolling state of one face pencil (windows indexed by cell s mod 4 or 2).
template <class V> struct CFace {
    V vt[4];   // face velocity (eq0361) at s
    V vh[4];   // smoothed velocity (eq0362) at s-1
    V bf[4];   // face field at s
    V w[2];    // cell product v b at s-1
    V f1[2];   // predictor flux at interface (s-2)'
    V wp[4];   // predicted product at s-2
    V f[2];    // corrector flux at interface (s-4)'
};

// Widths along d of cells s, s-1 .. s-5 (irregular mesh).
template <class V> struct CWid {
    V w0, w1, w2, w3, w4, w5;
};

// Edge velocity between cells a and b of a face pencil (eq0364): the mean,
// or with NU the linear interpolation to the interface (reading C-27).
template <class V, bool NU> __device__ __forceinline__ V cedge(V va, V vb_, V wa, V wb)
{
    if constexpr (!NU) return vb<V>(0.5f) * (va + vb_);
    else if constexpr (VT<V>::F64) return (wb * va + wa * vb_) / (wa + wb);
    else return vdiv(vfma(wb, va, wa * vb_), wa + wb);
}

// Advance a face pencil by cell s (K = s mod 4) with face velocity vt and
// field bf.  With OUT, bnew receives the updated face field of cell s-4 and
// f[K & 1] holds the corrector flux at (s-4)'.  NU: irregular mesh along d
// (widths in cw, eq037 and reading C-25/C-27; dt for the per-cell factors).
template <class V, int LIM, int K, bool PRE1, bool PRE2, bool CORR, bool OUT, bool NU = false>
__device__ __forceinline__ void cface(CFace<V> &P, V vt, V bf, V lamh, V lam, V &bnew, int lim,
                                      const CWid<V> &cw = CWid<V>(), V dt = V())
{
    constexpr int k1 = (K + 3) & 3, k2 = (K + 2) & 3, kp = (K + 1) & 3;
    constexpr int e = K & 1, o = (K + 1) & 1;
    // smoothed face velocity at s-1 (eq0362) and the cell product w_{s-1}
    V vh;
    if constexpr (VT<V>::F64) vh = 0.25 * (vt + 2.0 * P.vt[k1] + P.vt[k2]);
    else vh = vb<V>(0.25f) * (vfma(vb<V>(2.0f), P.vt[k1], vt) + P.vt[k2]);
    P.vh[k1] = vh;
    P.w[o] = vh * P.bf[k1];
    if constexpr (PRE1) {
        // first-order upwind flux at (s-2)' (eq0363, edge velocity eq0364;
        // tie v = 0 takes the right cell, reading C-7)
        const V vbar = cedge<V, NU>(P.vh[k2], vh, cw.w2, cw.w1);
        P.f1[e] = vsel_pos(vbar, P.w[e], P.w[o]);
    }
    if constexpr (PRE2) {
        // predictor half step of the face field at s-2
        V bp;
        V lh = lamh;
        if constexpr (NU) {
            if constexpr (VT<V>::F64) lh = dt / (2.0 * cw.w2);
            else lh = vdiv(vb<V>(0.5f) * dt, cw.w2);
        }
        if constexpr (VT<V>::F64) bp = P.bf[k2] - lh * (P.f1[e] - P.f1[o]);
        else bp = vfma(-lh, P.f1[e] - P.f1[o], P.bf[k2]);
        P.wp[k2] = P.vh[k2] * bp;
    }
    if constexpr (CORR) {
        // corrector flux at q' = (s-4)': piecewise-linear TVD about the
        // upwind cell (reading C-10)
        const V vbar = cedge<V, NU>(P.vh[K], P.vh[kp], cw.w4, cw.w3);
        const V wm = P.wp[k1], w0 = P.wp[K], w1 = P.wp[kp], w2 = P.wp[k2];
        if constexpr (NU) {
            // slopes per unit length over the centre distances, carried over
            // half the upwind cell (reading C-25)
            const V half = vb<V>(0.5f);
            const V gl = half * (cw.w5 + cw.w4), gc = half * (cw.w4 + cw.w3), gr = half * (cw.w3 + cw.w2);
            if constexpr (VT<V>::F64) {
                P.f[e] = vbar > 0.0 ? w0 + 0.5 * cw.w4 * vlimit<LIM>((w0 - wm) / gl, (w1 - w0) / gc, lim)
                                    : w1 - 0.5 * cw.w3 * vlimit<LIM>((w1 - w0) / gc, (w2 - w1) / gr, lim);
            } else {
                const V d0 = vdiv(w0 - wm, gl), d1 = vdiv(w1 - w0, gc), d2 = vdiv(w2 - w1, gr);
                const V la = vsel_pos(vbar, d0, d1);
                const V lb = vsel_pos(vbar, d1, d2);
                const V base = vsel_pos(vbar, w0, w1);
                const V sg = vsel_pos(vbar, half * cw.w4, -half * cw.w3);
                P.f[e] = vfma(sg, vlimit<LIM>(la, lb, lim), base);
            }
        } else if constexpr (VT<V>::F64) {
            P.f[e] = vbar > 0.0 ? w0 + 0.5 * vlimit<LIM>(w0 - wm, w1 - w0, lim) : w1 - 0.5 * vlimit<LIM>(w1 - w0, w2 - w1, lim);
        } else {
            // select the upwind operands, then limit once
            const V d0 = w0 - wm, d1 = w1 - w0, d2 = w2 - w1;
            const V la = vsel_pos(vbar, d0, d1);
            const V lb = vsel_pos(vbar, d1, d2);
            const V base = vsel_pos(vbar, w0, w1);
            const V sg = vsel_pos(vbar, vb<V>(0.5f), vb<V>(-0.5f));
            P.f[e] = vfma(sg, vlimit<LIM>(la, lb, lim), base);
        }
        if constexpr (OUT) {
            V lo = lam;
            if constexpr (NU) {
                if constexpr (VT<V>::F64) lo = dt / cw.w4;
                else lo = vdiv(dt, cw.w4);
            }
            if constexpr (VT<V>::F64) bnew = P.bf[K] - lo * (P.f[e] - P.f[o]);
            else bnew = vfma(-lo, P.f[e] - P.f[o], P.bf[K]);
        }
    }
    P.bf[K] = bf;
    P.vt[K] = vt;
}

// ---------------------------------------------------------------------------
// B_d column march.  A warp owns 31 W consecutive columns of one row of the
// other axis (lanes 1..31) plus a halo lane 0 holding the W columns below:
// every lane marches the face pencils above its columns along the fast axis
// (PF) and along the other axis (PO), and the pencil below along the other
// axis (PO-).  The fast-axis pencil below a column is the PF pencil of the
// lane beneath it, whose edge flux arrives by a warp shuffle.  Raw inputs of
// cell s+1 are loaded while cell s is computed.
// ---------------------------------------------------------------------------
// IX: element index type (int where every index of the launch fits, else
// long long); a load then costs one wide multiply-add for its address.
template <class S, class IX = long long> struct CTCtx {
    IX base;             // element offset of the lane's first column in cell 0
    IX ofp;              // offset to the fast-axis column above the lane's last column
    IX oom, oop;         // offsets to the other-axis rows below / above (mapped)
    bool active;         // lane stores its columns
    bool fixy;           // halo lane at an outflow edge: its upper column is a copy of the lower
    S wfa, wfb;          // irregular mesh: widths of the lane's column and the one above (fast axis)
    S woa, wop, wom;     // widths of the lane's row and the rows above / below (other axis)
};

template <class V> struct CTRaw {
    V rc, mc, ro, mo, rm, mm;   // rho, m_d of the lane's columns in this, the next and the previous row
    typename VT<V>::S rf, mf;   // rho, m_d of the column above the lane's last column
    V bF, bO, bOm;              // fast-axis faces; other-axis faces of this and the previous row
    V bdo;                      // b_d of the output cell s-4
    V w;                        // width along d of cell s (irregular mesh)
};

template <class V> __device__ __forceinline__ void fixy_(V &a, bool f)
{
    if constexpr (VT<V>::W == 2) {
        if (f) a.v.y = a.v.x;
    }
}

// load the raw inputs of cell s (MAPPED: s through the boundary map; OUTLD:
// also b_d of the output cell s-4, which is interior)
template <class V, bool MAPPED, bool OUTLD, bool NU, class IX = long long>
__device__ __forceinline__ void ctload(const ColCTArgs<typename VT<V>::S> &A, const CTCtx<typename VT<V>::S, IX> &X,
                                       int s, CTRaw<V> &R)
{
    const int sm = MAPPED ? gmap(s, A.n, A.bc) : s;
    const IX i = X.base + (IX)sm * (IX)A.sd;
    if constexpr (NU) R.w = A.wd[sm];  // a ghost has the width of its image (reading C-23)
    R.rc = vload<V>(A.rho, i);
    R.mc = vload<V>(A.md, i);
    R.ro = vload<V>(A.rho, i + X.oop);
    R.mo = vload<V>(A.md, i + X.oop);
    R.rm = vload<V>(A.rho, i + X.oom);
    R.mm = vload<V>(A.md, i + X.oom);
    R.rf = __ldg(A.rho + i + X.ofp);
    R.mf = __ldg(A.md + i + X.ofp);
    R.bF = vload<V>(A.bf, i);
    R.bO = vload<V>(A.bo, i);
    R.bOm = vload<V>(A.bo, i + X.oom);
    if constexpr (VT<V>::W == 2) {
        if (X.fixy) {
            fixy_(R.rc, true); fixy_(R.mc, true); fixy_(R.ro, true); fixy_(R.mo, true);
            fixy_(R.rm, true); fixy_(R.mm, true); fixy_(R.bF, true); fixy_(R.bO, true); fixy_(R.bOm, true);
        }
    }
    // (the tail's last step loads one cell past the march: keep its index in range)
    if constexpr (OUTLD) R.bdo = vload<V>(A.bd, X.base + (IX)(MAPPED ? min(s - 4, A.n - 1) : s - 4) * (IX)A.sd);
}

// prefetch into L2 the fields of interior cell i (the neighbour rows too
// with FISH_CT_PF_NEIGH: with the warps of a block on consecutive rows they
// are mostly the own rows of sibling warps)
#ifndef FISH_CT_PF_DIST
#define FISH_CT_PF_DIST 1
#endif
#ifndef FISH_CT_PF_NEIGH
#define FISH_CT_PF_NEIGH 1
#endif
template <class V, class IX = long long>
__device__ __forceinline__ void ctprefetch(const ColCTArgs<typename VT<V>::S> &A,
                                           const CTCtx<typename VT<V>::S, IX> &X, IX i)
{
    pf_l2(A.rho + i);
    pf_l2(A.md + i);
#if FISH_CT_PF_NEIGH
    pf_l2(A.rho + i + X.oom);
    pf_l2(A.md + i + X.oom);
    pf_l2(A.rho + i + X.oop);
    pf_l2(A.md + i + X.oop);
    pf_l2(A.bo + i + X.oom);
#endif
    pf_l2(A.bf + i);
    pf_l2(A.bo + i);
    pf_l2(A.bd + i);
}

// FP32 one-column CT (uniform mesh): the two face pencils above a column,
// along the fast and the other axis, have the same update; they advance
// together as one packed pencil (component x: fast axis, y: other axis),
// so one FP32x2 instruction serves both.
#ifndef FISH_CT_PACK
#define FISH_CT_PACK 1
#endif
template <class V, bool NU> constexpr bool ct_packs() { return FISH_CT_PACK && std::is_same<V, float>::value && !NU; }

template <class V> struct CTMarch {
    CFace<V> PF, PO, POm;   // fast-axis faces above, other-axis faces above / below
    CFace<P2> PFO;          // packed PF (x) and PO (y) of the FP32 one-column march
    CTRaw<V> R;             // raw inputs of the next cell
    CWid<V> cw;             // irregular mesh: widths along d of cells s-1 .. s-5
};

// L2 prefetch of one cell of a warp's march with a single instruction: lane
// l < 30 takes field row l / 3 of the ten the march reads (rho, m_d of this
// row and the rows below / above, b_o of the row below, b_f, b_o, b_d of this
// row) and the (l % 3)-th 128-byte line of the warp's span of that row.
#ifndef FISH_CT_PF_WARP
#define FISH_CT_PF_WARP 0   // measured slower than the per-field prefetch for this march
#endif
template <class S, class IX> struct CTPf {
    const S *p;   // the lane's line in cell 0 (nullptr: lane idle); cell c: p + c * sd
};

template <class S, class IX>
__device__ __forceinline__ void ctpf_setup(const ColCTArgs<S> &A, const CTCtx<S, IX> &X0, int c0, int c1, int lane,
                                           CTPf<S, IX> &P)
{
    P.p = nullptr;
    if (lane >= 30) return;
    const int r = lane / 3;
    // rows 0..5: rho, m_d of this row, the row below, the row above; 6: b_o
    // below; 7, 8, 9: b_f, b_o, b_d of this row (selects, no local array)
    const S *f = r == 6 || r == 8 ? A.bo : (r == 7 ? A.bf : (r == 9 ? A.bd : ((r & 1) ? A.md : A.rho)));
    const IX ro = (r == 2 || r == 3 || r == 6) ? X0.oom : ((r == 4 || r == 5) ? X0.oop : (IX)0);
    const IX r0 = X0.base + ro + (IX)c0;
    const IX line = (r0 & ~(IX)31) + (IX)(32 * (lane % 3));
    if (line <= X0.base + ro + (IX)c1) P.p = f + line;
}

template <class S, class IX>
__device__ __forceinline__ void ctpf_step(const ColCTArgs<S> &A, const CTPf<S, IX> &P, int s)
{
    if (P.p) pf_l2(P.p + (IX)s * (IX)A.sd);
}

template <class V> __device__ __forceinline__ V shfl_up1(V a)
{
    if constexpr (VT<V>::W == 2) return {make_float2(__shfl_up_sync(0xffffffffu, a.v.x, 1),
                                                     __shfl_up_sync(0xffffffffu, a.v.y, 1))};
    else return __shfl_up_sync(0xffffffffu, a, 1);
}

// Load kinds of a CT step (for cell s+1): none, interior, interior with L2
// prefetch, through the map.
enum : int { CL_NONE = 0, CL_DIRECT = 1, CL_DIRECT_PF = 2, CL_MAPPED = 3 };

// One cell s of the CT march (K = s mod 4); the raw inputs of s are in M.R.
// Next loads cell s+1 (kind LD; NOUT: with b_d of cell s-3 for its output).
template <class V, int LIM, bool FT1, bool NU, int K, bool PRE1, bool PRE2, bool CORR, bool OUT, int LD, bool NOUT,
          class IX = long long>
__device__ __forceinline__ void ctstep(const ColCTArgs<typename VT<V>::S> &A, const CTCtx<typename VT<V>::S, IX> &X,
                                       CTMarch<V> &M, int s, V lamh, V lam, V lamf, V lamo, V dt,
                                       const CTPf<typename VT<V>::S, IX> &PF)
{
    // widths of cells s .. s-5 for this step (the width of cell s arrived
    // with its raw inputs)
    if constexpr (NU) {
        M.cw.w5 = M.cw.w4;
        M.cw.w4 = M.cw.w3;
        M.cw.w3 = M.cw.w2;
        M.cw.w2 = M.cw.w1;
        M.cw.w1 = M.cw.w0;
        M.cw.w0 = M.R.w;
    }
    // consume the raw inputs of cell s
    const V vc = vdiv(M.R.mc, M.R.rc);
    const V vop = vdiv(M.R.mo, M.R.ro);
    const V vom = vdiv(M.R.mm, M.R.rm);
    V vfp;
    if constexpr (VT<V>::W == 2) vfp = vshift_hi(vc, __fdividef(M.R.mf, M.R.rf));
    else vfp = vdiv(V(M.R.mf), V(M.R.rf));
    const V bF = M.R.bF, bO = M.R.bO, bOm = M.R.bOm;
    const V bdo = M.R.bdo;
    // load cell s+1
    if constexpr (LD == CL_DIRECT || LD == CL_DIRECT_PF) {
        ctload<V, false, NOUT, NU, IX>(A, X, s + 1, M.R);
        if constexpr (LD == CL_DIRECT_PF) {
            const int pfc = min(s + 1 + FISH_CT_PF_DIST, A.n - 1);
            if constexpr (FISH_CT_PF_WARP) ctpf_step(A, PF, pfc);
            else ctprefetch<V, IX>(A, X, X.base + (IX)pfc * (IX)A.sd);
        }
    } else if constexpr (LD == CL_MAPPED) {
        ctload<V, true, NOUT, NU, IX>(A, X, s + 1, M.R);
    }
    const V half = vb<V>(0.5f);
    // face velocities (eq0361): the mean of the two cells across the face,
    // or on an irregular mesh their linear interpolation to it (reading C-27)
    V vtF, vtO, vtOm;
    if constexpr (!NU) {
        vtF = half * (vc + vfp);
        vtO = half * (vc + vop);
        vtOm = half * (vom + vc);
    } else if constexpr (VT<V>::F64) {
        vtF = (X.wfb * vc + X.wfa * vfp) / (X.wfa + X.wfb);
        vtO = (X.wop * vc + X.woa * vop) / (X.woa + X.wop);
        vtOm = (X.woa * vom + X.wom * vc) / (X.wom + X.woa);
    } else {
        vtF = vdiv(vfma(V(X.wfb), vc, V(X.wfa) * vfp), V(X.wfa + X.wfb));
        vtO = vdiv(vfma(V(X.wop), vc, V(X.woa) * vop), V(X.woa + X.wop));
        vtOm = vdiv(vfma(V(X.woa), vom, V(X.wom) * vc), V(X.wom + X.woa));
    }
    V nF, nO, dummy;
    constexpr bool PK = ct_packs<V, NU>();
    if constexpr (PK) {
        P2 n2;
        cface<P2, LIM, K, PRE1, PRE2, CORR, OUT, false>(M.PFO, P2{make_float2(vtF, vtO)}, P2{make_float2(bF, bO)},
                                                        vb<P2>(lamh), vb<P2>(lam), n2, A.lim);
        nF = n2.v.x;
        nO = n2.v.y;
    } else {
        cface<V, LIM, K, PRE1, PRE2, CORR, OUT, NU>(M.PF, vtF, bF, lamh, lam, nF, A.lim, M.cw, dt);
        cface<V, LIM, K, PRE1, PRE2, CORR, OUT, NU>(M.PO, vtO, bO, lamh, lam, nO, A.lim, M.cw, dt);
    }
    cface<V, LIM, K, PRE1, PRE2, CORR, false, NU>(M.POm, vtOm, bOm, lamh, lam, dummy, A.lim, M.cw, dt);
    if constexpr (OUT) {
        constexpr int e = K & 1;
        // edge flux of the fast-axis face below: the upper pencil of the lane beneath
        V fup, fpo;
        if constexpr (PK) {
            fup = M.PFO.f[e].v.x;
            fpo = M.PFO.f[e].v.y;
        } else {
            fup = M.PF.f[e];
            fpo = M.PO.f[e];
        }
        const V sh = shfl_up1(fup);
        V fdn;
        if constexpr (VT<V>::W == 2) fdn = vshift_lo(sh.v.y, fup);
        else fdn = sh;
        if (X.active) {
            const IX io = X.base + (IX)(s - 4) * (IX)A.sd;
            vstore(A.bfo, io, nF);
            vstore(A.boo, io, nO);
            const V tF = fup - fdn, tO = fpo - M.POm.f[e];
            V r;
            if constexpr (VT<V>::F64) {
                if constexpr (FT1) r = bdo + lamf * tF + lamo * tO;
                else r = bdo + lamo * tO + lamf * tF;
            } else {
                r = vfma(lamo, tO, vfma(lamf, tF, bdo));
            }
            vstore(A.bdo, io, r);
        }
    }
}

#ifndef FISH_CT_MINB
#define FISH_CT_MINB 4
#endif
#ifndef FISH_CT_MINB2
#define FISH_CT_MINB2 1   // FP64 and two-column CT blocks per SM (register bound)
#endif

// B_d over all columns (eq0350 advection of the transverse components,
// eq0360 constraint update of b_d from the same edge fluxes).  Every lane of
// a warp takes the same steps (shuffles); lanes without columns of their
// own repeat a valid column and store nothing.
// The march of warp gw (31 W columns of one row) of the box described by A.
template <class V, int LIM, bool FT1, bool NU = false, class IX = long long>
__device__ __forceinline__ void ct_columns(const ColCTArgs<typename VT<V>::S> &A, long long gw, int lane)
{
    using S = typename VT<V>::S;
    constexpr int W = VT<V>::W;
    constexpr int SEGC = 31 * W;  // output columns per warp
    const int nseg = (A.nf + SEGC - 1) / SEGC;
    if (gw >= (long long)nseg * A.no) return;  // whole warps only
    const int seg = (int)(gw % nseg), ob = (int)(gw / nseg);
    int cl = seg * SEGC + (lane - 1) * W;       // first logical column of the lane
    CTCtx<S, IX> X;
    X.active = lane >= 1 && cl < A.nf;
    if (lane >= 1 && cl >= A.nf) cl = A.nf - W;  // idle lane: repeat a valid column
    int cb;                                      // physical first column
    X.fixy = false;
    if (cl >= 0) {
        cb = cl;
    } else if (A.bc == BC_PERIODIC) {
        cb = cl + A.nf;
    } else {
        cb = 0;
        X.fixy = W == 2;
    }
    const int cfp = gmap(cl + W, A.nf, A.bc);
    X.base = (IX)A.off + (IX)cb + (IX)ob * (IX)A.so;
    X.ofp = (IX)(cfp - cb);
    X.oom = (IX)(gmap(ob - 1, A.no, A.bc) - ob) * (IX)A.so;
    X.oop = (IX)(gmap(ob + 1, A.no, A.bc) - ob) * (IX)A.so;
    // per-warp L2 prefetch: the span of physical columns the warp reads
    // (halo column to the column above the last lane's), clipped to the row
    CTPf<S, IX> PFw;
    {
        CTCtx<S, IX> X0 = X;
        X0.base = (IX)A.off + (IX)ob * (IX)A.so;
        const int c0 = max(seg * SEGC - W, 0);
        const int c1 = min(seg * SEGC + SEGC, A.nf - 1);
        ctpf_setup(A, X0, c0, c1, lane, PFw);
    }
    const double dtd = *A.dt;
    const V dtv = vb<V>(S(dtd));
    const V lamh = vb<V>(S(dtd / (2.0 * A.h)));
    const V lam = vb<V>(S(dtd / A.h));
    V lamf = vb<V>(S(dtd / A.hf));
    V lamo = vb<V>(S(dtd / A.ho));
    if constexpr (NU) {
        // irregular mesh: widths of the lane's column and its neighbours (a
        // halo or ghost column has the width of its image), and the
        // constraint factors of b_d over the cell's own transverse widths
        X.wfa = A.wf[cb];
        X.wfb = A.wf[cfp];
        X.woa = A.wo[ob];
        X.wop = A.wo[gmap(ob + 1, A.no, A.bc)];
        X.wom = A.wo[gmap(ob - 1, A.no, A.bc)];
        lamf = vb<V>(S(dtd / (double)X.wfa));
        lamo = vb<V>(S(dtd / (double)X.woa));
    }
    const int n = A.n;
    CTMarch<V> M;
    {
        CFace<V> z;
#pragma unroll
        for (int k = 0; k < 4; ++k) z.vt[k] = z.vh[k] = z.bf[k] = z.wp[k] = vb<V>(0.0f);
        z.w[0] = z.w[1] = z.f1[0] = z.f1[1] = z.f[0] = z.f[1] = vb<V>(0.0f);
        M.PF = M.PO = M.POm = z;
        CFace<P2> z2;
#pragma unroll
        for (int k = 0; k < 4; ++k) z2.vt[k] = z2.vh[k] = z2.bf[k] = z2.wp[k] = vb<P2>(0.0f);
        z2.w[0] = z2.w[1] = z2.f1[0] = z2.f1[1] = z2.f[0] = z2.f[1] = vb<P2>(0.0f);
        M.PFO = z2;
    }
    M.R.bdo = vb<V>(0.0f);
    M.cw.w0 = M.cw.w1 = M.cw.w2 = M.cw.w3 = M.cw.w4 = M.cw.w5 = vb<V>(1.0f);
    ctload<V, true, false, NU, IX>(A, X, -4, M.R);
    // prologue s = -4 .. 3 (stages switch on at -1, 0, 3); cells 0 .. 3 are
    // loaded directly when n >= 4
    ctstep<V, LIM, FT1, NU, 0, false, false, false, false, CL_MAPPED, false, IX>(A, X, M, -4, lamh, lam, lamf, lamo, dtv, PFw);
    ctstep<V, LIM, FT1, NU, 1, false, false, false, false, CL_MAPPED, false, IX>(A, X, M, -3, lamh, lam, lamf, lamo, dtv, PFw);
    ctstep<V, LIM, FT1, NU, 2, false, false, false, false, CL_MAPPED, false, IX>(A, X, M, -2, lamh, lam, lamf, lamo, dtv, PFw);
    int s = 4;
    if (n >= 8) {
        ctstep<V, LIM, FT1, NU, 3, true, false, false, false, CL_DIRECT, false, IX>(A, X, M, -1, lamh, lam, lamf, lamo, dtv, PFw);
        ctstep<V, LIM, FT1, NU, 0, true, true, false, false, CL_DIRECT, false, IX>(A, X, M, 0, lamh, lam, lamf, lamo, dtv, PFw);
        ctstep<V, LIM, FT1, NU, 1, true, true, false, false, CL_DIRECT, false, IX>(A, X, M, 1, lamh, lam, lamf, lamo, dtv, PFw);
        ctstep<V, LIM, FT1, NU, 2, true, true, false, false, CL_DIRECT, false, IX>(A, X, M, 2, lamh, lam, lamf, lamo, dtv, PFw);
        ctstep<V, LIM, FT1, NU, 3, true, true, true, false, CL_DIRECT, true, IX>(A, X, M, 3, lamh, lam, lamf, lamo, dtv, PFw);
        // steady state: the four steps s .. s+3 load interior cells s+1 .. s+4
#pragma unroll 1
        for (; s + 4 <= n - 1; s += 4) {
            ctstep<V, LIM, FT1, NU, 0, true, true, true, true, CL_DIRECT_PF, true, IX>(A, X, M, s, lamh, lam, lamf, lamo, dtv, PFw);
            ctstep<V, LIM, FT1, NU, 1, true, true, true, true, CL_DIRECT_PF, true, IX>(A, X, M, s + 1, lamh, lam, lamf, lamo, dtv, PFw);
            ctstep<V, LIM, FT1, NU, 2, true, true, true, true, CL_DIRECT_PF, true, IX>(A, X, M, s + 2, lamh, lam, lamf, lamo, dtv, PFw);
            ctstep<V, LIM, FT1, NU, 3, true, true, true, true, CL_DIRECT_PF, true, IX>(A, X, M, s + 3, lamh, lam, lamf, lamo, dtv, PFw);
        }
    } else {
        ctstep<V, LIM, FT1, NU, 3, true, false, false, false, CL_MAPPED, false, IX>(A, X, M, -1, lamh, lam, lamf, lamo, dtv, PFw);
        ctstep<V, LIM, FT1, NU, 0, true, true, false, false, CL_MAPPED, false, IX>(A, X, M, 0, lamh, lam, lamf, lamo, dtv, PFw);
        ctstep<V, LIM, FT1, NU, 1, true, true, false, false, CL_MAPPED, false, IX>(A, X, M, 1, lamh, lam, lamf, lamo, dtv, PFw);
        ctstep<V, LIM, FT1, NU, 2, true, true, false, false, CL_MAPPED, false, IX>(A, X, M, 2, lamh, lam, lamf, lamo, dtv, PFw);
        ctstep<V, LIM, FT1, NU, 3, true, true, true, false, CL_MAPPED, true, IX>(A, X, M, 3, lamh, lam, lamf, lamo, dtv, PFw);
    }
    // tail: cells s .. n+3 through the map (n-4 <= s <= n-1 after the loop,
    // s = 0 mod 4: at most eight cells)
    if (s <= n + 3) ctstep<V, LIM, FT1, NU, 0, true, true, true, true, CL_MAPPED, true, IX>(A, X, M, s, lamh, lam, lamf, lamo, dtv, PFw);
    if (s + 1 <= n + 3) ctstep<V, LIM, FT1, NU, 1, true, true, true, true, CL_MAPPED, true, IX>(A, X, M, s + 1, lamh, lam, lamf, lamo, dtv, PFw);
    if (s + 2 <= n + 3) ctstep<V, LIM, FT1, NU, 2, true, true, true, true, CL_MAPPED, true, IX>(A, X, M, s + 2, lamh, lam, lamf, lamo, dtv, PFw);
    if (s + 3 <= n + 3) ctstep<V, LIM, FT1, NU, 3, true, true, true, true, CL_MAPPED, true, IX>(A, X, M, s + 3, lamh, lam, lamf, lamo, dtv, PFw);
    if (s + 4 <= n + 3) ctstep<V, LIM, FT1, NU, 0, true, true, true, true, CL_MAPPED, true, IX>(A, X, M, s + 4, lamh, lam, lamf, lamo, dtv, PFw);
    if (s + 5 <= n + 3) ctstep<V, LIM, FT1, NU, 1, true, true, true, true, CL_MAPPED, true, IX>(A, X, M, s + 5, lamh, lam, lamf, lamo, dtv, PFw);
    if (s + 6 <= n + 3) ctstep<V, LIM, FT1, NU, 2, true, true, true, true, CL_MAPPED, true, IX>(A, X, M, s + 6, lamh, lam, lamf, lamo, dtv, PFw);
    if (s + 7 <= n + 3) ctstep<V, LIM, FT1, NU, 3, true, true, true, true, CL_NONE, false, IX>(A, X, M, s + 7, lamh, lam, lamf, lamo, dtv, PFw);
}

// The warps of a block take the same segment of FISH_CT_ROWS consecutive
// rows of the other axis, so the neighbour-row loads of each warp (rho, m_d
// of rows o-1 and o+1, the other-axis face of row o-1) are mostly the
// own-row loads of its sibling warps, served from L1.  Grid: segments x
// ceil(no/FISH_CT_ROWS).
#ifndef FISH_CT_ROWS
#define FISH_CT_ROWS 8   // rows (warps) per CT block
#endif
template <class V, int LIM, bool FT1, bool NU = false, class IX = long long>
__global__ void __launch_bounds__(32 * FISH_CT_ROWS, (VT<V>::F64 || VT<V>::W == 2) ? FISH_CT_MINB2 : FISH_CT_MINB * 4 / FISH_CT_ROWS)
    ct_col_kernel(const ColCTArgs<typename VT<V>::S> A)
{
    constexpr int SEGC = 31 * VT<V>::W;
    const long long nseg = (A.nf + SEGC - 1) / SEGC;
    const long long seg = blockIdx.x % nseg, ob = (blockIdx.x / nseg) * FISH_CT_ROWS + (threadIdx.x >> 5);
    ct_columns<V, LIM, FT1, NU, IX>(A, ob * nseg + seg, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// launchers (defined in fish_col_impl.cuh, instantiated per lane-vector type
// in their own translation units so they compile in parallel)
// ---------------------------------------------------------------------------
// L_d with the lane-vector type V: hse selects the hydrostatic correction,
// ft1 says whether the fast axis is t1 (FP32 callers always order the frame
// so that it is).  Limiter from A.lim.
template <class V>
cudaError_t col_fluid(const ColFluidArgs<typename VT<V>::S> &A, bool hse, bool ft1, cudaStream_t s);
// B_d with the lane-vector type V.
template <class V> cudaError_t col_ct(const ColCTArgs<typename VT<V>::S> &A, bool ft1, cudaStream_t s);
// L_d fed by a shared-memory ring of bulk copies (fish_ring.cu): FP32 pairs,
// t1 fast, no potential, uniform mesh, Van Leer / minmod / hybrid limiter,
// nf % 4 == 0 and 16-byte aligned rows.  cudaErrorNotSupported where it
// does not apply (the caller then runs the column kernel).
cudaError_t ring_fluid(const ColFluidArgs<float> &A, cudaStream_t s);

}  // namespace fish
