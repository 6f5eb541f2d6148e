// fish_kernels.cuh -- sm_103a kernels of FISH's operator-split sweep
// (Kaeppeli et al., arXiv:0910.2854), templated on the real type.
//
// Data layout: structure of arrays, x fastest, index i + nx*(j + ny*k);
// fields rho, m_x, m_y, m_z, E, b_x, b_y, b_z, b_x[i,j,k] being the face
// average at x_{i+1/2} (eq0080-eq0080b).  No ghost cells are stored: the
// ghost layer of every sweep is an index map (periodic wrap or zeroth-order
// extrapolation), and the paper's data rotation between sweeps (Sec. 3) is
// replaced by strided addressing -- each sweep direction has its own thread
// mapping, with consecutive threads on consecutive x wherever x is
// transverse, so every global access of the y and z sweeps is coalesced.
//
// Every operator reads the current buffers and writes the other ones
// (out-of-place), so no thread ever reads a value another thread writes in
// the same launch.
#pragma once

#include "fish_math.cuh"
#include "fish_types.h"

namespace fish {

// ---------------------------------------------------------------------------
// geometry of one sweep: axis d, transverse t1 = d+1, t2 = d+2 (cyclic)
// ---------------------------------------------------------------------------
struct Column {
    int a, b;          // coordinates along t1, t2
    long long base;    // a*st[t1] + b*st[t2]
};

// Column id -> (a, b).  Consecutive ids walk along x when x is transverse
// (d = y: t2 = x; d = z: t1 = x), along y for d = x.
__device__ __forceinline__ bool column_of(const Geom &g, int d, long long cid, Column &c)
{
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const long long nt1 = g.n[t1], nt2 = g.n[t2];
    if (cid >= nt1 * nt2) return false;
    if (t2 == 0) {
        c.b = (int)(cid % nt2);
        c.a = (int)(cid / nt2);
    } else {
        c.a = (int)(cid % nt1);
        c.b = (int)(cid / nt1);
    }
    c.base = (long long)c.a * g.st[t1] + (long long)c.b * g.st[t2];
    return true;
}

// ---------------------------------------------------------------------------
// L_d: relaxing-TVD fluid sweep (eq0090-eq0240, eq0253-eq0255, eq0321-eq03261)
// ---------------------------------------------------------------------------
template <class T> struct FluidArgs {
    const T *in[8];     // current state, global component order
    T *out[5];          // rho, m_x, m_y, m_z, E (other buffer)
    const T *phi;       // cell-centred potential or nullptr
    const double *dt;   // device time step
    Geom g;
    int d;
    int lim;
    T gamma, gm1, alpha;
    double h;           // cell width along d
    unsigned *flags;
};

// Raw inputs of one cell of the pencil, in the sweep frame.
template <class T> struct RawCell {
    T u[5];
    T bb[3];
    T phi;
    T bd;      // b_d at the cell's own face (the b_d[c-1] of the next cell)
};

// Per-thread constants of one pencil.
template <class T> struct Pencil {
    long long base;      // offset of cell 0 of the pencil
    long long sd;        // stride along the sweep
    long long o1, o2;    // offsets to the t1-1 and t2-1 neighbours (mapped)
    int a, b;
};

// Ghost or any cell: every index through the boundary map.
template <class T>
__device__ __forceinline__ void load_cell_mapped(const FluidArgs<T> &A, const Pencil<T> &P, int s, RawCell<T> &r)
{
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const Geom &g = A.g;
    const int cc = gmap(s, g.n[d], g.bc);
    const long long idx = P.base + (long long)cc * P.sd;
    r.u[0] = __ldg(A.in[0] + idx);
    r.u[1] = __ldg(A.in[1 + d] + idx);
    r.u[2] = __ldg(A.in[1 + t1] + idx);
    r.u[3] = __ldg(A.in[1 + t2] + idx);
    r.u[4] = __ldg(A.in[4] + idx);
    const long long im_d = P.base + (long long)gmap(cc - 1, g.n[d], g.bc) * P.sd;
    r.bd = __ldg(A.in[5 + d] + idx);
    r.bb[0] = T(0.5) * (__ldg(A.in[5 + d] + im_d) + r.bd);
    r.bb[1] = T(0.5) * (__ldg(A.in[5 + t1] + idx + P.o1) + __ldg(A.in[5 + t1] + idx));
    r.bb[2] = T(0.5) * (__ldg(A.in[5 + t2] + idx + P.o2) + __ldg(A.in[5 + t2] + idx));
    r.phi = A.phi ? __ldg(A.phi + idx) : T(0);
}

// Interior cell s (0 <= s < n): one address; b_d at face s-1/2 is the
// previous cell's own face value bd_prev.
template <class T>
__device__ __forceinline__ void load_cell_interior(const FluidArgs<T> &A, const Pencil<T> &P, int s, T bd_prev,
                                                   RawCell<T> &r)
{
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const long long idx = P.base + (long long)s * P.sd;
    r.u[0] = __ldg(A.in[0] + idx);
    r.u[1] = __ldg(A.in[1 + d] + idx);
    r.u[2] = __ldg(A.in[1 + t1] + idx);
    r.u[3] = __ldg(A.in[1 + t2] + idx);
    r.u[4] = __ldg(A.in[4] + idx);
    r.bd = __ldg(A.in[5 + d] + idx);
    r.bb[0] = T(0.5) * (bd_prev + r.bd);
    r.bb[1] = T(0.5) * (__ldg(A.in[5 + t1] + idx + P.o1) + __ldg(A.in[5 + t1] + idx));
    r.bb[2] = T(0.5) * (__ldg(A.in[5 + t2] + idx + P.o2) + __ldg(A.in[5 + t2] + idx));
    r.phi = A.phi ? __ldg(A.phi + idx) : T(0);
}

template <class T>
__device__ __forceinline__ void load_cell(const FluidArgs<T> &A, const Pencil<T> &P, int s, T bd_prev, RawCell<T> &r)
{
    if (s >= 0 && s < A.g.n[A.d])
        load_cell_interior(A, P, s, bd_prev, r);
    else
        load_cell_mapped(A, P, s, r);
}

// March state of one pencil.  The windows are indexed by the cell number
// modulo 4 (predicted cells, their potential) or modulo 2 (raw cells,
// fluxes); the main loop is unrolled by 4 so every index is a compile-time
// constant and the windows rotate without register moves.
template <class T> struct March {
    RawCell<T> R[2];     // raw input of cell r (slot r&1) and the prefetched r+1
    Cell<T> C[2];        // evaluated raw cells r-1, r
    T bbC[2][3];         // their cell-centred field
    T phC[2];            // their potential
    T F1[2][5];          // predictor fluxes at (r-2,r-1), (r-1,r)
    Cell<T> P[4];        // predicted cells r-4 .. r-1
    T q[4];              // their potential
    T F2[2][5];          // corrector fluxes
    T phm2;              // potential of raw cell r-2
    unsigned flags;
};

// One cell of the march: raw cell r enters, predicted cell r-1 is formed,
// corrected cell o = r-3 leaves (the paper's pipelined loop, Sec. 3).
// K = r mod 4.
template <class T, bool HSE, bool GRAV, int K>
__device__ __forceinline__ void march_cell(const FluidArgs<T> &A, const Pencil<T> &Pn, March<T> &M, int r,
                                           T lam, T lamh, T hdt, T dt, T twoh)
{
    constexpr int k2 = K & 1, p2 = (K + 1) & 1;
    const int n = A.g.n[A.d];
    if (r < -3 || r > n + 2) return;
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    // issue the loads early: next raw cell and the old state of the output cell
    if (r < n + 2) load_cell(A, Pn, r + 1, M.R[k2].bd, M.R[p2]);
    const int o = r - 3;
    const long long io = Pn.base + (long long)(o < 0 ? 0 : o) * Pn.sd;
    T un[5];
    if (o >= 0) {
        un[0] = __ldg(A.in[0] + io);
        un[1] = __ldg(A.in[1 + d] + io);
        un[2] = __ldg(A.in[1 + t1] + io);
        un[3] = __ldg(A.in[1 + t2] + io);
        un[4] = __ldg(A.in[4] + io);
    }
    constexpr bool grav = GRAV;
    const RawCell<T> &cur = M.R[k2];
    cell_eval<T>(cur.u, cur.bb, A.gamma, A.gm1, M.C[k2], M.flags);
    M.bbC[k2][0] = cur.bb[0]; M.bbC[k2][1] = cur.bb[1]; M.bbC[k2][2] = cur.bb[2];
    if (GRAV || HSE) M.phC[k2] = cur.phi;
    if (r >= -2) {
        // predictor flux at interface (r-1, r) (eq0140 / eq0324)
        flux1<T, HSE>(M.C[p2], M.C[k2], M.phC[p2], cur.phi, A.alpha, M.F1[k2]);
        if (r >= -1) {
            // predicted half step of cell r-1 (eq0253, source eq0254)
            const Cell<T> &cp = M.C[p2];
            T up[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) up[k] = cp.u[k] - lamh * (M.F1[k2][k] - M.F1[p2][k]);
            if (grav) {
                const T dphi = (cur.phi - M.phm2) / twoh;
                up[1] = up[1] - hdt * cp.u[0] * dphi;
                up[4] = up[4] - hdt * cp.u[1] * dphi;
            }
            constexpr int s3 = (K + 3) & 3;  // slot of cell r-1
            cell_eval<T>(up, M.bbC[p2], A.gamma, A.gm1, M.P[s3], M.flags);
            if (GRAV || HSE) M.q[s3] = M.phC[p2];
            if (r >= 2) {
                // corrector flux at (o, o+1) from predicted cells o-1 .. o+2 (eq0230)
                constexpr int s0 = K & 3, s1 = (K + 1) & 3, s2 = (K + 2) & 3;
                flux2<T, HSE>(A.lim, M.P[s0], M.P[s1], M.P[s2], M.P[s3], M.q[s0], M.q[s1], M.q[s2], M.q[s3],
                              M.F2[k2]);
                if (o >= 0) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) un[k] = un[k] - lam * (M.F2[k2][k] - M.F2[p2][k]);
                    if (grav) {
                        // corrector source from the predicted state (eq0255)
                        const T dphi = (M.q[s2] - M.q[s0]) / twoh;
                        un[1] = un[1] - dt * M.P[s1].u[0] * dphi;
                        un[4] = un[4] - dt * M.P[s1].u[1] * dphi;
                    }
                    A.out[0][io] = un[0];
                    A.out[1 + d][io] = un[1];
                    A.out[1 + t1][io] = un[2];
                    A.out[1 + t2][io] = un[3];
                    A.out[4][io] = un[4];
                }
            }
        }
    }
    if (GRAV) M.phm2 = M.phC[p2];
}

#ifndef FISH_FLUID_MINB
#define FISH_FLUID_MINB 4  // resident 128-thread blocks per SM for the FP32 fluid sweep
#endif

// One thread marches one pencil: each input is read once (plus an L1 re-read
// of the output cell's old state), each output written once.
template <class T, bool HSE, bool GRAV>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? FISH_FLUID_MINB : 1) fluid_sweep_kernel(FluidArgs<T> A)
{
    Column col;
    const long long cid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!column_of(A.g, A.d, cid, col)) return;
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int n = A.g.n[d];
    Pencil<T> Pn;
    Pn.base = col.base;
    Pn.sd = A.g.st[d];
    Pn.a = col.a;
    Pn.b = col.b;
    Pn.o1 = (long long)(gmap(col.a - 1, A.g.n[t1], A.g.bc) - col.a) * A.g.st[t1];
    Pn.o2 = (long long)(gmap(col.b - 1, A.g.n[t2], A.g.bc) - col.b) * A.g.st[t2];
    const double dtd = *A.dt;
    const T dt = T(dtd);
    const T lam = T(dtd / A.h);            // dt / h
    const T lamh = T(dtd / (2.0 * A.h));   // dt / (2 h)
    const T hdt = T(0.5 * dtd);            // dt / 2
    const T twoh = T(2.0 * A.h);

    March<T> M;
    M.flags = 0;
    M.phm2 = T(0);
    M.phC[0] = M.phC[1] = T(0);
    // raw cell -3 goes to slot 1 (-3 mod 4 = 1, odd)
    load_cell_mapped(A, Pn, -3, M.R[1]);
    // cells -3, -2, -1 (slots 1, 2, 3), then the main loop from 0 in steps of 4
    march_cell<T, HSE, GRAV, 1>(A, Pn, M, -3, lam, lamh, hdt, dt, twoh);
    march_cell<T, HSE, GRAV, 2>(A, Pn, M, -2, lam, lamh, hdt, dt, twoh);
    march_cell<T, HSE, GRAV, 3>(A, Pn, M, -1, lam, lamh, hdt, dt, twoh);
#pragma unroll 1
    for (int r = 0; r <= n + 2; r += 4) {
        march_cell<T, HSE, GRAV, 0>(A, Pn, M, r, lam, lamh, hdt, dt, twoh);
        march_cell<T, HSE, GRAV, 1>(A, Pn, M, r + 1, lam, lamh, hdt, dt, twoh);
        march_cell<T, HSE, GRAV, 2>(A, Pn, M, r + 2, lam, lamh, hdt, dt, twoh);
        march_cell<T, HSE, GRAV, 3>(A, Pn, M, r + 3, lam, lamh, hdt, dt, twoh);
    }
    if (M.flags) atomicOr(A.flags, M.flags);
}

// ---------------------------------------------------------------------------
// B_d: constrained transport (eq0330-eq0364, physical signs of reading C-5)
// ---------------------------------------------------------------------------
template <class T> struct CTArgs {
    const T *rho, *md;   // density and momentum along d (unchanged by B_d)
    const T *b[3];       // current field, global component order
    T *bout[3];          // other buffer
    const double *dt;
    Geom g;
    int d;
    int lim;
    double h[3];
    unsigned *flags;
};

// Rolling state of one face pencil: windows indexed by the cell number s
// modulo 4 (or 2), rotated by the x4-unrolled march without moves.
template <class T> struct FaceWin {
    T vt[4];   // face-averaged velocity (eq0361) at s
    T vh[4];   // smoothed velocity (eq0362) at s-1
    T bf[4];   // face field at s
    T w[2];    // cell product v b at s-1
    T f1[2];   // predictor flux at interface (s-2)'
    T wp[4];   // predicted product v b' at s-2
    T f[2];    // corrector flux at interface (s-4)'
};

// Advance a face pencil by cell s (K = s mod 4) with face velocity vt and
// field bf of that cell.  Returns, for s >= 4, the updated face field of
// cell o = s-4 in *bnew (if requested); fcur/fprev give the corrector fluxes
// at o' and (o-1)' for the constraint update.
template <class T, int K>
__device__ __forceinline__ void face_step(FaceWin<T> &P, int s, T vt, T bf, T lamh, T lam, int lim, T *bnew)
{
    constexpr int k1 = (K + 3) & 3, k2 = (K + 2) & 3, kp = (K + 1) & 3;
    constexpr int e = K & 1, o = (K + 1) & 1;
    // smoothed face velocity at s-1 (eq0362) and cell product w_{s-1}
    const T vh = T(0.25) * (vt + T(2) * P.vt[k1] + P.vt[k2]);
    P.vh[k1] = vh;
    P.w[o] = vh * P.bf[k1];
    if (s >= -1) {
        // first-order upwind flux at (s-2)' (eq0363 with the edge velocity eq0364)
        const T vbar = T(0.5) * (P.vh[k2] + vh);
        P.f1[e] = vbar > T(0) ? P.w[e] : P.w[o];
    }
    if (s >= 0) {
        // predictor half step of the face field at s-2
        const T bp = P.bf[k2] - lamh * (P.f1[e] - P.f1[o]);
        P.wp[k2] = P.vh[k2] * bp;
    }
    if (s >= 3) {
        // corrector flux at q' = (s-4)' from w'_{q-1..q+2}: piecewise-linear
        // TVD about the upwind cell (reading C-10)
        const T vbar = T(0.5) * (P.vh[K] + P.vh[kp]);
        const T wm = P.wp[k1], w0 = P.wp[K], w1 = P.wp[kp], w2 = P.wp[k2];
        P.f[e] = vbar > T(0) ? w0 + T(0.5) * limit(lim, w0 - wm, w1 - w0)
                             : w1 - T(0.5) * limit(lim, w1 - w0, w2 - w1);
        if (bnew && s >= 4) *bnew = P.bf[K] - lam * (P.f[e] - P.f[o]);
    }
    P.bf[K] = bf;
    P.vt[K] = vt;
}

// v_d = m_d / rho: IEEE in FP64, fast reciprocal in FP32
template <class T> __device__ __forceinline__ T vel(const CTArgs<T> &A, long long i)
{
    return div_(__ldg(A.md + i), __ldg(A.rho + i));
}

template <class T> struct CTCol {
    long long base, sd, oAm, oAp, oBm, oBp;
    T lamh, lam, lam1, lam2;
};

template <class T, int K>
__device__ __forceinline__ void ct_cell(const CTArgs<T> &A, const CTCol<T> &C, FaceWin<T> &PA, FaceWin<T> &PAm,
                                        FaceWin<T> &PB, FaceWin<T> &PBm, int s)
{
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int n = A.g.n[d];
    if (s > n + 3) return;
    const long long i = C.base + (long long)((s >= 0 && s < n) ? s : gmap(s, n, A.g.bc)) * C.sd;
    const T v0 = vel(A, i);
    const T vAm = vel(A, i + C.oAm), vAp = vel(A, i + C.oAp);
    const T vBm = vel(A, i + C.oBm), vBp = vel(A, i + C.oBp);
    const T bA = __ldg(A.b[t1] + i), bAm = __ldg(A.b[t1] + i + C.oAm);
    const T bB = __ldg(A.b[t2] + i), bBm = __ldg(A.b[t2] + i + C.oBm);
    T nA, nB;
    face_step<T, K>(PA, s, T(0.5) * (v0 + vAp), bA, C.lamh, C.lam, A.lim, &nA);
    face_step<T, K>(PAm, s, T(0.5) * (vAm + v0), bAm, C.lamh, C.lam, A.lim, (T *)nullptr);
    face_step<T, K>(PB, s, T(0.5) * (v0 + vBp), bB, C.lamh, C.lam, A.lim, &nB);
    face_step<T, K>(PBm, s, T(0.5) * (vBm + v0), bBm, C.lamh, C.lam, A.lim, (T *)nullptr);
    if (s >= 4) {
        constexpr int e = K & 1;
        const long long io = C.base + (long long)(s - 4) * C.sd;
        A.bout[t1][io] = nA;
        A.bout[t2][io] = nB;
        A.bout[d][io] = __ldg(A.b[d] + io) + C.lam1 * (PA.f[e] - PAm.f[e]) + C.lam2 * (PB.f[e] - PBm.f[e]);
    }
}

// One thread per output column: it marches the four face pencils its three
// output faces need (b_t1 at faces a-1/2 and a+1/2, b_t2 at faces b-1/2 and
// b+1/2) and updates b_t1, b_t2 (advection, eq0350) and b_d (constraint,
// eq0360) from the same edge fluxes (physical signs, reading C-5).
template <class T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) ct_sweep_kernel(CTArgs<T> A)
{
    Column col;
    const long long cid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!column_of(A.g, A.d, cid, col)) return;
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const Geom &g = A.g;
    const int n = g.n[d];
    const double dtd = *A.dt;
    CTCol<T> C;
    C.base = col.base;
    C.sd = g.st[d];
    C.lamh = T(dtd / (2.0 * A.h[d]));
    C.lam = T(dtd / A.h[d]);
    C.lam1 = T(dtd / A.h[t1]);
    C.lam2 = T(dtd / A.h[t2]);
    C.oAm = (long long)(gmap(col.a - 1, g.n[t1], g.bc) - col.a) * g.st[t1];
    C.oAp = (long long)(gmap(col.a + 1, g.n[t1], g.bc) - col.a) * g.st[t1];
    C.oBm = (long long)(gmap(col.b - 1, g.n[t2], g.bc) - col.b) * g.st[t2];
    C.oBp = (long long)(gmap(col.b + 1, g.n[t2], g.bc) - col.b) * g.st[t2];
    FaceWin<T> PA = {}, PAm = {}, PB = {}, PBm = {};
#pragma unroll 1
    for (int s = -4; s <= n + 3; s += 4) {
        ct_cell<T, 0>(A, C, PA, PAm, PB, PBm, s);
        ct_cell<T, 1>(A, C, PA, PAm, PB, PBm, s + 1);
        ct_cell<T, 2>(A, C, PA, PAm, PB, PBm, s + 2);
        ct_cell<T, 3>(A, C, PA, PAm, PB, PBm, s + 3);
    }
}

// ---------------------------------------------------------------------------
// CFL (eq0083-eq0084): min over cells and axes of h_d / (|v_d| + c_F,d)
// ---------------------------------------------------------------------------
// Coordinates of the element at memory offset idx (axes in memory order).
__device__ __forceinline__ void coords_of(const Geom &g, long long idx, int cc[3])
{
    const int f0 = g.ord[0], f1 = g.ord[1], f2 = g.ord[2];
    cc[f0] = (int)(idx % g.n[f0]);
    const long long r = idx / g.n[f0];
    cc[f1] = (int)(r % g.n[f1]);
    cc[f2] = (int)(r / g.n[f1]);
}

template <class T> struct CFLArgs {
    const T *in[8];
    Geom g;
    double h[3];
    T gamma, gm1;
    unsigned long long *minbits;  // order-preserving bits of the positive minimum (double)
    unsigned *flags;
    const T *w[3] = {nullptr, nullptr, nullptr};  // irregular mesh: cell widths per axis (eq0420)
};

// FP32 signal speeds along the three axes of one cell, sharing the
// primitives: out[d] = (|v_d| + c_F,d) / h_d (reading C-15), compensated
// pressure recovery as in the sweeps.
__device__ __forceinline__ float cfl_rate_f32(const float u[5], const float b[3], float gamma, float gm1,
                                              const float rh[3], unsigned &flags)
{
    const float ri = __fdividef(1.0f, u[0]);
    const float v[3] = {u[1] * ri, u[2] * ri, u[3] * ri};
    const float kin = 0.5f * (u[1] * v[0] + u[2] * v[1] + u[3] * v[2]);
    const float b2[3] = {b[0] * b[0], b[1] * b[1], b[2] * b[2]};
    const float mag = 0.5f * (b2[0] + b2[1] + b2[2]);
    const float p = gas_pressure<float>(gm1, u[4], kin, mag);
    const float a2 = gamma * p * ri;
    float best = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float bn2 = b2[d] * ri;
        const float bt2 = (b2[(d + 1) % 3] + b2[(d + 2) % 3]) * ri;
        const float B2 = bn2 + bt2;
        const float disc = (a2 - B2) * (a2 - B2) + 4.0f * a2 * bt2;
        const float cf = sqrtf(0.5f * (a2 + B2 + sqrtf(disc)));
        best = fmaxf(best, (fabsf(v[d]) + cf) * rh[d]);
        if (cf != cf) flags |= FLAG_NAN;
    }
    if (!(u[0] > 0.0f)) flags |= FLAG_RHO;
    if (!(p > 0.0f)) flags |= FLAG_P;
    return best;
}

// CFL minimum over the box: one block per group of rows along the fastest
// memory axis (no per-cell index division); per-block minimum, then one
// atomic on the order-preserving bits of the positive double.
template <class T>
__global__ void __launch_bounds__(256) cfl_kernel(CFLArgs<T> A)
{
    const Geom &g = A.g;
    const int f0 = g.ord[0], f1 = g.ord[1], f2 = g.ord[2];
    const int nf = g.n[f0], nm = g.n[f1], ns = g.n[f2];
    const long long rows = (long long)nm * ns;
    double best = 1e300;   // min of h_d / (|v_d| + c_F,d)
    float fbest = 0.0f;    // FP32 path: max of (|v_d| + c_F,d) / h_d
    unsigned flags = 0;
    float rh[3];
    for (int d = 0; d < 3; ++d) rh[d] = (float)(1.0 / A.h[d]);
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int m = (int)(row % nm), k = (int)(row / nm);
        const long long rbase = (long long)m * g.st[f1] + (long long)k * g.st[f2];
        const long long om = (long long)(gmap(m - 1, nm, g.bc) - m) * g.st[f1];
        const long long ok = (long long)(gmap(k - 1, ns, g.bc) - k) * g.st[f2];
        if (A.w[0]) {
            // irregular mesh: this row's widths along the two slower axes
            rh[f1] = (float)(1.0 / (double)A.w[f1][m]);
            rh[f2] = (float)(1.0 / (double)A.w[f2][k]);
        }
        for (int f = threadIdx.x; f < nf; f += blockDim.x) {
            const long long idx = rbase + f;
            const long long ofm = (long long)(gmap(f - 1, nf, g.bc) - f);
            int cc[3];
            cc[f0] = f;
            cc[f1] = m;
            cc[f2] = k;
            if (A.w[0]) rh[f0] = (float)(1.0 / (double)A.w[f0][f]);
            T bc[3];
            bc[f0] = T(0.5) * (__ldg(A.in[5 + f0] + idx + ofm) + __ldg(A.in[5 + f0] + idx));
            bc[f1] = T(0.5) * (__ldg(A.in[5 + f1] + idx + om) + __ldg(A.in[5 + f1] + idx));
            bc[f2] = T(0.5) * (__ldg(A.in[5 + f2] + idx + ok) + __ldg(A.in[5 + f2] + idx));
            if constexpr (sizeof(T) == 8) {
                // per axis in the paper's frame, the oracle's operation order
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                    T u[5] = {__ldg(A.in[0] + idx), __ldg(A.in[1 + d] + idx), __ldg(A.in[1 + t1] + idx),
                              __ldg(A.in[1 + t2] + idx), __ldg(A.in[4] + idx)};
                    T bb[3] = {bc[d], bc[t1], bc[t2]};
                    const T sp = signal_speed<T>(u, bb, A.gamma, A.gm1, flags);
                    const T hd = A.w[0] ? A.w[d][cc[d]] : T(A.h[d]);  // eq0420
                    const double r = (double)(hd / sp);
                    best = r < best ? r : best;
                }
            } else {
                const float u[5] = {__ldg(A.in[0] + idx), __ldg(A.in[1] + idx), __ldg(A.in[2] + idx),
                                    __ldg(A.in[3] + idx), __ldg(A.in[4] + idx)};
                const float b[3] = {(float)bc[0], (float)bc[1], (float)bc[2]};
                fbest = fmaxf(fbest, cfl_rate_f32(u, b, (float)A.gamma, (float)A.gm1, rh, flags));
            }
        }
    }
    if constexpr (sizeof(T) == 4) best = fbest > 0.0f ? 1.0 / (double)fbest : 1e300;
    // block minimum, then one atomic on the order-preserving bits
    for (int off = 16; off > 0; off >>= 1) {
        double o = __shfl_xor_sync(0xffffffffu, best, off);
        best = o < best ? o : best;
    }
    __shared__ double wmin[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wmin[wid] = best;
    __syncthreads();
    if (wid == 0) {
        best = lane < (int)(blockDim.x >> 5) ? wmin[lane] : 1e300;
        for (int off = 16; off > 0; off >>= 1) {
            double o = __shfl_xor_sync(0xffffffffu, best, off);
            best = o < best ? o : best;
        }
        if (lane == 0) {
            if (best != best || best <= 0.0) {
                flags |= FLAG_NAN;
            } else {
                atomicMin(A.minbits, (unsigned long long)__double_as_longlong(best));
            }
        }
    }
    if (flags) atomicOr(A.flags, flags);
}

// dt = k * min; resets the minimum for the next reduction.
static __global__ void cfl_finish_kernel(unsigned long long *minbits, double k, double *dt_out, double *dt_copy)
{
    const double m = __longlong_as_double((long long)*minbits);
    const double dt = k * m;
    *dt_out = dt;
    if (dt_copy) *dt_copy = dt;
    *minbits = 0x7FF0000000000000ull;  // +inf
}

static __global__ void set_scalar_kernel(double *p, double v) { *p = v; }

// ---------------------------------------------------------------------------
// diagnostics: per-block FP64 partial sums (fixed order) and max |div b|
// ---------------------------------------------------------------------------
template <class T> struct DiagArgs {
    const T *in[8];
    Geom g;
    double h[3];
    double *partial;  // [gridDim.x][9]
    // irregular mesh: cell widths per axis; the sums are then volume-weighted
    // in the kernel and the divergence takes each cell's own widths
    const T *w[3] = {nullptr, nullptr, nullptr};
};

template <class T>
__global__ void __launch_bounds__(256) diag_kernel(DiagArgs<T> A)
{
    const Geom &g = A.g;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double dmax = 0.0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        int cc[3];
        coords_of(g, idx, cc);
        if (A.w[0]) {
            const double vol = (double)A.w[0][cc[0]] * (double)A.w[1][cc[1]] * (double)A.w[2][cc[2]];
#pragma unroll
            for (int f = 0; f < 8; ++f) s[f] += (double)A.in[f][idx] * vol;
        } else {
#pragma unroll
            for (int f = 0; f < 8; ++f) s[f] += (double)A.in[f][idx];
        }
        bool skip = false;
        if (g.bc == BC_OUTFLOW)
            for (int ax = 0; ax < 3; ++ax)
                if (g.n[ax] > 1 && cc[ax] == 0) skip = true;
        if (!skip) {
            double dv = 0.0;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const long long lo = idx + (long long)(gmap(cc[ax] - 1, g.n[ax], g.bc) - cc[ax]) * g.st[ax];
                const double hx = A.w[0] ? (double)A.w[ax][cc[ax]] : A.h[ax];
                dv += ((double)A.in[5 + ax][idx] - (double)A.in[5 + ax][lo]) / hx;
            }
            dmax = fmax(dmax, fabs(dv));
        }
    }
    __shared__ double red[256][9];
    for (int f = 0; f < 8; ++f) red[threadIdx.x][f] = s[f];
    red[threadIdx.x][8] = dmax;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            for (int f = 0; f < 8; ++f) red[threadIdx.x][f] += red[threadIdx.x + w][f];
            red[threadIdx.x][8] = fmax(red[threadIdx.x][8], red[threadIdx.x + w][8]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 9) A.partial[(long long)blockIdx.x * 9 + threadIdx.x] = red[0][threadIdx.x];
}

// ---------------------------------------------------------------------------
// layout change: per z-plane 2-D transpose of every field between
// [z][y][x] (x fastest) and [z][x][y] (y fastest) -- the paper's data
// rotation between sweeps (Sec. 3) as a tiled shared-memory transpose with
// coalesced reads and writes.  src rows have length nr, there are nc rows.
// ---------------------------------------------------------------------------
template <class T> struct TransArgs {
    const T *src[8];
    T *dst[8];
    int nr, nc;          // source: nc rows of nr elements; destination: nr rows of nc
    int nf;              // number of fields (1..8)
    long long plane;     // elements per z-plane
};

// Tiles of 64 source rows x 32 elements: a thread keeps eight loads in
// flight, and the loads of field f+1 are issued before field f is stored
// (two tiles, one barrier per field: a tile is rewritten two fields later,
// after every thread has passed the barrier between).
template <class T>
__global__ void __launch_bounds__(256) transpose_kernel(TransArgs<T> A)
{
    __shared__ T tile[2][64][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 64;
    const long long zoff = (long long)blockIdx.z * A.plane;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int rl = r0 + tx;
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int c = c0 + ty + 8 * k;
        v[k] = (rl < A.nr && c < A.nc) ? A.src[0][zoff + (long long)c * A.nr + rl] : T(0);
    }
#pragma unroll 1
    for (int f = 0; f < A.nf; ++f) {
        const int b = f & 1;
#pragma unroll
        for (int k = 0; k < 8; ++k) tile[b][ty + 8 * k][tx] = v[k];
        __syncthreads();
        if (f + 1 < A.nf) {
            const T *__restrict__ src = A.src[f + 1] + zoff;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = c0 + ty + 8 * k;
                v[k] = (rl < A.nr && c < A.nc) ? src[(long long)c * A.nr + rl] : T(0);
            }
        }
        T *__restrict__ dst = A.dst[f] + zoff;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int idx = ty + 8 * k;  // 0 .. 63: destination row r0 + (idx & 31), column half idx >> 5
            const int r = r0 + (idx & 31), cl = tx + 32 * (idx >> 5), c = c0 + cl;
            if (r < A.nr && c < A.nc) dst[(long long)r * A.nc + c] = tile[b][cl][idx & 31];
        }
    }
}

// ---------------------------------------------------------------------------
// operator-split gravity G_d(tau) (eq025111-eq02513): in place on the current
// state, m_d -= tau rho dphi/dx_d with the centred potential difference, and
// E changes by the kinetic energy change (reading C-22), tau = frac * dt.
// FP64 reads the cell potential in the current layout; FP32 the differences
// to the next cell along d (formed in FP64), phi_{i+1} - phi_{i-1} = D_i +
// D_{i-1} with D_{-1} = 0 at an outflow boundary.
// ---------------------------------------------------------------------------
template <class T> struct GravArgs {
    const T *rho;
    T *md, *E;
    const T *phi;
    const double *dt;
    double frac;
    long long N, sd;
    int n, bc;
    double h;
    const T *wd = nullptr;  // irregular mesh: cell widths along d (centre span, reading C-26)
};

template <class T>
__global__ void __launch_bounds__(256) gravity_kernel(GravArgs<T> A)
{
    const double tau = A.frac * *A.dt;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.N;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)((i / A.sd) % A.n);
        if constexpr (sizeof(T) == 8) {
            const long long ip = i + (long long)(gmap(s + 1, A.n, A.bc) - s) * A.sd;
            const long long im = i + (long long)(gmap(s - 1, A.n, A.bc) - s) * A.sd;
            const double span = A.wd ? 0.5 * A.wd[gmap(s - 1, A.n, A.bc)] + A.wd[s] + 0.5 * A.wd[gmap(s + 1, A.n, A.bc)]
                                     : 2.0 * A.h;
            const double dphi = (A.phi[ip] - A.phi[im]) / span;
            const double rho = A.rho[i];
            const double mo = A.md[i];
            const double mn = mo - tau * rho * dphi;
            A.md[i] = mn;
            A.E[i] = A.E[i] + 0.5 * (mn * mn - mo * mo) / rho;
        } else {
            float dm1;
            if (s > 0) dm1 = A.phi[i - A.sd];
            else dm1 = A.bc == BC_PERIODIC ? A.phi[i + (long long)(A.n - 1) * A.sd] : 0.0f;
            float dphi;
            if (A.wd) {
                const float span = 0.5f * (float)A.wd[gmap(s - 1, A.n, A.bc)] + (float)A.wd[s] +
                                   0.5f * (float)A.wd[gmap(s + 1, A.n, A.bc)];
                dphi = (A.phi[i] + dm1) / span;
            } else {
                dphi = (A.phi[i] + dm1) * (float)(0.5 / A.h);
            }
            const float rho = A.rho[i];
            const float mo = A.md[i];
            const float dm = -((float)tau * rho) * dphi;
            A.md[i] = mo + dm;
            A.E[i] = A.E[i] + dm * (mo + 0.5f * dm) / rho;
        }
    }
}

// ---------------------------------------------------------------------------
// precision conversion of one field
// ---------------------------------------------------------------------------
template <class S, class D>
__global__ void convert_kernel(const S *__restrict__ src, D *__restrict__ dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (D)src[i];
}

}  // namespace fish
