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
};

template <class T>
__device__ __forceinline__ void load_cell(const FluidArgs<T> &A, const Column &c, int s, RawCell<T> &r)
{
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const Geom &g = A.g;
    const int cc = gmap(s, g.n[d], g.bc);
    const long long idx = c.base + (long long)cc * g.st[d];
    r.u[0] = __ldg(A.in[0] + idx);
    r.u[1] = __ldg(A.in[1 + d] + idx);
    r.u[2] = __ldg(A.in[1 + t1] + idx);
    r.u[3] = __ldg(A.in[1 + t2] + idx);
    r.u[4] = __ldg(A.in[4] + idx);
    // cell-centred field: mean of the faces c-1/2 and c+1/2 along each axis
    const long long im_d = c.base + (long long)gmap(cc - 1, g.n[d], g.bc) * g.st[d];
    const long long im_1 = idx + (long long)(gmap(c.a - 1, g.n[t1], g.bc) - c.a) * g.st[t1];
    const long long im_2 = idx + (long long)(gmap(c.b - 1, g.n[t2], g.bc) - c.b) * g.st[t2];
    r.bb[0] = T(0.5) * (__ldg(A.in[5 + d] + im_d) + __ldg(A.in[5 + d] + idx));
    r.bb[1] = T(0.5) * (__ldg(A.in[5 + t1] + im_1) + __ldg(A.in[5 + t1] + idx));
    r.bb[2] = T(0.5) * (__ldg(A.in[5 + t2] + im_2) + __ldg(A.in[5 + t2] + idx));
    r.phi = A.phi ? __ldg(A.phi + idx) : T(0);
}

// One thread marches one pencil with the paper's rolling window (Sec. 3):
// raw cell r enters, the predicted state of cell r-1 is formed from the
// first-order fluxes on either side of it, and the corrected state of cell
// r-3 leaves.  Each input is read once; outputs are written once.
template <class T, bool HSE>
__global__ void __launch_bounds__(128) fluid_sweep_kernel(FluidArgs<T> A)
{
    Column col;
    const long long cid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!column_of(A.g, A.d, cid, col)) return;
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int n = A.g.n[d];
    const long long sd = A.g.st[d];
    const bool grav = A.phi != nullptr;
    const double dtd = *A.dt;
    const T dt = T(dtd);
    const T lam = T(dtd / A.h);            // dt / h
    const T lamh = T(dtd / (2.0 * A.h));   // dt / (2 h)
    const T hdt = T(0.5 * dtd);            // dt / 2
    const T twoh = T(2.0 * A.h);
    unsigned flags = 0;

    Cell<T> cprev;          // raw cell r-1
    T bbprev[3];            // its cell-centred field
    T phim2 = 0, phim1 = 0; // potential at r-2, r-1
    T F1prev[5];            // predictor flux at interface (r-2, r-1)
    Cell<T> P0, P1, P2, P3; // predicted cells p-3 .. p (p = r-1)
    T q0 = 0, q1 = 0, q2 = 0, q3 = 0; // potential of the predicted cells
    T F2prev[5];            // corrector flux at interface (o-1, o)

    RawCell<T> nxt;
    load_cell(A, col, -3, nxt);
    for (int r = -3; r <= n + 2; ++r) {
        RawCell<T> cur = nxt;
        if (r < n + 2) load_cell(A, col, r + 1, nxt);   // prefetch
        Cell<T> craw;
        cell_eval<T>(cur.u, cur.bb, A.gamma, A.gm1, craw, flags);
        if (r >= -2) {
            T F1[5];
            flux1<T, HSE>(cprev, craw, phim1, cur.phi, A.alpha, F1);
            if (r >= -1) {
                // predicted half step of cell r-1 (eq0253, source eq0254)
                T up[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) up[k] = cprev.u[k] - lamh * (F1[k] - F1prev[k]);
                if (grav) {
                    const T dphi = (cur.phi - phim2) / twoh;
                    up[1] = up[1] - hdt * cprev.u[0] * dphi;
                    up[4] = up[4] - hdt * cprev.u[1] * dphi;
                }
                Cell<T> cp;
                cell_eval<T>(up, bbprev, A.gamma, A.gm1, cp, flags);
                P0 = P1; P1 = P2; P2 = P3; P3 = cp;
                q0 = q1; q1 = q2; q2 = q3; q3 = phim1;
                if (r >= 2) {
                    // corrector flux at interface (o, o+1), o = r-3 (eq0230)
                    T F2[5];
                    flux2<T, HSE>(A.lim, P0, P1, P2, P3, q0, q1, q2, q3, F2);
                    if (r >= 3) {
                        const int o = r - 3;
                        const long long io = col.base + (long long)o * sd;
                        T un[5];
                        un[0] = __ldg(A.in[0] + io);
                        un[1] = __ldg(A.in[1 + d] + io);
                        un[2] = __ldg(A.in[1 + t1] + io);
                        un[3] = __ldg(A.in[1 + t2] + io);
                        un[4] = __ldg(A.in[4] + io);
#pragma unroll
                        for (int k = 0; k < 5; ++k) un[k] = un[k] - lam * (F2[k] - F2prev[k]);
                        if (grav) {
                            // corrector source from the predicted state (eq0255)
                            const T dphi = (q2 - q0) / twoh;
                            un[1] = un[1] - dt * P1.u[0] * dphi;
                            un[4] = un[4] - dt * P1.u[1] * dphi;
                        }
                        A.out[0][io] = un[0];
                        A.out[1 + d][io] = un[1];
                        A.out[1 + t1][io] = un[2];
                        A.out[1 + t2][io] = un[3];
                        A.out[4][io] = un[4];
                    }
#pragma unroll
                    for (int k = 0; k < 5; ++k) F2prev[k] = F2[k];
                }
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) F1prev[k] = F1[k];
        }
        cprev = craw;
        bbprev[0] = cur.bb[0]; bbprev[1] = cur.bb[1]; bbprev[2] = cur.bb[2];
        phim2 = phim1;
        phim1 = cur.phi;
    }
    if (flags) atomicOr(A.flags, flags);
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

// Rolling state of one face pencil (face velocity, predictor, corrector).
// At entry of face_step for the new cell s the members hold:
//   vt1, vt2 = face velocity at s-1, s-2
//   vh1, vh2, vh3 = smoothed velocity at s-2, s-3, s-4
//   bf1 .. bf4 = face field at s-1 .. s-4 (bf5: at s-5)
//   w2 = cell product at s-2;  f1p = predictor flux at interface (s-3)'
//   wp2, wp3, wp4 = predicted products at s-3, s-4, s-5
template <class T> struct FacePencil {
    T vt1, vt2;
    T vh1, vh2, vh3;
    T bf1, bf2, bf3, bf4, bf5;
    T w2;
    T f1p;
    T wp2, wp3, wp4;
    T fprev;   // corrector flux at (o-1)'
    T fcur;    // corrector flux at o', o = s-4 (valid once s >= 3)
};

// Advance a face pencil by the new cell s (face velocity vt_s, field bf_s).
// On return, for s >= 4: bf5 is the face field at o = s-4, fcur/fprev the
// corrector fluxes at o' and (o-1)'.
template <class T>
__device__ __forceinline__ void face_step(FacePencil<T> &P, int s, T vt, T bf, T lamh, int lim)
{
    // smoothed face velocity at s-1 (eq0361-eq0362) and cell product w_{s-1}
    const T vh = T(0.25) * (vt + T(2) * P.vt1 + P.vt2);
    const T w1 = vh * P.bf1;
    T f1 = 0;
    if (s >= -1) {
        // first-order upwind flux at interface (s-2)' (eq0363 with eq0364)
        const T vbar = T(0.5) * (P.vh1 + vh);
        f1 = vbar > T(0) ? P.w2 : w1;
    }
    T wp = 0;
    if (s >= 0) {
        // predictor half step of the face field at s-2, product w'_{s-2}
        const T bp = P.bf2 - lamh * (f1 - P.f1p);
        wp = P.vh1 * bp;
    }
    if (s >= 3) {
        // corrector flux at q' = (s-4)' from w'_{q-1..q+2}: piecewise-linear
        // TVD about the upwind cell (reading C-10)
        const T vbar = T(0.5) * (P.vh3 + P.vh2);
        T f;
        if (vbar > T(0))
            f = P.wp3 + T(0.5) * limit(lim, P.wp3 - P.wp4, P.wp2 - P.wp3);
        else
            f = P.wp2 - T(0.5) * limit(lim, P.wp2 - P.wp3, wp - P.wp2);
        P.fprev = P.fcur;
        P.fcur = f;
    }
    P.wp4 = P.wp3; P.wp3 = P.wp2; P.wp2 = wp;
    P.f1p = f1;
    P.w2 = w1;
    P.bf5 = P.bf4; P.bf4 = P.bf3; P.bf3 = P.bf2; P.bf2 = P.bf1; P.bf1 = bf;
    P.vh3 = P.vh2; P.vh2 = P.vh1; P.vh1 = vh;
    P.vt2 = P.vt1; P.vt1 = vt;
}

template <class T>
__device__ __forceinline__ T vel(const CTArgs<T> &A, long long i)
{
    return __ldg(A.md + i) / __ldg(A.rho + i);
}

// One thread per output column: it marches the four face pencils that its
// three output faces need (b_t1 at faces a-1/2 and a+1/2, b_t2 at faces
// b-1/2 and b+1/2) and updates b_t1, b_t2 (advection) and b_d (constraint)
// from the same edge fluxes.
template <class T>
__global__ void __launch_bounds__(128) ct_sweep_kernel(CTArgs<T> A)
{
    Column col;
    const long long cid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!column_of(A.g, A.d, cid, col)) return;
    const int d = A.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const Geom &g = A.g;
    const int n = g.n[d];
    const long long sd = g.st[d];
    const double dtd = *A.dt;
    const T lamh = T(dtd / (2.0 * A.h[d]));
    const T lam = T(dtd / A.h[d]);
    const T lam1 = T(dtd / A.h[t1]);
    const T lam2 = T(dtd / A.h[t2]);
    // neighbouring columns (mapped per coordinate)
    const long long oAm = (long long)(gmap(col.a - 1, g.n[t1], g.bc) - col.a) * g.st[t1];
    const long long oAp = (long long)(gmap(col.a + 1, g.n[t1], g.bc) - col.a) * g.st[t1];
    const long long oBm = (long long)(gmap(col.b - 1, g.n[t2], g.bc) - col.b) * g.st[t2];
    const long long oBp = (long long)(gmap(col.b + 1, g.n[t2], g.bc) - col.b) * g.st[t2];

    FacePencil<T> PA = {}, PAm = {}, PB = {}, PBm = {};
    for (int s = -4; s <= n + 3; ++s) {
        const long long i = col.base + (long long)gmap(s, n, g.bc) * sd;
        const T v0 = vel(A, i);
        const T vAm = vel(A, i + oAm), vAp = vel(A, i + oAp);
        const T vBm = vel(A, i + oBm), vBp = vel(A, i + oBp);
        face_step(PA, s, T(0.5) * (v0 + vAp), __ldg(A.b[t1] + i), lamh, A.lim);
        face_step(PAm, s, T(0.5) * (vAm + v0), __ldg(A.b[t1] + i + oAm), lamh, A.lim);
        face_step(PB, s, T(0.5) * (v0 + vBp), __ldg(A.b[t2] + i), lamh, A.lim);
        face_step(PBm, s, T(0.5) * (vBm + v0), __ldg(A.b[t2] + i + oBm), lamh, A.lim);
        if (s >= 4) {
            const int o = s - 4;
            const long long io = col.base + (long long)o * sd;
            A.bout[t1][io] = PA.bf5 - lam * (PA.fcur - PA.fprev);
            A.bout[t2][io] = PB.bf5 - lam * (PB.fcur - PB.fprev);
            A.bout[d][io] = __ldg(A.b[d] + io) + lam1 * (PA.fcur - PAm.fcur) + lam2 * (PB.fcur - PBm.fcur);
        }
    }
}

// ---------------------------------------------------------------------------
// CFL (eq0083-eq0084): min over cells and axes of h_d / (|v_d| + c_F,d)
// ---------------------------------------------------------------------------
template <class T> struct CFLArgs {
    const T *in[8];
    Geom g;
    double h[3];
    T gamma, gm1;
    unsigned long long *minbits;  // order-preserving bits of the positive minimum (double)
    unsigned *flags;
};

template <class T>
__global__ void __launch_bounds__(256) cfl_kernel(CFLArgs<T> A)
{
    const Geom &g = A.g;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    double best = 1e300;
    unsigned flags = 0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % g.n[0]);
        const int j = (int)((idx / g.n[0]) % g.n[1]);
        const int k = (int)(idx / ((long long)g.n[0] * g.n[1]));
        const int cc[3] = {i, j, k};
        T bc[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const long long lo = idx + (long long)(gmap(cc[ax] - 1, g.n[ax], g.bc) - cc[ax]) * g.st[ax];
            bc[ax] = T(0.5) * (__ldg(A.in[5 + ax] + lo) + __ldg(A.in[5 + ax] + idx));
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            T u[5] = {__ldg(A.in[0] + idx), __ldg(A.in[1 + d] + idx), __ldg(A.in[1 + t1] + idx),
                      __ldg(A.in[1 + t2] + idx), __ldg(A.in[4] + idx)};
            T bb[3] = {bc[d], bc[t1], bc[t2]};
            Cell<T> c;
            cell_eval<T>(u, bb, A.gamma, A.gm1, c, flags);
            const double r = A.h[d] / (double)(Real<T>::abs_(c.vn) + c.cf);
            best = r < best ? r : best;
        }
    }
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
#pragma unroll
        for (int f = 0; f < 8; ++f) s[f] += (double)A.in[f][idx];
        const int i = (int)(idx % g.n[0]);
        const int j = (int)((idx / g.n[0]) % g.n[1]);
        const int k = (int)(idx / ((long long)g.n[0] * g.n[1]));
        const int cc[3] = {i, j, k};
        bool skip = false;
        if (g.bc == BC_OUTFLOW)
            for (int ax = 0; ax < 3; ++ax)
                if (g.n[ax] > 1 && cc[ax] == 0) skip = true;
        if (!skip) {
            double dv = 0.0;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const long long lo = idx + (long long)(gmap(cc[ax] - 1, g.n[ax], g.bc) - cc[ax]) * g.st[ax];
                dv += ((double)A.in[5 + ax][idx] - (double)A.in[5 + ax][lo]) / A.h[ax];
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
