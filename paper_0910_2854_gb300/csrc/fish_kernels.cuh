// fish_kernels.cuh -- sm_103a kernels around FISH's operator-split sweep
// (Kaeppeli et al., arXiv:0910.2854), templated on the real type: the CFL
// reduction, the diagnostics, the layout change between sweep directions,
// the operator-split gravity and precision conversions.  The sweeps
// themselves (L_d and B_d) are the column marches of fish_column.cuh.
//
// Data layout: structure of arrays; fields rho, m_x, m_y, m_z, E, b_x, b_y,
// b_z, b_x[i,j,k] being the face average at x_{i+1/2} (eq0080-eq0080b), in
// one of two layouts (x fastest, or y fastest for the x sweeps; Geom says
// which).  No ghost cells are stored: the ghost layer of every sweep is an
// index map (periodic wrap or zeroth-order extrapolation).
#pragma once

#include "fish_math.cuh"
#include "fish_types.h"

namespace fish {

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
    int k0 = 0, nk = -1;  // z-planes k0 .. k0+nk-1 only (nk < 0: all)
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
    const int kb = A.nk < 0 ? 0 : A.k0;
    const long long rows = (long long)nm * (A.nk < 0 ? ns : A.nk);
    double best = 1e300;   // min of h_d / (|v_d| + c_F,d)
    float fbest = 0.0f;    // FP32 path: max of (|v_d| + c_F,d) / h_d
    unsigned flags = 0;
    float rh[3];
    for (int d = 0; d < 3; ++d) rh[d] = (float)(1.0 / A.h[d]);
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int m = (int)(row % nm), k = kb + (int)(row / nm);
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

// Tiles of FISH_TR_ROWS source rows x 32 elements: a thread keeps
// FISH_TR_ROWS/8 loads in flight, and the loads of field f+1 are issued
// before field f is stored (two tiles, one barrier per field: a tile is
// rewritten two fields later, after every thread has passed the barrier
// between).
#ifndef FISH_TR_ROWS
#define FISH_TR_ROWS 64
#endif
// tile height: FP64 tiles stay within the 48 KB of static shared memory
// FP32 transpose with 16-byte accesses: tiles of 64 x 64 elements, each
// thread moves four float4 of a field per tile (source rows of 256 bytes
// read whole, destination rows of 256 bytes written whole), the next
// field's float4 loads in flight while the current tile is stored.  Needs
// nr and nc multiples of 4 (16-byte aligned rows).  Grid: ceil(nr/64) x
// ceil(nc/64) x nz, 256 threads.
template <class T>
__global__ void __launch_bounds__(256) transpose4_kernel(TransArgs<T> A)
{
    static_assert(sizeof(T) == 4, "16-byte accesses of four 4-byte elements");
    __shared__ T tile[2][64][65];
    const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
    const long long zoff = (long long)blockIdx.z * A.plane;
    const int t = threadIdx.x;
    const int lr = t >> 4, l4 = (t & 15) * 4;  // row within a 16-row band, first element of the float4
    float4 v[4];
    auto load = [&](const T *src) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = c0 + lr + 16 * k, r = r0 + l4;
            v[k] = (c < A.nc && r < A.nr) ? __ldg(reinterpret_cast<const float4 *>(src + zoff + (long long)c * A.nr + r))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    load(A.src[0]);
#pragma unroll 1
    for (int f = 0; f < A.nf; ++f) {
        const int b = f & 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            T *row = &tile[b][lr + 16 * k][l4];
            row[0] = v[k].x;
            row[1] = v[k].y;
            row[2] = v[k].z;
            row[3] = v[k].w;
        }
        __syncthreads();
        if (f + 1 < A.nf) load(A.src[f + 1]);
        T *__restrict__ dst = A.dst[f] + zoff;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // destination row r0 + lr + 16k holds source column r0 + lr + 16k
            const int rl = lr + 16 * k, r = r0 + rl, c = c0 + l4;
            if (r < A.nr && c < A.nc) {
                float4 o;
                o.x = tile[b][l4 + 0][rl];
                o.y = tile[b][l4 + 1][rl];
                o.z = tile[b][l4 + 2][rl];
                o.w = tile[b][l4 + 3][rl];
                *reinterpret_cast<float4 *>(dst + (long long)r * A.nc + c) = o;
            }
        }
    }
}

template <class T> constexpr int tr_rows() { return sizeof(T) == 8 && FISH_TR_ROWS > 64 ? 64 : FISH_TR_ROWS; }
template <class T>
__global__ void __launch_bounds__(256) transpose_kernel(TransArgs<T> A)
{
    constexpr int TR = tr_rows<T>(), KL = TR / 8;
    __shared__ T tile[2][TR][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * TR;
    const long long zoff = (long long)blockIdx.z * A.plane;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int rl = r0 + tx;
    T v[KL];
#pragma unroll
    for (int k = 0; k < KL; ++k) {
        const int c = c0 + ty + 8 * k;
        v[k] = (rl < A.nr && c < A.nc) ? A.src[0][zoff + (long long)c * A.nr + rl] : T(0);
    }
#pragma unroll 1
    for (int f = 0; f < A.nf; ++f) {
        const int b = f & 1;
#pragma unroll
        for (int k = 0; k < KL; ++k) tile[b][ty + 8 * k][tx] = v[k];
        __syncthreads();
        if (f + 1 < A.nf) {
            const T *__restrict__ src = A.src[f + 1] + zoff;
#pragma unroll
            for (int k = 0; k < KL; ++k) {
                const int c = c0 + ty + 8 * k;
                v[k] = (rl < A.nr && c < A.nc) ? src[(long long)c * A.nr + rl] : T(0);
            }
        }
        T *__restrict__ dst = A.dst[f] + zoff;
#pragma unroll
        for (int k = 0; k < KL; ++k) {
            const int idx = ty + 8 * k;  // destination row r0 + (idx & 31), column block idx >> 5
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
    Geom g;                 // layout; d is not its fastest axis
    int d;
    double h;
    const T *wd = nullptr;  // irregular mesh: cell widths along d (centre span, reading C-26)
};

// One block per row of the fastest memory axis at a time (grid-stride over
// rows): the coordinate along d, the neighbour offsets and the centre span
// are constant along a row, so the per-cell work is the kick alone.
template <class T>
__global__ void __launch_bounds__(256) gravity_kernel(GravArgs<T> A)
{
    const Geom &g = A.g;
    const int f0 = g.ord[0], f1 = g.ord[1], f2 = g.ord[2];
    const int nf = g.n[f0], nm = g.n[f1];
    const long long rows = (long long)nm * g.n[f2];
    const int n = g.n[A.d];
    const double tau = A.frac * *A.dt;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int m = (int)(row % nm), k = (int)(row / nm);
        const long long base = (long long)m * g.st[f1] + (long long)k * g.st[f2];
        const int s = A.d == f1 ? m : k;
        const long long sd = g.st[A.d];
        const long long op = (long long)(gmap(s + 1, n, g.bc) - s) * sd;
        const long long om = (long long)(gmap(s - 1, n, g.bc) - s) * sd;
        if constexpr (sizeof(T) == 8) {
            const double span = A.wd ? 0.5 * A.wd[gmap(s - 1, n, g.bc)] + A.wd[s] + 0.5 * A.wd[gmap(s + 1, n, g.bc)]
                                     : 2.0 * A.h;
            for (int f = threadIdx.x; f < nf; f += blockDim.x) {
                const long long i = base + f;
                const double dphi = (A.phi[i + op] - A.phi[i + om]) / span;
                const double rho = A.rho[i];
                const double mo = A.md[i];
                const double mn = mo - tau * rho * dphi;
                A.md[i] = mn;
                A.E[i] = A.E[i] + 0.5 * (mn * mn - mo * mo) / rho;
            }
        } else {
            // phi_{s+1} - phi_{s-1} = D_s + D_{s-1}; D_{-1} = 0 at an outflow boundary
            const bool lower = s > 0 || g.bc == BC_PERIODIC;
            float rspan;
            if (A.wd) {
                rspan = 1.0f / (0.5f * (float)A.wd[gmap(s - 1, n, g.bc)] + (float)A.wd[s] +
                                0.5f * (float)A.wd[gmap(s + 1, n, g.bc)]);
            } else {
                rspan = (float)(0.5 / A.h);
            }
            const float ftau = (float)tau;
            for (int f = threadIdx.x; f < nf; f += blockDim.x) {
                const long long i = base + f;
                const float dm1 = lower ? A.phi[i + om] : 0.0f;
                const float dphi = (A.phi[i] + dm1) * rspan;
                const float rho = A.rho[i];
                const float mo = A.md[i];
                const float dm = -(ftau * rho) * dphi;
                A.md[i] = mo + dm;
                A.E[i] = A.E[i] + __fdividef(dm * (mo + 0.5f * dm), rho);
            }
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
