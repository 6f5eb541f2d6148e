// fish_launch.cuh -- definitions of the launchers declared in fish_launch.h.
// Included only by the per-precision translation units.
#pragma once

#include "fish_column.cuh"
#include "fish_kernels.cuh"
#include "fish_launch.h"

namespace fish {

static inline unsigned grid_for(long long work, int block)
{
    long long g = (work + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

// Sweep frame of axis d in the layout of g: the fast transverse axis is the
// one with unit stride (it must not be d), the other transverse axis the
// remaining one.
struct Frame {
    int d, t1, t2, fast, other;
    bool ft1;
    long long sd, so;
    int n, nf, no;
};

static inline bool frame_of(const Geom &g, int d, Frame &F)
{
    F.d = d;
    F.t1 = (d + 1) % 3;
    F.t2 = (d + 2) % 3;
    F.fast = g.ord[0];
    if (F.fast == d) return false;
    F.other = F.fast == F.t1 ? F.t2 : F.t1;
    F.ft1 = F.fast == F.t1;
    F.sd = g.st[d];
    F.so = g.st[F.other];
    F.n = g.n[d];
    F.nf = g.n[F.fast];
    F.no = g.n[F.other];
    return true;
}

// The two-column FP32 kernels are used for even fast extents without the
// hydrostatic correction and with the Van Leer, minmod or hybrid limiter.
template <class T> static bool uses_pairs(const Frame &F, int lim, bool hse, bool nu = false)
{
#ifdef FISH_FLUID_SCALAR
    return false;
#else
    if (nu && lim != LIM_VANLEER) return false;
    return sizeof(T) == 4 && F.nf % 2 == 0 && !hse && (lim == LIM_VANLEER || lim == LIM_MINMOD || lim == LIM_HYBRID);
#endif
}

template <class T> bool Launch<T>::fluid_fuses_cfl(const Geom &g, int d, int lim, bool hse)
{
    Frame F;
    return frame_of(g, d, F) && uses_pairs<T>(F, lim, hse);
}

template <class T>
cudaError_t Launch<T>::fluid(const T *const in[8], T *const out[5], const T *phi, const double *dt,
                             const Geom &g, int d, int lim, bool hse, double gamma, double alpha,
                             const double h3[3], unsigned *flags, unsigned long long *cfl_min, cudaStream_t s,
                             const T *const *w3, bool split_gravity, int kernels)
{
    // split gravity: phi drives kicks G_d(dt/2) folded into the march
    // (uniform meshes with a potential, no hydrostatic correction)
    if (split_gravity && (!phi || w3 || hse)) return cudaErrorInvalidValue;
    Frame F;
    if (!frame_of(g, d, F)) return cudaErrorInvalidValue;
    if (w3 && (!w3[0] || !w3[1] || !w3[2])) return cudaErrorInvalidValue;
    if (cfl_min && (w3 || !uses_pairs<T>(F, lim, hse))) return cudaErrorInvalidValue;
    const double h = h3[d];
    ColFluidArgs<T> A;
    // FP32 orders the frame so that t1 is the fast axis (the formulas are
    // symmetric in t1 and t2); FP64 keeps the cyclic frame of the paper's
    // rotation so that every sum is added in the plain order
    const bool swap = sizeof(T) == 4 && !F.ft1;
    const int a1 = swap ? F.t2 : F.t1, a2 = swap ? F.t1 : F.t2;
    const int perm[5] = {0, 1 + d, 1 + a1, 1 + a2, 4};
    for (int k = 0; k < 5; ++k) {
        A.u[k] = in[perm[k]];
        A.uo[k] = out[perm[k]];
    }
    A.bd = in[5 + d];
    A.bt1 = in[5 + a1];
    A.bt2 = in[5 + a2];
    A.phi = phi;
    A.dt = dt;
    A.off = 0;
    A.sd = F.sd;
    A.so = F.so;
    A.n = F.n;
    A.nf = F.nf;
    A.no = F.no;
    A.bc = g.bc;
    A.lim = lim;
    A.gamma = T(gamma);
    A.gm1 = T(gamma - 1.0);
    A.alpha = T(alpha);
    A.h = h;
    A.flags = flags;
    A.cfl_min = cfl_min;
    A.rh[0] = T(1.0 / h3[d]);
    A.rh[1] = T(1.0 / h3[a1]);
    A.rh[2] = T(1.0 / h3[a2]);
    A.wd = w3 ? w3[d] : nullptr;
    A.sg = split_gravity ? 1 : 0;
    if constexpr (sizeof(T) == 8) {
        return col_fluid<double>(A, hse, F.ft1, s);
    } else {
        // two columns per thread (packed FP32x2) when the fast extent is even;
        // the ring-fed march if asked for and it applies
        if (uses_pairs<T>(F, lim, hse, w3 != nullptr)) {
            if (kernels == 1) {
                const cudaError_t e = ring_fluid(A, s);
                if (e != cudaErrorNotSupported) return e;
            }
            return col_fluid<P2>(A, hse, true, s);
        }
        return col_fluid<float>(A, hse, true, s);
    }
}

template <class T>
cudaError_t Launch<T>::ct(const T *rho, const T *md, const T *const b[3], T *const bout[3],
                          const double *dt, const Geom &g, int d, int lim, const double h[3],
                          unsigned *flags, cudaStream_t s, const T *const *w3)
{
    (void)flags;
    Frame F;
    if (!frame_of(g, d, F)) return cudaErrorInvalidValue;
    if (w3 && (!w3[0] || !w3[1] || !w3[2])) return cudaErrorInvalidValue;
    ColCTArgs<T> A;
    A.rho = rho;
    A.md = md;
    A.bd = b[d];
    A.bf = b[F.fast];
    A.bo = b[F.other];
    A.bdo = bout[d];
    A.bfo = bout[F.fast];
    A.boo = bout[F.other];
    A.dt = dt;
    A.off = 0;
    A.sd = F.sd;
    A.so = F.so;
    A.n = F.n;
    A.nf = F.nf;
    A.no = F.no;
    A.bc = g.bc;
    // the hybrid limiter steers the fluid fluxes only; the face fluxes of
    // the constrained transport keep Van Leer (reading C-21)
    if (lim == LIM_HYBRID) lim = LIM_VANLEER;
    A.lim = lim;
    A.h = h[d];
    A.hf = h[F.fast];
    A.ho = h[F.other];
    if (w3) {
        A.wd = w3[d];
        A.wf = w3[F.fast];
        A.wo = w3[F.other];
    }
    if constexpr (sizeof(T) == 8) {
        return col_ct<double>(A, F.ft1, s);
    } else {
#ifdef FISH_CT_PAIRS
        if (!w3 && F.nf % 2 == 0 && lim != LIM_NONE) return col_ct<P2>(A, true, s);
#endif
        return col_ct<float>(A, true, s);
    }
}

template <class T>
cudaError_t Launch<T>::cfl(const T *const in[8], const Geom &g, const double h[3], double gamma,
                           unsigned long long *minbits, unsigned *flags, cudaStream_t s, const T *const *w3,
                           int k0, int nk)
{
    CFLArgs<T> A;
    A.k0 = k0;
    A.nk = nk;
    if (w3)
        for (int a = 0; a < 3; ++a) A.w[a] = w3[a];
    for (int f = 0; f < 8; ++f) A.in[f] = in[f];
    A.g = g;
    for (int f = 0; f < 3; ++f) A.h[f] = h[f];
    A.gamma = T(gamma);
    A.gm1 = T(gamma - 1.0);
    A.minbits = minbits;
    A.flags = flags;
    // one block per row of the fastest axis, at most 8 resident blocks per SM
    const long long rows = (long long)g.n[g.ord[1]] * (nk < 0 ? g.n[g.ord[2]] : nk);
    const unsigned grid = (unsigned)(rows < 1 ? 1 : (rows < 152ll * 8 ? rows : 152ll * 8));
    cfl_kernel<T><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::diag(const T *const in[8], const Geom &g, const double h[3], double *partial,
                            int nblocks, cudaStream_t s, const T *const *w3)
{
    DiagArgs<T> A;
    if (w3)
        for (int a = 0; a < 3; ++a) A.w[a] = w3[a];
    for (int f = 0; f < 8; ++f) A.in[f] = in[f];
    A.g = g;
    for (int f = 0; f < 3; ++f) A.h[f] = h[f];
    A.partial = partial;
    diag_kernel<T><<<nblocks, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::transpose(const T *const src[8], T *const dst[8], int nf, int nr, int nc, int nz,
                                 cudaStream_t s)
{
    TransArgs<T> A;
    for (int f = 0; f < 8; ++f) {
        A.src[f] = f < nf ? src[f] : nullptr;
        A.dst[f] = f < nf ? dst[f] : nullptr;
    }
    A.nf = nf;
    A.nr = nr;
    A.nc = nc;
    A.plane = (long long)nr * nc;
#ifndef FISH_TR_SCALAR
    if constexpr (sizeof(T) == 4) {
        // 16-byte accesses where every row starts 16-byte aligned
        bool al = nr % 4 == 0 && nc % 4 == 0;
        for (int f = 0; f < nf; ++f) al = al && ((uintptr_t)src[f] & 15) == 0 && ((uintptr_t)dst[f] & 15) == 0;
        if (al) {
            dim3 grid4((nr + 63) / 64, (nc + 63) / 64, nz);
            transpose4_kernel<T><<<grid4, 256, 0, s>>>(A);
            return cudaGetLastError();
        }
    }
#endif
    dim3 grid((nr + 31) / 32, (nc + tr_rows<T>() - 1) / tr_rows<T>(), nz);
    transpose_kernel<T><<<grid, dim3(32, 8), 0, s>>>(A);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::gravity(T *const u[5], const T *phi, const double *dt, double frac, const Geom &g, int d,
                               double h, cudaStream_t s, const T *wd)
{
    if (!phi || d < 0 || d > 2 || g.ord[0] == d) return cudaErrorInvalidValue;
    GravArgs<T> A;
    A.rho = u[0];
    A.md = u[1 + d];
    A.E = u[4];
    A.phi = phi;
    A.dt = dt;
    A.frac = frac;
    A.g = g;
    A.d = d;
    A.h = h;
    A.wd = wd;
    const long long rows = (long long)g.n[g.ord[1]] * g.n[g.ord[2]];
    const unsigned grid = (unsigned)(rows < 152ll * 8 ? rows : 152ll * 8);
    gravity_kernel<T><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::from_f64(const double *src, T *dst, long long n, cudaStream_t s)
{
    unsigned g = grid_for(n, 256);
    if (g > 152u * 32u) g = 152u * 32u;
    convert_kernel<double, T><<<g, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::from_f32(const float *src, T *dst, long long n, cudaStream_t s)
{
    unsigned g = grid_for(n, 256);
    if (g > 152u * 32u) g = 152u * 32u;
    convert_kernel<float, T><<<g, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::to_f64(const T *src, double *dst, long long n, cudaStream_t s)
{
    unsigned g = grid_for(n, 256);
    if (g > 152u * 32u) g = 152u * 32u;
    convert_kernel<T, double><<<g, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::to_f32(const T *src, float *dst, long long n, cudaStream_t s)
{
    unsigned g = grid_for(n, 256);
    if (g > 152u * 32u) g = 152u * 32u;
    convert_kernel<T, float><<<g, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace fish
