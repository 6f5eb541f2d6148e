// fish_launch.cuh -- definitions of the launchers declared in fish_launch.h.
// Included only by the per-precision translation units.
#pragma once

#include "fish_kernels.cuh"
#include "fish_launch.h"

namespace fish {

static inline unsigned grid_for(long long work, int block)
{
    long long g = (work + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

template <class T>
cudaError_t Launch<T>::fluid(const T *const in[8], T *const out[5], const T *phi, const double *dt,
                             const Geom &g, int d, int lim, bool hse, double gamma, double alpha,
                             double h, unsigned *flags, cudaStream_t s)
{
    FluidArgs<T> A;
    for (int f = 0; f < 8; ++f) A.in[f] = in[f];
    for (int f = 0; f < 5; ++f) A.out[f] = out[f];
    A.phi = phi;
    A.dt = dt;
    A.g = g;
    A.d = d;
    A.lim = lim;
    A.gamma = T(gamma);
    A.gm1 = T(gamma - 1.0);
    A.alpha = T(alpha);
    A.h = h;
    A.flags = flags;
    const long long cols = (long long)g.n[(d + 1) % 3] * g.n[(d + 2) % 3];
    const unsigned grid = grid_for(cols, 128);
    if (hse)
        fluid_sweep_kernel<T, true, true><<<grid, 128, 0, s>>>(A);   // HSE needs the potential
    else if (phi)
        fluid_sweep_kernel<T, false, true><<<grid, 128, 0, s>>>(A);
    else
        fluid_sweep_kernel<T, false, false><<<grid, 128, 0, s>>>(A);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::ct(const T *rho, const T *md, const T *const b[3], T *const bout[3],
                          const double *dt, const Geom &g, int d, int lim, const double h[3],
                          unsigned *flags, cudaStream_t s)
{
    CTArgs<T> A;
    A.rho = rho;
    A.md = md;
    for (int f = 0; f < 3; ++f) {
        A.b[f] = b[f];
        A.bout[f] = bout[f];
        A.h[f] = h[f];
    }
    A.dt = dt;
    A.g = g;
    A.d = d;
    A.lim = lim;
    A.flags = flags;
    const long long cols = (long long)g.n[(d + 1) % 3] * g.n[(d + 2) % 3];
    ct_sweep_kernel<T><<<grid_for(cols, 128), 128, 0, s>>>(A);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::cfl(const T *const in[8], const Geom &g, const double h[3], double gamma,
                           unsigned long long *minbits, unsigned *flags, cudaStream_t s)
{
    CFLArgs<T> A;
    for (int f = 0; f < 8; ++f) A.in[f] = in[f];
    A.g = g;
    for (int f = 0; f < 3; ++f) A.h[f] = h[f];
    A.gamma = T(gamma);
    A.gm1 = T(gamma - 1.0);
    A.minbits = minbits;
    A.flags = flags;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    unsigned grid = grid_for(N, 256);
    if (grid > 152u * 16u) grid = 152u * 16u;
    cfl_kernel<T><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::diag(const T *const in[8], const Geom &g, const double h[3], double *partial,
                            int nblocks, cudaStream_t s)
{
    DiagArgs<T> A;
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
    dim3 grid((nr + 31) / 32, (nc + 31) / 32, nz);
    transpose_kernel<T><<<grid, dim3(32, 8), 0, s>>>(A);
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
