// fish_launch.h -- host-side launchers of the sweep kernels for one real type.
// The definitions (and the kernel instantiations) live in fish_f64.cu and
// fish_f32.cu so that each precision is compiled with its own flags.
#pragma once

#include <cuda_runtime.h>

#include "fish_types.h"

namespace fish {

template <class T> struct Launch {
    // L_d: in[8] current state, out[5] fluid fields of the other buffer.
    // With cfl_min, the sweep also reduces the CFL rate of its output state
    // (all three axes, cell widths h3) into *cfl_min (only where
    // fluid_fuses_cfl says so).  kernels: 0 the register-prefetch column
    // marches, 1 the shared-memory ring march where it applies.  w3: nullptr (uniform mesh) or the device
    // arrays of cell widths along x, y, z (irregular mesh, eq037).
    static cudaError_t fluid(const T *const in[8], T *const out[5], const T *phi, const double *dt,
                             const Geom &g, int d, int lim, bool hse, double gamma, double alpha,
                             const double h3[3], unsigned *flags, unsigned long long *cfl_min, cudaStream_t s,
                             const T *const *w3 = nullptr, bool split_gravity = false, int kernels = 0);
    static bool fluid_fuses_cfl(const Geom &g, int d, int lim, bool hse);
    // B_d: rho, m_d of the current state; b[3] current field, bout[3] other.
    static cudaError_t ct(const T *rho, const T *md, const T *const b[3], T *const bout[3],
                          const double *dt, const Geom &g, int d, int lim, const double h[3],
                          unsigned *flags, cudaStream_t s, const T *const *w3 = nullptr);
    // CFL minimum into *minbits (order-preserving bits of a positive double).
    // k0, nk: only the z-planes k0 .. k0+nk-1 (nk < 0: all)
    static cudaError_t cfl(const T *const in[8], const Geom &g, const double h[3], double gamma,
                           unsigned long long *minbits, unsigned *flags, cudaStream_t s,
                           const T *const *w3 = nullptr, int k0 = 0, int nk = -1);
    // Per-block FP64 partial totals and max |div b| into partial[nblocks][9].
    static cudaError_t diag(const T *const in[8], const Geom &g, const double h[3], double *partial,
                            int nblocks, cudaStream_t s, const T *const *w3 = nullptr);
    // per z-plane transpose of the 8 fields: nc rows of nr -> nr rows of nc
    static cudaError_t transpose(const T *const src[8], T *const dst[8], int nf, int nr, int nc, int nz,
                                 cudaStream_t s);
    // G_d(frac * dt) in place on u[5] (operator-split gravity); phi as the
    // fluid sweep of d reads it (FP64 potential, FP32 differences along d)
    static cudaError_t gravity(T *const u[5], const T *phi, const double *dt, double frac, const Geom &g, int d,
                               double h, cudaStream_t s, const T *wd = nullptr);
    static cudaError_t from_f64(const double *src, T *dst, long long n, cudaStream_t s);
    static cudaError_t from_f32(const float *src, T *dst, long long n, cudaStream_t s);
    static cudaError_t to_f64(const T *src, double *dst, long long n, cudaStream_t s);
    static cudaError_t to_f32(const T *src, float *dst, long long n, cudaStream_t s);
};

cudaError_t launch_cfl_finish(unsigned long long *minbits, double k, double *dt, double *dt_copy,
                              cudaStream_t s);
cudaError_t launch_set_scalar(double *p, double v, cudaStream_t s);
// reset a CFL minimum to +infinity before a reduction
cudaError_t launch_reset_min(unsigned long long *minbits, cudaStream_t s);
// FP64 pipe probe: blocks x 256 threads, each 8 x iters fused multiply-adds
cudaError_t launch_dfma_probe(double *out, int blocks, int iters, cudaStream_t s);

}  // namespace fish
