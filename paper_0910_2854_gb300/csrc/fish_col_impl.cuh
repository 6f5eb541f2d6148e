// fish_col_impl.cuh -- launchers of the column-march kernels for one
// lane-vector type; included by the translation unit that instantiates them.
#pragma once

#include <type_traits>

#include "fish_column.cuh"

namespace fish {

static inline unsigned col_grid(long long work, int block)
{
    long long g = (work + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

// Whether every element index of a sweep over the box of A fits in an int
// (with margin for the prefetch lines past the last column).
template <class A_> static bool fits_int(const A_ &A)
{
#ifdef FISH_NO_I32
    (void)A;
    return false;
#else
    return A.off + (long long)A.nf * A.no * A.n + 1024 < (1ll << 31);
#endif
}

// blocks of fluid_col_kernel: one thread per column group
template <class V> static unsigned fluid_blocks(const ColFluidArgs<typename VT<V>::S> &A)
{
    return col_grid((long long)(A.nf / VT<V>::W) * A.no, 128);
}

// (external linkage: the packed instantiations are spread over several
// translation units that compile in parallel)
template <class V, bool HSE, int GRAV, int LIM, bool FT1, bool NU = false>
cudaError_t col_fluid_launch(const ColFluidArgs<typename VT<V>::S> &A, cudaStream_t s)
{
    if constexpr (NU) {
        if (A.cfl_min) return cudaErrorInvalidValue;
        fluid_col_kernel<V, HSE, GRAV, LIM, FT1, false, true><<<fluid_blocks<V>(A), 128, 0, s>>>(A);
        return cudaGetLastError();
    }
    // the packed FP32 kernels index with int where the box allows it
    constexpr bool I32 = std::is_same<V, P2>::value;
    const bool small = I32 && fits_int(A);
    if constexpr (std::is_same<V, P2>::value && !HSE) {
        if (A.cfl_min) {
            if (small) fluid_col_kernel<V, HSE, GRAV, LIM, FT1, true, false, int><<<fluid_blocks<V>(A), 128, 0, s>>>(A);
            else fluid_col_kernel<V, HSE, GRAV, LIM, FT1, true><<<fluid_blocks<V>(A), 128, 0, s>>>(A);
            return cudaGetLastError();
        }
    }
    if (A.cfl_min) return cudaErrorInvalidValue;  // only the two-column kernels carry the CFL epilogue
    if constexpr (I32) {
        if (small) {
            fluid_col_kernel<V, HSE, GRAV, LIM, FT1, false, false, int><<<fluid_blocks<V>(A), 128, 0, s>>>(A);
            return cudaGetLastError();
        }
    }
    fluid_col_kernel<V, HSE, GRAV, LIM, FT1><<<fluid_blocks<V>(A), 128, 0, s>>>(A);
    return cudaGetLastError();
}

#ifndef FISH_F64_VL
#define FISH_F64_VL 1   // FP64 sweeps without gravity: compile-time Van Leer limiter
#endif

// GRAV: 0 no potential, 1 unsplit source terms, 2 split kicks in the march
// (uniform meshes; with an irregular mesh the kicks run as separate passes)
template <class V, bool HSE, int GRAV, bool FT1>
static cudaError_t col_fluid_lim(const ColFluidArgs<typename VT<V>::S> &A, cudaStream_t s)
{
    if constexpr (GRAV == 2) {
        if (A.wd) return cudaErrorInvalidValue;
    }
    if constexpr (std::is_same<V, P2>::value) {
        // compile-time limiters for the throughput path (an irregular mesh
        // with Van Leer; its other limiters run on the one-column kernels)
        if constexpr (GRAV != 2) {
            if (A.wd) {
                if (A.lim == LIM_VANLEER) return col_fluid_launch<V, HSE, GRAV, LIM_VANLEER, FT1, true>(A, s);
                return cudaErrorInvalidValue;
            }
        }
        if (A.lim == LIM_VANLEER) return col_fluid_launch<V, HSE, GRAV, LIM_VANLEER, FT1>(A, s);
        if (A.lim == LIM_MINMOD) return col_fluid_launch<V, HSE, GRAV, LIM_MINMOD, FT1>(A, s);
        if (A.lim == LIM_HYBRID) return col_fluid_launch<V, HSE, GRAV, LIM_HYBRID, FT1>(A, s);
        return cudaErrorInvalidValue;
    } else {
        // irregular mesh: widths along d (limiter read at run time)
        if constexpr (GRAV != 2) {
            if (A.wd) return col_fluid_launch<V, HSE, GRAV, -1, FT1, true>(A, s);
        }
        if constexpr (VT<V>::F64 && !HSE && GRAV == 0 && FISH_F64_VL) {
            // the plain FP64 sweeps with a compile-time Van Leer limiter
            if (A.lim == LIM_VANLEER) return col_fluid_launch<V, HSE, GRAV, LIM_VANLEER, FT1>(A, s);
        }
        if constexpr (HSE && std::is_same<V, float>::value) {
            // the hydrostatic sweeps (one column per thread): compile-time
            // limiters (13.2 against 15.4 ms per 384^3 polytrope step with
            // the limiter read per interface)
            if (A.lim == LIM_VANLEER) return col_fluid_launch<V, HSE, GRAV, LIM_VANLEER, FT1>(A, s);
            if (A.lim == LIM_MINMOD) return col_fluid_launch<V, HSE, GRAV, LIM_MINMOD, FT1>(A, s);
        }
        return col_fluid_launch<V, HSE, GRAV, -1, FT1>(A, s);
    }
}

template <class V, bool FT1>
static cudaError_t col_fluid_ft(const ColFluidArgs<typename VT<V>::S> &A, bool hse, cudaStream_t s)
{
    if constexpr (std::is_same<V, P2>::value) {
        if (hse) return cudaErrorInvalidValue;  // the packed kernels carry no hydrostatic terms
        if (A.phi && A.sg) return col_fluid_lim<V, false, 2, FT1>(A, s);
        if (A.phi) return col_fluid_lim<V, false, 1, FT1>(A, s);
        return col_fluid_lim<V, false, 0, FT1>(A, s);
    } else {
        if (hse && A.sg) return cudaErrorInvalidValue;  // split gravity and the correction exclude each other
        if (hse && A.phi) return col_fluid_lim<V, true, 1, FT1>(A, s);
        if (hse) return col_fluid_lim<V, true, 0, FT1>(A, s);  // correction with phi = 0
        if (A.phi && A.sg) return col_fluid_lim<V, false, 2, FT1>(A, s);
        if (A.phi) return col_fluid_lim<V, false, 1, FT1>(A, s);
        return col_fluid_lim<V, false, 0, FT1>(A, s);
    }
}

template <class V>
cudaError_t col_fluid(const ColFluidArgs<typename VT<V>::S> &A, bool hse, bool ft1, cudaStream_t s)
{
    if constexpr (VT<V>::F64) {
        return ft1 ? col_fluid_ft<V, true>(A, hse, s) : col_fluid_ft<V, false>(A, hse, s);
    } else {
        if (!ft1) return cudaErrorInvalidValue;
        return col_fluid_ft<V, true>(A, hse, s);
    }
}

template <class V, int LIM, bool FT1, bool NU = false>
cudaError_t col_ct_launch(const ColCTArgs<typename VT<V>::S> &A, cudaStream_t s)
{
    // one warp per 31 W columns of a row (plus a halo lane); a block takes
    // one segment of FISH_CT_ROWS consecutive rows
    const int segc = 31 * VT<V>::W;
    const long long blocks = (long long)((A.nf + segc - 1) / segc) * ((A.no + FISH_CT_ROWS - 1) / FISH_CT_ROWS);
    // (64-bit indices: int indices measured slower for this march)
    ct_col_kernel<V, LIM, FT1, NU><<<(unsigned)blocks, 32 * FISH_CT_ROWS, 0, s>>>(A);
    return cudaGetLastError();
}

template <class V> cudaError_t col_ct(const ColCTArgs<typename VT<V>::S> &A, bool ft1, cudaStream_t s)
{
    const bool nu = A.wd != nullptr;
    if (nu && (!A.wf || !A.wo)) return cudaErrorInvalidValue;
    if constexpr (VT<V>::F64) {
        if (nu) return ft1 ? col_ct_launch<V, -1, true, true>(A, s) : col_ct_launch<V, -1, false, true>(A, s);
        if (FISH_F64_VL && A.lim == LIM_VANLEER)
            return ft1 ? col_ct_launch<V, LIM_VANLEER, true>(A, s) : col_ct_launch<V, LIM_VANLEER, false>(A, s);
        return ft1 ? col_ct_launch<V, -1, true>(A, s) : col_ct_launch<V, -1, false>(A, s);
    } else if constexpr (std::is_same<V, P2>::value) {
        if (nu) return cudaErrorInvalidValue;
        if (A.lim == LIM_VANLEER) return col_ct_launch<V, LIM_VANLEER, true>(A, s);
        if (A.lim == LIM_MINMOD) return col_ct_launch<V, LIM_MINMOD, true>(A, s);
        return cudaErrorInvalidValue;
    } else {
        if (nu) return col_ct_launch<V, -1, true, true>(A, s);
        // FP32: compile-time limiters for the throughput path
        if (A.lim == LIM_VANLEER) return col_ct_launch<V, LIM_VANLEER, true>(A, s);
        if (A.lim == LIM_MINMOD) return col_ct_launch<V, LIM_MINMOD, true>(A, s);
        return col_ct_launch<V, -1, true>(A, s);
    }
}

}  // namespace fish
