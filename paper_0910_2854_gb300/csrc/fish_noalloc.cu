// fish_noalloc.cu -- fish_diagnostics_noalloc: the conserved totals and
// max |div b| of a device-resident state, computed without allocating any
// memory (declared in include/fish.h).
//
// Some callers cannot let a library call cudaMalloc: host codes that own
// every byte of device memory through their own pool or arena, runtimes
// that forbid allocation inside their time loop (cudaMalloc may synchronise
// the device and its cost is unbounded), or callers that hand the library a
// fixed memory budget.  For them this entry point keeps its scratch -- one
// row of nine partial results per z-plane -- in a fixed file-scope device
// array instead of in memory obtained at run time.
//
// Scratch rules (the array lives on every GPU that loads the library, until
// the process exits):
//   - size: kMaxPlanes rows of 9 doubles (4096 * 9 * 8 B = 288 KiB), so
//     boxes with nz > kMaxPlanes are rejected with FISH_ERR_ARG;
//   - every call shares the array; each call writes every row it later reads
//     (no accumulation), so nothing depends on what a previous call left;
//   - two calls whose kernels overlap on the GPU (different streams, no
//     ordering between them) race on the array and may return wrong
//     results: order them on one stream or synchronise in between;
//   - the device address of the array is looked up on every call
//     (cudaGetSymbolAddress, with the caller's device current), so a device
//     reset between calls, which loads the module anew, is followed; the
//     first call on a device may load the module, so make it outside any
//     stream capture.
#include <cuda_runtime.h>

#include "../../include/fish.h"

namespace {

constexpr int kMaxPlanes = 4096;
constexpr int kThreads = 256;

// per-plane partial results: sums of the 8 fields, then max |div b|
static __device__ __align__(256) double g_plane_partials[kMaxPlanes * 9];

// Device address of g_plane_partials on the current device, looked up on
// every call (cheap once the module is loaded; a cached address would go
// stale if the caller reset the device in between).  Host code must not pass
// the symbol itself to a kernel: on the host it names a stand-in, not device
// memory.
cudaError_t scratch_for_current_device(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_plane_partials);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

__device__ __forceinline__ int wrap_or_clamp(int s, int n, int bc)
{
    if (bc == FISH_BC_PERIODIC) return s < 0 ? s + n : (s >= n ? s - n : s);
    return s < 0 ? 0 : (s >= n ? n - 1 : s);
}

// One block per z-plane k: FP64 sums of the 8 fields over the plane and the
// largest |div b| (eq0341) over its cells whose six faces are stored; the
// block's threads reduce in a fixed tree order, so the row is deterministic.
template <class T>
__global__ void __launch_bounds__(kThreads) plane_diag_kernel(const T *__restrict__ q, int nx, int ny, int nz,
                                                              int bc, double dx, double dy, double dz,
                                                              double *__restrict__ rows)
{
    const int k = blockIdx.x;
    const long long N = (long long)nx * ny * nz;
    const long long plane = (long long)nx * ny;
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double dmax = 0.0;
    const int km = wrap_or_clamp(k - 1, nz, bc);
    const bool skip_k = bc == FISH_BC_OUTFLOW && nz > 1 && k == 0;
    for (long long c = threadIdx.x; c < plane; c += blockDim.x) {
        const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
        const long long idx = (long long)k * plane + c;
#pragma unroll
        for (int f = 0; f < 8; ++f) s[f] += (double)q[f * N + idx];
        const bool skip = skip_k || (bc == FISH_BC_OUTFLOW && ((nx > 1 && i == 0) || (ny > 1 && j == 0)));
        if (!skip) {
            const long long ixm = (long long)k * plane + (long long)j * nx + wrap_or_clamp(i - 1, nx, bc);
            const long long iym = (long long)k * plane + (long long)wrap_or_clamp(j - 1, ny, bc) * nx + i;
            const long long izm = (long long)km * plane + c;
            const double dv = ((double)q[5 * N + idx] - (double)q[5 * N + ixm]) / dx +
                              ((double)q[6 * N + idx] - (double)q[6 * N + iym]) / dy +
                              ((double)q[7 * N + idx] - (double)q[7 * N + izm]) / dz;
            dmax = fmax(dmax, fabs(dv));
        }
    }
    __shared__ double red[kThreads][9];
#pragma unroll
    for (int f = 0; f < 8; ++f) red[threadIdx.x][f] = s[f];
    red[threadIdx.x][8] = dmax;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int f = 0; f < 8; ++f) red[threadIdx.x][f] += red[threadIdx.x + w][f];
            red[threadIdx.x][8] = fmax(red[threadIdx.x][8], red[threadIdx.x + w][8]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 9) rows[(long long)k * 9 + threadIdx.x] = red[0][threadIdx.x];
}

// Nine threads: thread f adds column f of the nz rows in plane order (or
// takes the maximum for f = 8) and writes the result to the caller's out[f].
__global__ void plane_finish_kernel(const double *__restrict__ rows, int nz, double vol, double *__restrict__ out)
{
    const int f = threadIdx.x;
    if (f >= 9) return;
    double acc = 0.0;
    for (int k = 0; k < nz; ++k) {
        const double v = rows[(long long)k * 9 + f];
        acc = f < 8 ? acc + v : fmax(acc, v);
    }
    out[f] = f < 8 ? acc * vol : acc;
}

}  // namespace

extern "C" int fish_diagnostics_noalloc(const void *state, int dtype, int nx, int ny, int nz, int bc, double dx,
                                        double dy, double dz, double *out, void *stream)
{
    if (!state || !out) return FISH_ERR_ARG;
    if (dtype != FISH_F64 && dtype != FISH_F32) return FISH_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || (bc != FISH_BC_PERIODIC && bc != FISH_BC_OUTFLOW)) return FISH_ERR_ARG;
    if (nz > kMaxPlanes) return FISH_ERR_ARG;  // scratch holds kMaxPlanes rows
    if ((long long)nx * ny * nz > (1ll << 33)) return FISH_ERR_ARG;
    if (!(dx > 0.0) || !(dy > 0.0) || !(dz > 0.0)) return FISH_ERR_ARG;
    double *rows = nullptr;
    cudaError_t e = scratch_for_current_device(&rows);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return FISH_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == FISH_F64)
        plane_diag_kernel<double><<<nz, kThreads, 0, s>>>(static_cast<const double *>(state), nx, ny, nz, bc,
                                                          dx, dy, dz, rows);
    else
        plane_diag_kernel<float><<<nz, kThreads, 0, s>>>(static_cast<const float *>(state), nx, ny, nz, bc,
                                                         dx, dy, dz, rows);
    plane_finish_kernel<<<1, 32, 0, s>>>(rows, nz, dx * dy * dz, out);
    e = cudaGetLastError();
    return e == cudaSuccess ? FISH_OK : FISH_ERR_CUDA;
}
