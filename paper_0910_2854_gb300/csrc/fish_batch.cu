// fish_batch.cu -- many independent boxes of uneven sizes advanced together
// (declared in include/fish.h, fish_batch_*).  FP32 path.
//
// All boxes live in one set of field arrays (box b at element offset off[b],
// x fastest inside the box), so a sweep over the whole batch is one launch
// of the column-march kernels: a persistent grid whose blocks take work items
// (a box and a group of 128 columns, or 4 warps of CT columns) from a device
// counter until the queue is empty.  Each box keeps its own time step on the
// device: the last x sweep of a double step reduces every box's CFL minimum
// and the next replay turns it into that box's dt.  The double step of the
// whole batch -- counter reset, dt update, twelve sweeps and the two layout
// changes -- is one CUDA graph.  The sweep boundary is the kernel boundary,
// so no block ever waits for another.
//
// Tuning (fish_batch_set_option, chosen by the autotuner in
// paper_0910_2854_gb300/autotune.py): the order of the work items, the
// number of column groups per item and the size of the persistent grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "../../include/fish.h"
#include "fish_column.cuh"
#include "fish_launch.h"

namespace fish {

// one box as seen by one sweep direction
struct BatchBox {
    long long off;
    long long sd, so;
    int n, nf, no, bc;
    float gamma, gm1;
    double h, hf, ho;
    float rh[3];
    int box;
};

// a work item: box table entry and the first column group (fluid: thread
// index, CT: warp index) of a run of `groups` groups of 128 threads
struct BatchItem {
    int bb;
    int first;
    int groups;
};

template <int LIM, bool CFLF>
__global__ void __launch_bounds__(128, FISH_COL_MINB)
    fluid_batch_kernel(const ColFluidArgs<float> A, const BatchBox *__restrict__ boxes,
                       const BatchItem *__restrict__ items, int nitems, int *counter, const double *dt,
                       unsigned *flags, unsigned long long *minbits)
{
    // the work item's arguments, set up by thread 0, stay in shared memory:
    // a register copy of the per-box fields spills the march, which holds
    // about 250 registers (10.4 against 10.6 ms per batch step)
    __shared__ ColFluidArgs<float> Ab;
    __shared__ BatchItem I;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            I.groups = 0;
            if (it < nitems) {
                I = items[it];
                const BatchBox B = boxes[I.bb];
                Ab = A;
                Ab.off = B.off;
                Ab.sd = B.sd;
                Ab.so = B.so;
                Ab.n = B.n;
                Ab.nf = B.nf;
                Ab.no = B.no;
                Ab.bc = B.bc;
                Ab.gamma = B.gamma;
                Ab.gm1 = B.gm1;
                Ab.h = B.h;
                Ab.dt = dt + B.box;
                Ab.flags = flags + B.box;
                Ab.cfl_min = CFLF ? minbits + B.box : nullptr;
                Ab.rh[0] = B.rh[0];
                Ab.rh[1] = B.rh[1];
                Ab.rh[2] = B.rh[2];
            }
        }
        __syncthreads();
        const int groups = I.groups;
        if (groups == 0) return;
        const int first = I.first;
        for (int g = 0; g < groups; ++g)
            fluid_columns<P2, false, false, LIM, true, CFLF, false, int, false>(Ab, (long long)first + 128ll * g + threadIdx.x);
    }
}

// ROWS: warps per work-item group, each on one of ROWS consecutive rows of a
// segment (the tile height; blocks of 32 * ROWS threads)
template <int LIM, int ROWS>
__global__ void __launch_bounds__(32 * ROWS, FISH_CT_MINB * 4 / ROWS)
    ct_batch_kernel(const ColCTArgs<float> A, const BatchBox *__restrict__ boxes,
                    const BatchItem *__restrict__ items, int nitems, int *counter, const double *dt)
{
    // the work item's arguments, set up by thread 0 in shared memory and
    // copied to registers by every thread (the CT march, at 128 registers,
    // runs faster with them in registers: 10.4 against 11.0 ms per batch step)
    __shared__ ColCTArgs<float> Abs;
    __shared__ BatchItem I;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            I.groups = 0;
            if (it < nitems) {
                I = items[it];
                const BatchBox B = boxes[I.bb];
                ColCTArgs<float> &Ab = Abs;
                Ab = A;
                Ab.off = B.off;
                Ab.sd = B.sd;
                Ab.so = B.so;
                Ab.n = B.n;
                Ab.nf = B.nf;
                Ab.no = B.no;
                Ab.bc = B.bc;
                Ab.h = B.h;
                Ab.hf = B.hf;
                Ab.ho = B.ho;
                Ab.dt = dt + B.box;
            }
        }
        __syncthreads();
        const int groups = I.groups;
        if (groups == 0) return;
        const int first = I.first;
        const ColCTArgs<float> Ab = Abs;
        // a group of ROWS warps takes one segment of ROWS consecutive rows
        // (neighbour-row loads served from L1, as in the single-box kernel)
        const long long nseg = (Ab.nf + 30) / 31;
        for (int g = 0; g < groups; ++g) {
            const long long q = (long long)first / ROWS + g;
            const long long ob = (q / nseg) * ROWS + (threadIdx.x >> 5);
            ct_columns<float, LIM, true>(Ab, ob * nseg + q % nseg, threadIdx.x & 31);
        }
    }
}

// layout change of every box: per z-plane transposes, blocks enumerated over
// all boxes' tiles (first[b] = first block of box b)
struct BatchTile {
    long long off;
    int nr, nc, nz;
    int tr, tc;         // tiles along rows / columns of a plane
    long long first;    // first block index
};

__global__ void __launch_bounds__(256) transpose_batch_kernel(const float *const *src, float *const *dst,
                                                              const BatchTile *__restrict__ tiles, int nbox)
{
    __shared__ float tile[32][33];
    __shared__ int s_box;
    const long long bid = blockIdx.x + (long long)gridDim.x * blockIdx.y;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int lo = 0, hi = nbox - 1;
        while (lo < hi) {  // last box whose first block <= bid
            const int mid = (lo + hi + 1) >> 1;
            if (tiles[mid].first <= bid) lo = mid;
            else hi = mid - 1;
        }
        s_box = lo;
    }
    __syncthreads();
    const BatchTile T = tiles[s_box];
    const long long t = bid - T.first;
    if (t >= (long long)T.tr * T.tc * T.nz) return;
    const int z = (int)(t / ((long long)T.tr * T.tc));
    const int rem = (int)(t - (long long)z * T.tr * T.tc);
    const int r0 = (rem % T.tr) * 32, c0 = (rem / T.tr) * 32;
    const long long zoff = T.off + (long long)z * T.nr * T.nc;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll 1
    for (int f = 0; f < 8; ++f) {
        const float *__restrict__ sp = src[f] + zoff;
        float *__restrict__ dp = dst[f] + zoff;
#pragma unroll
        for (int k = 0; k < 32; k += 8) {
            const int r = r0 + tx, c = c0 + ty + k;
            if (r < T.nr && c < T.nc) tile[ty + k][tx] = __ldg(sp + (long long)c * T.nr + r);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 32; k += 8) {
            const int c = c0 + tx, r = r0 + ty + k;
            if (r < T.nr && c < T.nc) dp[(long long)r * T.nc + c] = tile[tx][ty + k];
        }
        __syncthreads();
    }
}

// The same with 16-byte accesses on 64 x 64 tiles (the single-box FP32
// transpose's scheme: four float4 per thread and field, the next field's
// loads in flight); every box needs nr, nc and its offset multiples of 4.
__global__ void __launch_bounds__(256) transpose4_batch_kernel(const float *const *src, float *const *dst,
                                                               const BatchTile *__restrict__ tiles, int nbox)
{
    __shared__ float tile[2][64][65];
    __shared__ int s_box;
    const long long bid = blockIdx.x + (long long)gridDim.x * blockIdx.y;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nbox - 1;
        while (lo < hi) {  // last box whose first block <= bid
            const int mid = (lo + hi + 1) >> 1;
            if (tiles[mid].first <= bid) lo = mid;
            else hi = mid - 1;
        }
        s_box = lo;
    }
    __syncthreads();
    const BatchTile T = tiles[s_box];
    const long long tb = bid - T.first;
    if (tb >= (long long)T.tr * T.tc * T.nz) return;  // whole block
    const int z = (int)(tb / ((long long)T.tr * T.tc));
    const int rem = (int)(tb - (long long)z * T.tr * T.tc);
    const int r0 = (rem % T.tr) * 64, c0 = (rem / T.tr) * 64;
    const long long zoff = T.off + (long long)z * T.nr * T.nc;
    const int t = threadIdx.x;
    const int lr = t >> 4, l4 = (t & 15) * 4;
    float4 v[4];
    auto load = [&](const float *sp) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = c0 + lr + 16 * k, r = r0 + l4;
            v[k] = (c < T.nc && r < T.nr) ? __ldg(reinterpret_cast<const float4 *>(sp + zoff + (long long)c * T.nr + r))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    load(src[0]);
#pragma unroll 1
    for (int f = 0; f < 8; ++f) {
        const int b = f & 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float *row = &tile[b][lr + 16 * k][l4];
            row[0] = v[k].x;
            row[1] = v[k].y;
            row[2] = v[k].z;
            row[3] = v[k].w;
        }
        __syncthreads();
        if (f + 1 < 8) load(src[f + 1]);
        float *__restrict__ dp = dst[f] + zoff;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int rl = lr + 16 * k, r = r0 + rl, c = c0 + l4;
            if (r < T.nr && c < T.nc) {
                float4 o;
                o.x = tile[b][l4 + 0][rl];
                o.y = tile[b][l4 + 1][rl];
                o.z = tile[b][l4 + 2][rl];
                o.w = tile[b][l4 + 3][rl];
                *reinterpret_cast<float4 *>(dp + (long long)r * T.nc + c) = o;
            }
        }
    }
}

// dt[b] = k * min[b] for every box; resets the minima
__global__ void batch_finish_kernel(unsigned long long *minbits, int nbox, double k, double *dt, double *dt_last)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const double m = __longlong_as_double((long long)minbits[b]);
    dt[b] = k * m;
    dt_last[b] = k * m;
    minbits[b] = 0x7FF0000000000000ull;
}

__global__ void batch_reset_kernel(unsigned long long *minbits, int nbox)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox) minbits[b] = 0x7FF0000000000000ull;
}

}  // namespace fish

using namespace fish;

namespace {

constexpr int kCounters = 16;  // work-queue counters per double step (12 sweeps used)

}  // namespace

struct fish_batch {
    int nbox = 0;
    std::vector<int> dims;        // 3 per box
    std::vector<double> gamma, h; // h: 3 per box
    std::vector<int> bc;
    std::vector<long long> off;   // element offset of each box
    long long total = 0;
    int lim = FISH_LIM_VANLEER;
    int order = 0;                // 0 box order, 1 longest work first, 2 interleaved
    int groups = 1;               // column groups per work item
    int grid_factor = 1;          // persistent grid = SMs * resident blocks * factor
    int ctrows = 4;               // constrained-transport rows (warps) per work-item group

    cudaStream_t own = nullptr, stream = nullptr;
    float *fl[2][5] = {};
    float *bf[2][3] = {};
    int cu = 0, cb = 0, layout = 0;
    double *dt = nullptr, *dt_last = nullptr;
    unsigned long long *minbits = nullptr;
    unsigned *flags = nullptr;
    int *counters = nullptr;
    BatchBox *boxes[3] = {};      // per sweep direction
    BatchItem *fitems[3] = {}, *citems[3] = {};
    int nfitems[3] = {0, 0, 0}, ncitems[3] = {0, 0, 0};
    BatchTile *ttiles[2] = {};    // layout 0 -> 1 and 1 -> 0 (32 x 32 tiles)
    long long ttotal[2] = {0, 0};
    BatchTile *ttiles4[2] = {};   // the same in 64 x 64 tiles (16-byte accesses)
    long long ttotal4[2] = {0, 0};
    bool t4 = false;              // every box allows the 16-byte transpose
    const float **tsrc = nullptr;  // device tables: per buffer parity, 8 source then 8 destination field pointers
    std::vector<void *> owned;
    bool tables = false;
    bool pending = false;         // minbits hold the CFL minima of the current states
    cudaGraphExec_t gexec = nullptr;
    double gk = -1.0;
    int gparity = -1;
    bool gdirty = true;
    int sms = 0, fluid_blocks = 0, ct_blocks = 0;
    long long launches = 0;
    std::string err;
};

namespace {

int bfail(fish_batch *b, int code, const std::string &m)
{
    if (b) b->err = m;
    return code;
}

int bcuda(fish_batch *b, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return bfail(b, e == cudaErrorMemoryAllocation ? FISH_ERR_OOM : FISH_ERR_CUDA, m);
}

#define FISH_BCK(b, expr, what)                              \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return bcuda(b, e_, what);    \
    } while (0)

void *balloc(fish_batch *b, size_t bytes)
{
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    b->owned.push_back(p);
    return p;
}

// Geometry of box k in layout L (0: x fastest, 1: y fastest)
Geom box_geom(const fish_batch *b, int k, int L)
{
    Geom g;
    const int *n = &b->dims[3 * k];
    for (int a = 0; a < 3; ++a) g.n[a] = n[a];
    if (L == 0) {
        g.st[0] = 1;
        g.st[1] = n[0];
        g.ord[0] = 0;
        g.ord[1] = 1;
    } else {
        g.st[0] = n[1];
        g.st[1] = 1;
        g.ord[0] = 1;
        g.ord[1] = 0;
    }
    g.st[2] = (long long)n[0] * n[1];
    g.ord[2] = 2;
    g.bc = b->bc[k];
    return g;
}

int layout_of(int d) { return d == 0 ? 1 : 0; }

// Box tables and work lists for the current tuning.
int build_tables(fish_batch *b)
{
    for (int d = 0; d < 3; ++d) {
        std::vector<BatchBox> bx(b->nbox);
        std::vector<BatchItem> fi, ci;
        std::vector<std::pair<long long, BatchItem>> fw, cw;  // (work, item)
        for (int k = 0; k < b->nbox; ++k) {
            const Geom g = box_geom(b, k, layout_of(d));
            const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            const int fast = g.ord[0];
            const int other = fast == t1 ? t2 : t1;
            BatchBox &B = bx[k];
            B.off = b->off[k];
            B.sd = g.st[d];
            B.so = g.st[other];
            B.n = g.n[d];
            B.nf = g.n[fast];
            B.no = g.n[other];
            B.bc = g.bc;
            B.gamma = (float)b->gamma[k];
            B.gm1 = (float)(b->gamma[k] - 1.0);
            B.h = b->h[3 * k + d];
            B.hf = b->h[3 * k + fast];
            B.ho = b->h[3 * k + other];
            B.rh[0] = (float)(1.0 / b->h[3 * k + d]);
            B.rh[1] = (float)(1.0 / b->h[3 * k + fast]);
            B.rh[2] = (float)(1.0 / b->h[3 * k + other]);
            B.box = k;
            const long long fcols = (long long)(B.nf / 2) * B.no;          // two columns per thread
            const long long fgroups = (fcols + 127) / 128;
            for (long long g0 = 0; g0 < fgroups; g0 += b->groups) {
                BatchItem I{k, (int)(g0 * 128), (int)std::min<long long>(b->groups, fgroups - g0)};
                fw.push_back({(long long)B.n * I.groups, I});
            }
            // 31 columns per warp; a group is one segment of ctrows rows
            const int R = b->ctrows;
            const long long cgroups = (long long)((B.nf + 30) / 31) * ((B.no + R - 1) / R);
            for (long long g0 = 0; g0 < cgroups; g0 += b->groups) {
                BatchItem I{k, (int)(g0 * R), (int)std::min<long long>(b->groups, cgroups - g0)};
                cw.push_back({(long long)B.n * I.groups, I});
            }
        }
        auto arrange = [&](std::vector<std::pair<long long, BatchItem>> &w, std::vector<BatchItem> &out) {
            if (b->order == 1) {
                std::stable_sort(w.begin(), w.end(),
                                 [](const std::pair<long long, BatchItem> &x, const std::pair<long long, BatchItem> &y) {
                                     return x.first > y.first;
                                 });
                for (auto &p : w) out.push_back(p.second);
            } else if (b->order == 2) {
                // round robin over boxes
                std::vector<std::vector<BatchItem>> per(b->nbox);
                for (auto &p : w) per[p.second.bb].push_back(p.second);
                size_t rounds = 0;
                for (auto &v : per) rounds = std::max(rounds, v.size());
                for (size_t r = 0; r < rounds; ++r)
                    for (auto &v : per)
                        if (r < v.size()) out.push_back(v[r]);
            } else {
                for (auto &p : w) out.push_back(p.second);
            }
        };
        arrange(fw, fi);
        arrange(cw, ci);
        if (!b->boxes[d] && !(b->boxes[d] = (BatchBox *)balloc(b, sizeof(BatchBox) * b->nbox)))
            return bfail(b, FISH_ERR_OOM, "batch table allocation failed");
        // item lists may change length with the tuning: reallocate
        b->fitems[d] = (BatchItem *)balloc(b, sizeof(BatchItem) * fi.size());
        b->citems[d] = (BatchItem *)balloc(b, sizeof(BatchItem) * ci.size());
        if (!b->fitems[d] || !b->citems[d]) return bfail(b, FISH_ERR_OOM, "batch work list allocation failed");
        FISH_BCK(b, cudaMemcpy(b->boxes[d], bx.data(), sizeof(BatchBox) * b->nbox, cudaMemcpyHostToDevice), "tables");
        FISH_BCK(b, cudaMemcpy(b->fitems[d], fi.data(), sizeof(BatchItem) * fi.size(), cudaMemcpyHostToDevice), "tables");
        FISH_BCK(b, cudaMemcpy(b->citems[d], ci.data(), sizeof(BatchItem) * ci.size(), cudaMemcpyHostToDevice), "tables");
        b->nfitems[d] = (int)fi.size();
        b->ncitems[d] = (int)ci.size();
    }
    // transposes: from layout L to 1-L
    for (int L = 0; L < 2; ++L) {
        std::vector<BatchTile> tt(b->nbox);
        long long first = 0;
        for (int k = 0; k < b->nbox; ++k) {
            const int *n = &b->dims[3 * k];
            BatchTile &T = tt[k];
            T.off = b->off[k];
            T.nr = L == 0 ? n[0] : n[1];
            T.nc = L == 0 ? n[1] : n[0];
            T.nz = n[2];
            T.tr = (T.nr + 31) / 32;
            T.tc = (T.nc + 31) / 32;
            T.first = first;
            first += (long long)T.tr * T.tc * T.nz;
        }
        if (!b->ttiles[L] && !(b->ttiles[L] = (BatchTile *)balloc(b, sizeof(BatchTile) * b->nbox)))
            return bfail(b, FISH_ERR_OOM, "batch table allocation failed");
        FISH_BCK(b, cudaMemcpy(b->ttiles[L], tt.data(), sizeof(BatchTile) * b->nbox, cudaMemcpyHostToDevice), "tables");
        b->ttotal[L] = first;
        // 64 x 64 tiles for the 16-byte transpose
        bool ok = true;
        long long first4 = 0;
        for (int k = 0; k < b->nbox; ++k) {
            BatchTile &T = tt[k];
            ok = ok && T.nr % 4 == 0 && T.nc % 4 == 0 && T.off % 4 == 0;
            T.tr = (T.nr + 63) / 64;
            T.tc = (T.nc + 63) / 64;
            T.first = first4;
            first4 += (long long)T.tr * T.tc * T.nz;
        }
        if (!b->ttiles4[L] && !(b->ttiles4[L] = (BatchTile *)balloc(b, sizeof(BatchTile) * b->nbox)))
            return bfail(b, FISH_ERR_OOM, "batch table allocation failed");
        FISH_BCK(b, cudaMemcpy(b->ttiles4[L], tt.data(), sizeof(BatchTile) * b->nbox, cudaMemcpyHostToDevice),
                 "tables");
        b->ttotal4[L] = first4;
#ifdef FISH_TR_SCALAR
        ok = false;
#endif
        b->t4 = (L == 0 ? ok : (b->t4 && ok));
    }
    // field pointer tables of the transposes, one per buffer parity
    for (int cu = 0; cu < 2; ++cu)
        for (int cb = 0; cb < 2; ++cb) {
            const float *tab[16];
            for (int f = 0; f < 5; ++f) {
                tab[f] = b->fl[cu][f];
                tab[8 + f] = b->fl[1 - cu][f];
            }
            for (int f = 0; f < 3; ++f) {
                tab[5 + f] = b->bf[cb][f];
                tab[13 + f] = b->bf[1 - cb][f];
            }
            FISH_BCK(b, cudaMemcpy((void *)(b->tsrc + (cu * 2 + cb) * 16), tab, sizeof(tab), cudaMemcpyHostToDevice),
                     "tables");
        }
    b->tables = true;
    b->gdirty = true;
    return FISH_OK;
}

// ---- operators over the whole batch ----------------------------------------

int batch_transpose(fish_batch *b)
{
    // field pointers of the current and the other buffers (table by parity)
    const float **dsrc = b->tsrc + (b->cu * 2 + b->cb) * 16;
    // (the field arrays come from the allocator, 256-byte aligned)
    if (b->t4) {
        const long long nblk = b->ttotal4[b->layout];
        dim3 grid((unsigned)std::min<long long>(nblk, 1 << 30), (unsigned)((nblk + (1 << 30) - 1) / (1 << 30)));
        transpose4_batch_kernel<<<grid, 256, 0, b->stream>>>(dsrc, (float *const *)(dsrc + 8), b->ttiles4[b->layout],
                                                             b->nbox);
    } else {
        const long long nblk = b->ttotal[b->layout];
        dim3 grid((unsigned)std::min<long long>(nblk, 1 << 30), (unsigned)((nblk + (1 << 30) - 1) / (1 << 30)));
        transpose_batch_kernel<<<grid, dim3(32, 8), 0, b->stream>>>(dsrc, (float *const *)(dsrc + 8),
                                                                    b->ttiles[b->layout], b->nbox);
    }
    FISH_BCK(b, cudaGetLastError(), "batch transpose launch");
    b->cu = 1 - b->cu;
    b->cb = 1 - b->cb;
    b->layout = 1 - b->layout;
    b->launches += 1;
    return FISH_OK;
}

int batch_layout(fish_batch *b, int L) { return b->layout == L ? FISH_OK : batch_transpose(b); }

int batch_fluid(fish_batch *b, int d, bool cfl, int counter)
{
    int r = batch_layout(b, layout_of(d));
    if (r) return r;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    // the fast axis of the d sweep: y for x sweeps (layout 1), x otherwise
    const int fast = d == 0 ? 1 : 0;
    const int a1 = fast, a2 = fast == t1 ? t2 : t1;
    ColFluidArgs<float> A{};
    const int perm[5] = {0, 1 + d, 1 + a1, 1 + a2, 4};
    for (int k = 0; k < 5; ++k) {
        A.u[k] = b->fl[b->cu][perm[k]];
        A.uo[k] = b->fl[1 - b->cu][perm[k]];
    }
    A.bd = b->bf[b->cb][d];
    A.bt1 = b->bf[b->cb][a1];
    A.bt2 = b->bf[b->cb][a2];
    A.phi = nullptr;
    A.lim = b->lim;
    A.alpha = 1.0f;
    const int grid = b->fluid_blocks;
    int *ctr = b->counters + counter;
    if (b->lim == FISH_LIM_VANLEER) {
        if (cfl)
            fluid_batch_kernel<LIM_VANLEER, true><<<grid, 128, 0, b->stream>>>(
                A, b->boxes[d], b->fitems[d], b->nfitems[d], ctr, b->dt, b->flags, b->minbits);
        else
            fluid_batch_kernel<LIM_VANLEER, false><<<grid, 128, 0, b->stream>>>(
                A, b->boxes[d], b->fitems[d], b->nfitems[d], ctr, b->dt, b->flags, b->minbits);
    } else {
        if (cfl)
            fluid_batch_kernel<LIM_MINMOD, true><<<grid, 128, 0, b->stream>>>(
                A, b->boxes[d], b->fitems[d], b->nfitems[d], ctr, b->dt, b->flags, b->minbits);
        else
            fluid_batch_kernel<LIM_MINMOD, false><<<grid, 128, 0, b->stream>>>(
                A, b->boxes[d], b->fitems[d], b->nfitems[d], ctr, b->dt, b->flags, b->minbits);
    }
    FISH_BCK(b, cudaGetLastError(), "batch fluid launch");
    b->cu = 1 - b->cu;
    b->launches += 1;
    return FISH_OK;
}

int batch_ct(fish_batch *b, int d, int counter)
{
    int r = batch_layout(b, layout_of(d));
    if (r) return r;
    const int fast = d == 0 ? 1 : 0;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int other = fast == t1 ? t2 : t1;
    ColCTArgs<float> A{};
    A.rho = b->fl[b->cu][0];
    A.md = b->fl[b->cu][1 + d];
    A.bd = b->bf[b->cb][d];
    A.bf = b->bf[b->cb][fast];
    A.bo = b->bf[b->cb][other];
    A.bdo = b->bf[1 - b->cb][d];
    A.bfo = b->bf[1 - b->cb][fast];
    A.boo = b->bf[1 - b->cb][other];
    A.lim = b->lim;
    int *ctr = b->counters + counter;
    const bool vl = b->lim == FISH_LIM_VANLEER;
    if (b->ctrows == 8) {
        if (vl)
            ct_batch_kernel<LIM_VANLEER, 8><<<b->ct_blocks, 256, 0, b->stream>>>(A, b->boxes[d], b->citems[d],
                                                                               b->ncitems[d], ctr, b->dt);
        else
            ct_batch_kernel<LIM_MINMOD, 8><<<b->ct_blocks, 256, 0, b->stream>>>(A, b->boxes[d], b->citems[d],
                                                                              b->ncitems[d], ctr, b->dt);
    } else {
        if (vl)
            ct_batch_kernel<LIM_VANLEER, 4><<<b->ct_blocks, 128, 0, b->stream>>>(A, b->boxes[d], b->citems[d],
                                                                               b->ncitems[d], ctr, b->dt);
        else
            ct_batch_kernel<LIM_MINMOD, 4><<<b->ct_blocks, 128, 0, b->stream>>>(A, b->boxes[d], b->citems[d],
                                                                              b->ncitems[d], ctr, b->dt);
    }
    FISH_BCK(b, cudaGetLastError(), "batch constrained-transport launch");
    b->cb = 1 - b->cb;
    b->launches += 1;
    return FISH_OK;
}

// CFL minima of every box's current state (one CFL launch per box)
int batch_cfl(fish_batch *b)
{
    batch_reset_kernel<<<(b->nbox + 127) / 128, 128, 0, b->stream>>>(b->minbits, b->nbox);
    FISH_BCK(b, cudaGetLastError(), "batch reset launch");
    b->launches += 1;
    for (int k = 0; k < b->nbox; ++k) {
        const float *in[8];
        for (int f = 0; f < 5; ++f) in[f] = b->fl[b->cu][f] + b->off[k];
        for (int f = 0; f < 3; ++f) in[5 + f] = b->bf[b->cb][f] + b->off[k];
        const double hk[3] = {b->h[3 * k], b->h[3 * k + 1], b->h[3 * k + 2]};
        FISH_BCK(b, Launch<float>::cfl(in, box_geom(b, k, b->layout), hk, b->gamma[k], b->minbits + k,
                                       b->flags + k, b->stream),
                 "batch cfl launch");
        b->launches += 1;
    }
    return FISH_OK;
}

// one double step of every box: dt from the minima, twelve sweeps in the
// order of reading C-4, the last one reducing the next minima
int batch_queue_step(fish_batch *b, double k)
{
    FISH_BCK(b, cudaMemsetAsync(b->counters, 0, sizeof(int) * kCounters, b->stream), "counters");
    batch_finish_kernel<<<(b->nbox + 127) / 128, 128, 0, b->stream>>>(b->minbits, b->nbox, k, b->dt, b->dt_last);
    FISH_BCK(b, cudaGetLastError(), "batch finish launch");
    b->launches += 1;
    int r, c = 0;
    for (int d = 0; d < 3; ++d) {
        if ((r = batch_fluid(b, d, false, c++))) return r;
        if ((r = batch_ct(b, d, c++))) return r;
    }
    for (int d = 2; d >= 0; --d) {
        if ((r = batch_ct(b, d, c++))) return r;
        if ((r = batch_fluid(b, d, d == 0, c++))) return r;
    }
    return FISH_OK;
}

int batch_ready(fish_batch *b)
{
    if (!b) return FISH_ERR_ARG;
    if (!b->tables) {
        int r = build_tables(b);
        if (r) return r;
    }
    return FISH_OK;
}

int batch_flags(fish_batch *b)
{
    std::vector<unsigned> fl(b->nbox);
    FISH_BCK(b, cudaMemcpyAsync(fl.data(), b->flags, sizeof(unsigned) * b->nbox, cudaMemcpyDeviceToHost, b->stream),
             "flags");
    FISH_BCK(b, cudaStreamSynchronize(b->stream), "sync");
    for (int k = 0; k < b->nbox; ++k)
        if (fl[k]) {
            char buf[128];
            snprintf(buf, sizeof buf, "box %d: non-physical state met on the device (flags 0x%x)", k, fl[k]);
            return bfail(b, FISH_ERR_NONPHYSICAL, buf);
        }
    return FISH_OK;
}

}  // namespace

extern "C" {

int fish_batch_create(int nbox, const int *dims, const double *gamma, const int *bc, const double *h,
                      fish_batch **out)
{
    if (!out) return FISH_ERR_ARG;
    *out = nullptr;
    if (nbox < 1 || !dims || !gamma || !bc) return FISH_ERR_ARG;
    long long total = 0;
    for (int k = 0; k < nbox; ++k) {
        for (int a = 0; a < 3; ++a)
            if (dims[3 * k + a] < 1) return FISH_ERR_ARG;
        if (dims[3 * k] % 2 || dims[3 * k + 1] % 2) return FISH_ERR_ARG;  // x and y are paired in the sweeps
        if (!(gamma[k] > 1.0) || (bc[k] != FISH_BC_PERIODIC && bc[k] != FISH_BC_OUTFLOW)) return FISH_ERR_ARG;
        if (h)
            for (int a = 0; a < 3; ++a)
                if (!(h[3 * k + a] > 0.0)) return FISH_ERR_ARG;
        total += (long long)dims[3 * k] * dims[3 * k + 1] * dims[3 * k + 2];
    }
    // every element index of the batch fits an int (the fluid sweeps index
    // with int; margin for the prefetch lines past a box's last column)
    if (total > (1ll << 31) - (1ll << 20)) return FISH_ERR_ARG;
    fish_batch *b = new (std::nothrow) fish_batch;
    if (!b) return FISH_ERR_OOM;
    b->nbox = nbox;
    b->dims.assign(dims, dims + 3 * nbox);
    b->gamma.assign(gamma, gamma + nbox);
    b->bc.assign(bc, bc + nbox);
    b->h.resize(3 * nbox);
    b->off.resize(nbox);
    for (int k = 0; k < nbox; ++k) {
        for (int a = 0; a < 3; ++a) b->h[3 * k + a] = h ? h[3 * k + a] : 1.0 / dims[3 * k + a];
        b->off[k] = b->total;
        b->total += (long long)dims[3 * k] * dims[3 * k + 1] * dims[3 * k + 2];
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess ||
        cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        delete b;
        return FISH_ERR_CUDA;
    }
    b->stream = b->own;
    const size_t bytes = sizeof(float) * (size_t)b->total;
    bool ok = true;
    for (int p = 0; p < 2 && ok; ++p) {
        for (int f = 0; f < 5 && ok; ++f) ok = (b->fl[p][f] = (float *)balloc(b, bytes)) != nullptr;
        for (int f = 0; f < 3 && ok; ++f) ok = (b->bf[p][f] = (float *)balloc(b, bytes)) != nullptr;
    }
    ok = ok && (b->dt = (double *)balloc(b, sizeof(double) * nbox)) && (b->dt_last = (double *)balloc(b, sizeof(double) * nbox)) &&
         (b->minbits = (unsigned long long *)balloc(b, sizeof(unsigned long long) * nbox)) &&
         (b->flags = (unsigned *)balloc(b, sizeof(unsigned) * nbox)) &&
         (b->counters = (int *)balloc(b, sizeof(int) * kCounters)) &&
         (b->tsrc = (const float **)balloc(b, sizeof(float *) * 16 * 4));
    if (!ok) {
        fish_batch_destroy(b);
        return FISH_ERR_OOM;
    }
    if (cudaMemset(b->flags, 0, sizeof(unsigned) * nbox) != cudaSuccess ||
        cudaMemset(b->dt_last, 0, sizeof(double) * nbox) != cudaSuccess) {
        fish_batch_destroy(b);
        return FISH_ERR_CUDA;
    }
    *out = b;
    return FISH_OK;
}

int fish_batch_set_option(fish_batch *b, int key, double v)
{
    if (!b) return FISH_ERR_ARG;
    switch (key) {
    case FISH_BATCH_OPT_LIMITER:
        if (v != FISH_LIM_VANLEER && v != FISH_LIM_MINMOD) return bfail(b, FISH_ERR_ARG, "batch limiter: Van Leer or minmod");
        b->lim = (int)v;
        b->gdirty = true;
        return FISH_OK;
    case FISH_BATCH_OPT_ORDER:
        if (v != 0 && v != 1 && v != 2) return bfail(b, FISH_ERR_ARG, "bad work order");
        b->order = (int)v;
        break;
    case FISH_BATCH_OPT_GROUPS:
        if (v != 1 && v != 2 && v != 4 && v != 8) return bfail(b, FISH_ERR_ARG, "groups per item: 1, 2, 4 or 8");
        b->groups = (int)v;
        break;
    case FISH_BATCH_OPT_GRID:
        if (v != 1 && v != 2 && v != 4) return bfail(b, FISH_ERR_ARG, "grid factor: 1, 2 or 4");
        b->grid_factor = (int)v;
        break;
    case FISH_BATCH_OPT_CTROWS:
        if (v != 4 && v != 8) return bfail(b, FISH_ERR_ARG, "constrained-transport rows per item: 4 or 8");
        b->ctrows = (int)v;
        break;
    default:
        return bfail(b, FISH_ERR_ARG, "unknown batch option");
    }
    b->tables = false;  // rebuilt (and the graph recaptured) before the next step
    b->gdirty = true;
    return FISH_OK;
}

int fish_batch_set_stream(fish_batch *b, void *stream)
{
    if (!b) return FISH_ERR_ARG;
    b->stream = stream ? (cudaStream_t)stream : b->own;
    b->gdirty = true;
    return FISH_OK;
}

int fish_batch_set_state(fish_batch *b, int box, const double *state)
{
    int r = batch_ready(b);
    if (r) return r;
    if (box < 0 || box >= b->nbox || !state) return bfail(b, FISH_ERR_ARG, "bad box or state");
    if ((r = batch_layout(b, 0))) return r;
    const long long N = (long long)b->dims[3 * box] * b->dims[3 * box + 1] * b->dims[3 * box + 2];
    std::vector<float> tmp(N);
    for (int f = 0; f < 8; ++f) {
        for (long long i = 0; i < N; ++i) tmp[i] = (float)state[f * N + i];
        float *dst = (f < 5 ? b->fl[b->cu][f] : b->bf[b->cb][f - 5]) + b->off[box];
        FISH_BCK(b, cudaMemcpyAsync(dst, tmp.data(), sizeof(float) * N, cudaMemcpyHostToDevice, b->stream), "upload");
        FISH_BCK(b, cudaStreamSynchronize(b->stream), "upload");
    }
    b->pending = false;
    return FISH_OK;
}

int fish_batch_get_state(fish_batch *b, int box, double *state)
{
    int r = batch_ready(b);
    if (r) return r;
    if (box < 0 || box >= b->nbox || !state) return bfail(b, FISH_ERR_ARG, "bad box or state");
    if ((r = batch_layout(b, 0))) return r;
    const long long N = (long long)b->dims[3 * box] * b->dims[3 * box + 1] * b->dims[3 * box + 2];
    std::vector<float> tmp(N);
    for (int f = 0; f < 8; ++f) {
        const float *src = (f < 5 ? b->fl[b->cu][f] : b->bf[b->cb][f - 5]) + b->off[box];
        FISH_BCK(b, cudaMemcpyAsync(tmp.data(), src, sizeof(float) * N, cudaMemcpyDeviceToHost, b->stream), "download");
        FISH_BCK(b, cudaStreamSynchronize(b->stream), "download");
        for (long long i = 0; i < N; ++i) state[f * N + i] = tmp[i];
    }
    return batch_flags(b);
}

int fish_batch_step(fish_batch *b, double k, int nsteps)
{
    int r = batch_ready(b);
    if (r) return r;
    if (!(k > 0.0) || nsteps < 0) return bfail(b, FISH_ERR_ARG, "bad arguments");
    if (nsteps == 0) return FISH_OK;
    if ((r = batch_layout(b, layout_of(0)))) return r;
    const int parity = b->cu * 2 + b->cb;
    if (b->gdirty || !b->gexec || b->gk != k || b->gparity != parity) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        // persistent grids: every resident block slot, times the tuning factor
        int occ_f = 0, occ_c = 0;
        FISH_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, fluid_batch_kernel<LIM_VANLEER, true>, 128, 0),
                 "occupancy");
        if (b->ctrows == 8)
            FISH_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, ct_batch_kernel<LIM_VANLEER, 8>, 256, 0),
                     "occupancy");
        else
            FISH_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, ct_batch_kernel<LIM_VANLEER, 4>, 128, 0),
                     "occupancy");
        b->fluid_blocks = std::max(1, occ_f) * b->sms * b->grid_factor;
        b->ct_blocks = std::max(1, occ_c) * b->sms * b->grid_factor;
        cudaGraph_t graph = nullptr;
        const long long l0 = b->launches;
        FISH_BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        r = batch_queue_step(b, k);
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (r) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return bcuda(b, e, "end capture");
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
        b->launches = l0;
        b->gk = k;
        b->gparity = parity;
        b->gdirty = false;
    }
    if (!b->pending)
        if ((r = batch_cfl(b))) return r;
    for (int s = 0; s < nsteps; ++s) {
        FISH_BCK(b, cudaGraphLaunch(b->gexec, b->stream), "graph launch");
        b->launches += 15;
    }
    b->pending = true;
    return FISH_OK;
}

int fish_batch_last_dt(fish_batch *b, double *dt)
{
    if (!b || !dt) return FISH_ERR_ARG;
    FISH_BCK(b, cudaMemcpyAsync(dt, b->dt_last, sizeof(double) * b->nbox, cudaMemcpyDeviceToHost, b->stream), "dt");
    return batch_flags(b);
}

int fish_batch_sync(fish_batch *b)
{
    if (!b) return FISH_ERR_ARG;
    return batch_flags(b);
}

const char *fish_batch_last_error(fish_batch *b) { return b ? b->err.c_str() : "null batch"; }

long long fish_batch_launch_count(fish_batch *b) { return b ? b->launches : -1; }

long long fish_batch_cells(fish_batch *b) { return b ? b->total : -1; }

void fish_batch_destroy(fish_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (void *p : b->owned) cudaFree(p);
    if (b->own) cudaStreamDestroy(b->own);
    delete b;
}

}  // extern "C"
