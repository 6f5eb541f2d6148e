// fish_ring.cuh -- ring-fed column march of FISH's fluid operator L_d
// (Kaeppeli et al., arXiv:0910.2854, Sec. 2.2 and the pipelined loop of
// Sec. 3), FP32 two-column pairs.
//
// The arithmetic is that of fluid_col_kernel<P2> (ceval, cflux1, cflux2 of
// fish_column.cuh, same operations in the same order, so both kernels give
// bitwise the same result); what differs is how the cells reach the
// registers.  A block of 128 threads owns 256 consecutive columns of one row
// of the other transverse axis.  Its input rows (the five fluid fields, b_d,
// the fast- and other-axis faces and the other-axis faces of the row below)
// are brought into a ring of shared-memory stages by bulk copies of the TMA
// engine, one stage per cell along the sweep, issued a few cells ahead of
// the march and signalled through mbarriers.  The threads then read their
// cells from shared memory: no per-thread address arithmetic, no L2
// prefetch instructions, and the old state of the output cell (three cells
// behind the raw cell) is re-read from the ring instead of L2.  Ghost cells
// are stages copied from the mapped cell (periodic wrap or the boundary cell
// of zeroth-order extrapolation), so prologue and tail need no special
// loads.
//
// Ring protocol: stage q (raw cell q = -3 .. n+2) lives in slot (q+3) mod D.
// Its copies are issued by lane 0 of warp q mod 4 while the march is at
// cell q-1-L; the march waits on the slot's `full` barrier before reading
// it; every warp arrives on the slot's `empty` barrier after its last use of
// the stage (march cell q+4: the lower b_d face of the CFL epilogue), and
// the producer waits for that before the slot takes stage q+D.
#pragma once

#include "fish_async.cuh"
#include "fish_column.cuh"

namespace fish {

#ifndef FISH_RING_D
#define FISH_RING_D 11   // stages in the ring
#endif
#ifndef FISH_RING_L
#define FISH_RING_L 3    // stages issued ahead of the one being read
#endif
#ifndef FISH_RING_PF
#define FISH_RING_PF 0   // stages beyond the copies whose rows are prefetched into L2 (0: none)
#endif
static_assert(FISH_RING_D >= FISH_RING_L + 6, "a slot must be released before it is refilled");

#ifndef FISH_RING_T
#define FISH_RING_T 128  // threads per block (two columns each)
#endif
constexpr int RF_THREADS = FISH_RING_T;
constexpr int RF_COLS = 2 * RF_THREADS;  // columns per block
// floats of one stage: u0..u4, b_d, b_o, b_o of the row below, then b_f
// behind a four-float prefix that holds the faces left of the block
enum : int { RF_U = 0, RF_BD = 5 * RF_COLS, RF_BO = 6 * RF_COLS, RF_BOM = 7 * RF_COLS, RF_BF = 8 * RF_COLS,
             RF_ROWS = 9, RF_STAGE = RF_ROWS * RF_COLS + 4 };
static_assert((RF_STAGE * 4) % 16 == 0, "stages must stay 16-byte aligned");
// side rows (after the ring): b_d of the cell below raw cell -3, and b_d of
// cell n-2 (the lower face of the outflow ghosts above the box)
enum : int { RF_SIDE_LO = 0, RF_SIDE_TOP = RF_COLS, RF_SIDE = 2 * RF_COLS };

constexpr size_t ring_fluid_smem()
{
    return sizeof(float) * ((size_t)FISH_RING_D * RF_STAGE + RF_SIDE) + 2 * FISH_RING_D * sizeof(uint64_t);
}

struct FRing {
    float *st;           // stage data
    float *side;         // side rows
    uint64_t *full, *empty;
    int f0, ob, cols;    // first column, row of the other axis, columns of the block
    int c2;              // the thread's first column within the block (clamped for idle threads)
    int bfm;             // index in the b_f row (prefix included) of the face below the first column
    bool active;         // the thread owns columns of the box (else it only keeps the warp complete)
    bool dead;           // a bounded wait timed out: skip further waits
};

__device__ __forceinline__ int rf_slot(int q) { return (q + 3) % FISH_RING_D; }
__device__ __forceinline__ unsigned rf_par(int q) { return (unsigned)(((q + 3) / FISH_RING_D) & 1); }

// Issue the copies of stage q (one thread).  The fast transverse axis is t1
// (FP32 orders the frame so), so b_f = b_t1 and b_o = b_t2.
__device__ __forceinline__ void rf_produce(const ColFluidArgs<float> &A, FRing &R, int q)
{
    const int slot = rf_slot(q);
    const int occ = (q + 3) / FISH_RING_D;
    if (occ > 0 && !R.dead)
        if (!mbar_wait(&R.empty[slot], (unsigned)((occ - 1) & 1), A.flags)) R.dead = true;
    const long long cc = gmap(q, A.n, A.bc);
    const long long row = A.off + R.f0 + (long long)R.ob * A.so + cc * A.sd;
    const long long rowm = A.off + R.f0 + (long long)gmap(R.ob - 1, A.no, A.bc) * A.so + cc * A.sd;
    const int pf = R.f0 > 0 ? R.f0 - 4 : (A.bc == BC_PERIODIC ? A.nf - 4 : 0);
    const long long rowp = A.off + pf + (long long)R.ob * A.so + cc * A.sd;
    const unsigned rb = 4u * (unsigned)R.cols;
    float *s = R.st + (size_t)slot * RF_STAGE;
    uint64_t *bar = &R.full[slot];
    // transaction bytes of the stage: RF_ROWS rows of the block plus the
    // 16-byte prefix (the copies below)
    mbar_arrive_expect_tx(bar, (unsigned)RF_ROWS * rb + 16u);
#pragma unroll
    for (int k = 0; k < 5; ++k) bulk_g2s(s + RF_U + k * RF_COLS, A.u[k] + row, rb, bar);
    bulk_g2s(s + RF_BD, A.bd + row, rb, bar);
    bulk_g2s(s + RF_BO, A.bt2 + row, rb, bar);
    bulk_g2s(s + RF_BOM, A.bt2 + rowm, rb, bar);
    bulk_g2s(s + RF_BF, A.bt1 + rowp, 16u, bar);
    bulk_g2s(s + RF_BF + 4, A.bt1 + row, rb, bar);
    if constexpr (FISH_RING_PF > 0) {
        // the rows of stage q+PF into L2 (interior cells only)
        const int qp = q + FISH_RING_PF;
        if (qp < A.n) {
            const long long d = (long long)(qp - cc) * A.sd;
#pragma unroll
            for (int k = 0; k < 5; ++k) bulk_prefetch_l2(A.u[k] + row + d, rb);
            bulk_prefetch_l2(A.bd + row + d, rb);
            bulk_prefetch_l2(A.bt2 + row + d, rb);
            bulk_prefetch_l2(A.bt2 + rowm + d, rb);
            bulk_prefetch_l2(A.bt1 + row + d, rb);
        }
    }
}

// Wait for stage q and read the thread's raw cell from it (b_d of the lower
// face is set by the caller).
__device__ __forceinline__ void rf_read(const ColFluidArgs<float> &A, FRing &R, int q, FRaw<P2> &W)
{
    const int slot = rf_slot(q);
    if (!R.dead)
        if (!mbar_wait(&R.full[slot], rf_par(q), A.flags)) R.dead = true;
    const float *s = R.st + (size_t)slot * RF_STAGE;
#pragma unroll
    for (int k = 0; k < 5; ++k) W.u[k].v = *reinterpret_cast<const float2 *>(s + RF_U + k * RF_COLS + R.c2);
    W.bd.v = *reinterpret_cast<const float2 *>(s + RF_BD + R.c2);
    W.bo.v = *reinterpret_cast<const float2 *>(s + RF_BO + R.c2);
    W.bom.v = *reinterpret_cast<const float2 *>(s + RF_BOM + R.c2);
    W.bf.v = *reinterpret_cast<const float2 *>(s + RF_BF + 4 + R.c2);
    W.bfm = s[RF_BF + R.bfm];
}

__device__ __forceinline__ P2 rf_get(const FRing &R, int q, int off)
{
    return {*reinterpret_cast<const float2 *>(R.st + (size_t)rf_slot(q) * RF_STAGE + off + R.c2)};
}

// One step of the ring march for raw cell r (K = r mod 4): the fluid part
// of fstep<P2, HSE = false, GM = 0, FT1 = true, NU = false> with the loads
// taken from the ring.  RD: read raw cell r+1 (if it exists).
template <int LIM, bool CFLF, int K, int ST, bool RD>
__device__ __forceinline__ void rstep(const ColFluidArgs<float> &A, FRing &R, FMarch<P2> &M, int r, P2 lam, P2 lamh)
{
    constexpr int k2 = K & 1, p2 = (K + 1) & 1;
    const P2 half = vb<P2>(0.5f);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // consume the raw input of cell r
    P2 bbr[3];
    P2 ur[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) ur[k] = M.R.u[k];
    bbr[0] = half * (M.R.bdm + M.R.bd);
    const P2 bd_r = M.R.bd;
    bbr[1] = half * (vshift_lo(M.R.bfm, M.R.bf) + M.R.bf);
    bbr[2] = half * (M.R.bom + M.R.bo);
    // raw cell r+1 from the ring (its lower face: this cell's, or b_d of
    // cell n-2 for the outflow ghosts above the box)
    if (RD && r + 1 <= A.n + 2) {
        rf_read(A, R, r + 1, M.R);
        if (A.bc == BC_OUTFLOW && r + 1 >= A.n) M.R.bdm.v = *reinterpret_cast<const float2 *>(R.side + RF_SIDE_TOP + R.c2);
        else M.R.bdm = bd_r;
    }
    // copies of stage r+1+L (one lane of one warp, the warps in turn)
    if (warp == ((K + 1 + FISH_RING_L) & 3) && lane == 0 && r + 1 + FISH_RING_L <= A.n + 2)
        rf_produce(A, R, r + 1 + FISH_RING_L);
    // old state of the output cell o = r-3
    const int o = r - 3;
    P2 un[5];
    if constexpr ((ST & ST_OUT) != 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) un[k] = rf_get(R, o, RF_U + k * RF_COLS);
    }
    ceval<P2>(ur, bbr, vb<P2>(A.gamma), vb<P2>(A.gm1), M.C[k2], M.chk);
#pragma unroll
    for (int k = 0; k < 3; ++k) M.bb[k2][k] = bbr[k];
    if constexpr ((ST & ST_F1) != 0) {
        // predictor flux at (r-1, r) (eq0140)
        cflux1<P2, false>(M.C[p2], M.C[k2], vb<P2>(0.f), vb<P2>(0.f), vb<P2>(A.alpha), M.F1[k2]);
    }
    if constexpr ((ST & ST_PRED) != 0) {
        // predicted half step of cell r-1 (eq0253 without source)
        const CCell<P2> &cp = M.C[p2];
        P2 up[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) up[k] = vfma(-lamh, M.F1[k2][k] - M.F1[p2][k], cp.u[k]);
        constexpr int s3 = (K + 3) & 3;  // slot of cell r-1
        ceval<P2>(up, M.bb[p2], vb<P2>(A.gamma), vb<P2>(A.gm1), M.P[s3], M.chk);
        if constexpr ((ST & ST_F2) != 0) {
            // corrector flux at (r-3, r-2) from predicted cells r-4 .. r-1 (eq0230)
            constexpr int s0 = K & 3, s1 = (K + 1) & 3, s2 = (K + 2) & 3;
            const P2 z = vb<P2>(0.f);
            cflux2<P2, false, LIM, false>(M.P[s0], M.P[s1], M.P[s2], M.P[s3], z, z, z, z, M.F2[k2], A.lim);
            if constexpr ((ST & ST_OUT) != 0) {
#pragma unroll
                for (int k = 0; k < 5; ++k) un[k] = vfma(-lam, M.F2[k2][k] - M.F2[p2][k], un[k]);
                if (R.active) {
                    const long long io = A.off + R.f0 + R.c2 + (long long)R.ob * A.so + (long long)o * A.sd;
#pragma unroll
                    for (int k = 0; k < 5; ++k) vstore(A.uo[k], io, un[k]);
                }
                if constexpr (CFLF) {
                    // CFL rate of the updated cell with its cell-centred field
                    // (lower b_d face: stage o-1, the map of cell o-1)
                    P2 bc[3];
                    bc[0] = half * (rf_get(R, o - 1, RF_BD) + rf_get(R, o, RF_BD));
                    const float *so = R.st + (size_t)rf_slot(o) * RF_STAGE;
                    const P2 bfv = rf_get(R, o, RF_BF + 4);
                    bc[1] = half * (vshift_lo(so[RF_BF + R.bfm], bfv) + bfv);
                    bc[2] = half * (rf_get(R, o, RF_BOM) + rf_get(R, o, RF_BO));
                    const P2 rh[3] = {vb<P2>(A.rh[0]), vb<P2>(A.rh[1]), vb<P2>(A.rh[2])};
                    M.cflr = vmax(M.cflr, cfl_rate3<P2>(un, bc, vb<P2>(A.gamma), vb<P2>(A.gm1), rh));
                }
            }
        }
    }
    // release stage r-4 (its last use was this step's lower CFL face)
    if (r - 4 >= -3) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&R.empty[rf_slot(r - 4)]);
    }
}

// L_d of one block: 256 columns of one row of the other axis, the whole
// sweep extent.  Grid: ceil(nf / 256) x no blocks; dynamic shared memory
// ring_fluid_smem().  Requires nf % 4 == 0 and 16-byte aligned rows (the
// launcher checks); FP32 frame with t1 fast, no potential, uniform mesh.
template <int LIM, bool CFLF>
__global__ void __launch_bounds__(RF_THREADS, 256 / RF_THREADS) fluid_ring_kernel(const ColFluidArgs<float> A)
{
    extern __shared__ __align__(128) unsigned char rf_smem[];
    FRing R;
    R.st = reinterpret_cast<float *>(rf_smem);
    R.side = R.st + (size_t)FISH_RING_D * RF_STAGE;
    R.full = reinterpret_cast<uint64_t *>(R.side + RF_SIDE);
    R.empty = R.full + FISH_RING_D;
    R.dead = false;
    const int nbf = (A.nf + RF_COLS - 1) / RF_COLS;
    R.f0 = (int)(blockIdx.x % nbf) * RF_COLS;
    R.ob = (int)(blockIdx.x / nbf);
    R.cols = min(RF_COLS, A.nf - R.f0);
    const int t = threadIdx.x;
    const bool active = 2 * t < R.cols;
    R.active = active;
    R.c2 = active ? 2 * t : R.cols - 2;
    R.bfm = R.c2 > 0 ? R.c2 + 3 : ((R.f0 == 0 && A.bc == BC_OUTFLOW) ? 0 : 3);
    const int n = A.n;
    if (t == 0) {
        for (int i = 0; i < FISH_RING_D; ++i) {
            mbar_init(&R.full[i], 1);
            mbar_init(&R.empty[i], RF_THREADS / 32);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (t == 0) {
        // side rows ride on stage -3's barrier, then stages -3 .. -3+L
        const long long base = A.off + R.f0 + (long long)R.ob * A.so;
        const unsigned rb = 4u * (unsigned)R.cols;
        uint64_t *bar = &R.full[rf_slot(-3)];
        mbar_expect_tx(bar, 2u * rb);
        bulk_g2s(R.side + RF_SIDE_LO, A.bd + base + (long long)gmap(gmap(-3, n, A.bc) - 1, n, A.bc) * A.sd, rb, bar);
        bulk_g2s(R.side + RF_SIDE_TOP, A.bd + base + (long long)gmap(n - 2, n, A.bc) * A.sd, rb, bar);
        for (int q = -3; q <= -3 + FISH_RING_L && q <= n + 2; ++q) rf_produce(A, R, q);
    }
    const double dtd = *A.dt;
    const P2 lam = vb<P2>(float(dtd / A.h));
    const P2 lamh = vb<P2>(float(dtd / (2.0 * A.h)));

    FMarch<P2> M;
    checks_init(M.chk);
    M.cflr = vb<P2>(0.0f);
    rf_read(A, R, -3, M.R);
    M.R.bdm.v = *reinterpret_cast<const float2 *>(R.side + RF_SIDE_LO + R.c2);
    constexpr int ALL = ST_F1 | ST_PRED | ST_F2 | ST_OUT;
    rstep<LIM, CFLF, 1, 0, true>(A, R, M, -3, lam, lamh);
    rstep<LIM, CFLF, 2, ST_F1, true>(A, R, M, -2, lam, lamh);
    rstep<LIM, CFLF, 3, ST_F1 | ST_PRED, true>(A, R, M, -1, lam, lamh);
    rstep<LIM, CFLF, 0, ST_F1 | ST_PRED, true>(A, R, M, 0, lam, lamh);
    rstep<LIM, CFLF, 1, ST_F1 | ST_PRED, true>(A, R, M, 1, lam, lamh);
    rstep<LIM, CFLF, 2, ST_F1 | ST_PRED | ST_F2, true>(A, R, M, 2, lam, lamh);
    int r = 3;
#pragma unroll 1
    for (; r + 4 <= n - 1; r += 4) {
        rstep<LIM, CFLF, 3, ALL, true>(A, R, M, r, lam, lamh);
        rstep<LIM, CFLF, 0, ALL, true>(A, R, M, r + 1, lam, lamh);
        rstep<LIM, CFLF, 1, ALL, true>(A, R, M, r + 2, lam, lamh);
        rstep<LIM, CFLF, 2, ALL, true>(A, R, M, r + 3, lam, lamh);
    }
    // tail: raw cells r .. n+2 (r = 3 mod 4, at most seven)
    if (r <= n + 2) rstep<LIM, CFLF, 3, ALL, true>(A, R, M, r, lam, lamh);
    if (r + 1 <= n + 2) rstep<LIM, CFLF, 0, ALL, true>(A, R, M, r + 1, lam, lamh);
    if (r + 2 <= n + 2) rstep<LIM, CFLF, 1, ALL, true>(A, R, M, r + 2, lam, lamh);
    if (r + 3 <= n + 2) rstep<LIM, CFLF, 2, ALL, true>(A, R, M, r + 3, lam, lamh);
    if (r + 4 <= n + 2) rstep<LIM, CFLF, 3, ALL, true>(A, R, M, r + 4, lam, lamh);
    if (r + 5 <= n + 2) rstep<LIM, CFLF, 0, ALL, true>(A, R, M, r + 5, lam, lamh);
    if (r + 6 <= n + 2) rstep<LIM, CFLF, 1, ALL, false>(A, R, M, r + 6, lam, lamh);

    if (active) {
        const unsigned fl = checks_flags(M.chk);
        if (fl) atomicOr(A.flags, fl);
    }
    if constexpr (CFLF) {
        // warp maximum of the rates (order-preserving bits of non-negative
        // floats), then one atomic minimum of 1/rate per warp
        float m = 0.0f;
        if (active) m = fmaxf(M.cflr.v.x, M.cflr.v.y);
        const unsigned wm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
        if ((t & 31) == 0 && wm != 0u) {
            const float mx = __uint_as_float(wm);
            if (mx > 0.0f && mx == mx) {
                atomicMin(A.cfl_min, (unsigned long long)__double_as_longlong(1.0 / (double)mx));
            } else {
                atomicOr(A.flags, FLAG_NAN);
            }
        }
    }
    // every issued stage was waited on by the march (the last one, n+2, by
    // the step at n+1), so no copy is in flight here unless a wait gave up;
    // then give the copies a bounded time to land before the block leaves
    if (R.dead && t == 0) {
        for (int q = max(-3, n + 2 - FISH_RING_D + 1); q <= n + 2; ++q) {
            if (!mbar_test(&R.full[rf_slot(q)], rf_par(q))) {
                const long long t0 = clock64();
                while (!mbar_test(&R.full[rf_slot(q)], rf_par(q)) && clock64() - t0 < (1ll << 31)) {
                }
            }
        }
    }
}

// launcher: FP32 pairs, t1 fast, no potential, uniform mesh, Van Leer /
// minmod / hybrid limiter; cudaErrorNotSupported where the ring kernel does
// not apply (the caller then runs the column kernel)
cudaError_t ring_fluid(const ColFluidArgs<float> &A, cudaStream_t s);
bool ring_fluid_applies(const ColFluidArgs<float> &A);

}  // namespace fish
