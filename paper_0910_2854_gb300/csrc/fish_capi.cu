// fish_capi.cu -- C ABI of libfish.so (declared in include/fish.h): context,
// device memory, state transfer, the x-y-z-z-y-x double step (eq0081-eq0082,
// reading C-4) and its CUDA-graph replay, CFL (eq0083-eq0084), diagnostics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/fish.h"
#include "fish_launch.h"

using fish::Geom;
using fish::Launch;

namespace {

constexpr int kDiagBlocks = 1024;
constexpr long long kStageChunk = 1ll << 25;  // doubles per conversion chunk (256 MB)

}  // namespace

struct fish_ctx {
    int n[3] = {0, 0, 0};
    long long N = 0;
    double gamma = 0.0;
    int bc = 0;
    int prec = FISH_PREC_FP64;
    int lim = FISH_LIM_VANLEER;
    int hse = 0;
    int gsplit = 0;        // FISH_GRAV_SPLIT: gravity as G_d(dt/2) L_d G_d(dt/2)
    double alpha = 1.0;
    double h[3] = {0, 0, 0};
    int kernels = FISH_KERNELS_COLUMN;  // FISH_OPT_KERNELS

    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    void *(*ualloc)(size_t, void *) = nullptr;
    void (*ufree)(void *, void *) = nullptr;
    void *uud = nullptr;
    std::vector<void *> owned;

    bool allocated = false;
    void *fl[2][5] = {};   // fluid fields rho, m_x, m_y, m_z, E (two buffers)
    void *bf[2][3] = {};   // face fields b_x, b_y, b_z (two buffers)
    int cu = 0, cb = 0;    // current buffer of each group
    int layout = 0;        // 0: x fastest (y, z sweeps); 1: y fastest (x sweeps)
    void *phi = nullptr;   // FP64: potential, x-fastest layout
    void *phiT = nullptr;  // FP64: potential, y-fastest layout
    void *phiD[3] = {};    // FP32: phi(next cell along d) - phi(cell) formed in FP64, in the layout of the d sweeps
    bool has_phi = false;

    // irregular Cartesian mesh (eq037): host widths per axis (empty: h of
    // the axis), device copies of all three in the state's precision
    bool nu = false;
    std::vector<double> wmesh[3];
    void *wdev[3] = {};
    int wdev_prec = -1;
    bool mesh_dirty = false;

    double *dt_dev = nullptr;       // time step read by the sweep kernels
    double *dt_last = nullptr;      // dt of the last step
    unsigned long long *minbits = nullptr;
    unsigned *flags = nullptr;
    double *partial = nullptr;
    double *stage = nullptr;        // conversion staging (kStageChunk doubles)

    // one captured double step per starting buffer parity (cu*2 + cb): a step
    // whose sweeps also change the layout ends on the other parity
    cudaGraphExec_t gexec[4] = {};
    int gend[4] = {0, 0, 0, 0};   // parity after the step
    double gk = -1.0;
    bool gdirty = true;
    bool gfused = false;       // the graph's last sweep reduces the next CFL
    long long glaunches = 0;   // kernels per graph replay
    bool cfl_pending = false;  // minbits holds the CFL minimum of the current state

    long long launches = 0;
    std::string err;
};

namespace {

int fail(fish_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(fish_ctx *c, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? FISH_ERR_OOM : FISH_ERR_CUDA, m);
}

#define FISH_CK(c, expr, what)                            \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

size_t esize(const fish_ctx *c) { return c->prec == FISH_PREC_FP64 ? sizeof(double) : sizeof(float); }

void *dev_alloc(fish_ctx *c, size_t bytes)
{
    void *p = nullptr;
    if (c->ualloc) {
        p = c->ualloc(bytes, c->uud);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        p = nullptr;
    }
    if (p) c->owned.push_back(p);
    return p;
}

void dev_free_all(fish_ctx *c)
{
    for (void *p : c->owned) {
        if (c->ufree)
            c->ufree(p, c->uud);
        else
            cudaFree(p);
    }
    c->owned.clear();
}

Geom geom_of(const fish_ctx *c, int layout)
{
    Geom g;
    for (int a = 0; a < 3; ++a) g.n[a] = c->n[a];
    if (layout == 0) {
        g.st[0] = 1;
        g.st[1] = c->n[0];
        g.ord[0] = 0;
        g.ord[1] = 1;
    } else {
        g.st[0] = c->n[1];
        g.st[1] = 1;
        g.ord[0] = 1;
        g.ord[1] = 0;
    }
    g.st[2] = (long long)c->n[0] * c->n[1];
    g.ord[2] = 2;
    g.bc = c->bc;
    return g;
}

Geom geom(const fish_ctx *c) { return geom_of(c, c->layout); }

int ensure_alloc(fish_ctx *c)
{
    if (c->allocated) return FISH_OK;
    const size_t bytes = (size_t)c->N * esize(c);
    for (int b = 0; b < 2; ++b) {
        for (int f = 0; f < 5; ++f)
            if (!(c->fl[b][f] = dev_alloc(c, bytes))) return fail(c, FISH_ERR_OOM, "state allocation failed");
        for (int f = 0; f < 3; ++f)
            if (!(c->bf[b][f] = dev_alloc(c, bytes))) return fail(c, FISH_ERR_OOM, "state allocation failed");
    }
    c->dt_dev = (double *)dev_alloc(c, sizeof(double));
    c->dt_last = (double *)dev_alloc(c, sizeof(double));
    c->minbits = (unsigned long long *)dev_alloc(c, sizeof(unsigned long long));
    c->flags = (unsigned *)dev_alloc(c, sizeof(unsigned));
    c->partial = (double *)dev_alloc(c, sizeof(double) * 9 * kDiagBlocks);
    if (!c->dt_dev || !c->dt_last || !c->minbits || !c->flags || !c->partial)
        return fail(c, FISH_ERR_OOM, "scalar allocation failed");
    const unsigned long long inf = 0x7FF0000000000000ull;
    FISH_CK(c, cudaMemcpyAsync(c->minbits, &inf, sizeof(inf), cudaMemcpyHostToDevice, c->stream), "init");
    FISH_CK(c, cudaMemsetAsync(c->flags, 0, sizeof(unsigned), c->stream), "init");
    FISH_CK(c, cudaMemsetAsync(c->dt_dev, 0, sizeof(double), c->stream), "init");
    FISH_CK(c, cudaMemsetAsync(c->dt_last, 0, sizeof(double), c->stream), "init");
    FISH_CK(c, cudaStreamSynchronize(c->stream), "init");
    c->allocated = true;
    return FISH_OK;
}

int ensure_stage(fish_ctx *c)
{
    if (c->stage) return FISH_OK;
    c->stage = (double *)dev_alloc(c, sizeof(double) * kStageChunk);
    return c->stage ? FISH_OK : fail(c, FISH_ERR_OOM, "staging allocation failed");
}

void *field_ptr(fish_ctx *c, int f)
{
    return f < 5 ? c->fl[c->cu][f] : c->bf[c->cb][f - 5];
}

// Move the state of the current buffers into the other buffers in the
// other layout (the paper's data rotation, Sec. 3, as a transpose).
template <class T> int transpose_state(fish_ctx *c)
{
    const T *src[8];
    T *dst[8];
    for (int f = 0; f < 5; ++f) {
        src[f] = (const T *)c->fl[c->cu][f];
        dst[f] = (T *)c->fl[1 - c->cu][f];
    }
    for (int f = 0; f < 3; ++f) {
        src[5 + f] = (const T *)c->bf[c->cb][f];
        dst[5 + f] = (T *)c->bf[1 - c->cb][f];
    }
    const int nr = c->layout == 0 ? c->n[0] : c->n[1];
    const int nc = c->layout == 0 ? c->n[1] : c->n[0];
    FISH_CK(c, Launch<T>::transpose(src, dst, 8, nr, nc, c->n[2], c->stream), "transpose launch");
    c->cu = 1 - c->cu;
    c->cb = 1 - c->cb;
    c->layout = 1 - c->layout;
    c->launches += 1;
    return FISH_OK;
}

int set_layout(fish_ctx *c, int layout)
{
    if (c->layout == layout) return FISH_OK;
    // a layout change is only needed when both sizes are > 1
    return c->prec == FISH_PREC_FP64 ? transpose_state<double>(c) : transpose_state<float>(c);
}

// layout an operator along d reads coalesced: y fastest for x sweeps
inline int layout_for(int d) { return d == 0 ? 1 : 0; }

int check_flags(fish_ctx *c)
{
    unsigned fl = 0;
    FISH_CK(c, cudaMemcpyAsync(&fl, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream), "flags");
    FISH_CK(c, cudaStreamSynchronize(c->stream), "sync");
    if (fl & fish::FLAG_TIMEOUT) return fail(c, FISH_ERR_TIMEOUT, "device wait timed out");
    if (fl) {
        char buf[160];
        snprintf(buf, sizeof buf, "non-physical state met on the device (flags 0x%x:%s%s%s)", fl,
                 (fl & fish::FLAG_RHO) ? " rho<=0" : "", (fl & fish::FLAG_P) ? " p<=0" : "",
                 (fl & fish::FLAG_NAN) ? " NaN" : "");
        return fail(c, FISH_ERR_NONPHYSICAL, buf);
    }
    return FISH_OK;
}

// ---- operators -------------------------------------------------------------

// Potential data of the d sweep: FP64 the cell potential in the current
// layout, FP32 the FP64-formed differences along d.
template <class T> const T *sweep_potential(const fish_ctx *c, int d)
{
    if (!c->has_phi) return nullptr;
    if (sizeof(T) == 4) return (const T *)c->phiD[d];
    return (const T *)(c->layout ? c->phiT : c->phi);
}

// Device cell widths of the three axes (irregular mesh), else nullptr.
template <class T> struct MeshPtrs {
    const T *w[3] = {nullptr, nullptr, nullptr};
    const T *const *get() const { return w[0] ? w : nullptr; }
};
template <class T> MeshPtrs<T> mesh_of(const fish_ctx *c)
{
    MeshPtrs<T> m;
    if (c->nu)
        for (int a = 0; a < 3; ++a) m.w[a] = (const T *)c->wdev[a];
    return m;
}

// G_d(dt/2) in place on the current fluid buffer (operator-split gravity)
template <class T> int op_gravity(fish_ctx *c, int d)
{
    T *u[5];
    for (int f = 0; f < 5; ++f) u[f] = (T *)c->fl[c->cu][f];
    const MeshPtrs<T> m = mesh_of<T>(c);
    FISH_CK(c, Launch<T>::gravity(u, sweep_potential<T>(c, d), c->dt_dev, 0.5, geom(c), d, c->h[d], c->stream, m.w[d]),
            "gravity launch");
    c->launches += 1;
    return FISH_OK;
}

bool split_gravity(const fish_ctx *c) { return c->gsplit && c->has_phi; }

// L_d, or G_d(dt/2) L_d G_d(dt/2) with operator-split gravity (eq025111):
// on a uniform mesh the kicks run inside the fluid march, on an irregular
// one as separate passes around it
template <class T> int op_fluid(fish_ctx *c, int d, bool fuse_cfl)
{
    const bool fused_split = split_gravity(c) && !c->nu;
    const bool split = split_gravity(c) && !fused_split;
    int r;
    if (split && (r = op_gravity<T>(c, d))) return r;
    const T *in[8];
    T *out[5];
    for (int f = 0; f < 5; ++f) {
        in[f] = (const T *)c->fl[c->cu][f];
        out[f] = (T *)c->fl[1 - c->cu][f];
    }
    for (int f = 0; f < 3; ++f) in[5 + f] = (const T *)c->bf[c->cb][f];
    FISH_CK(c,
            Launch<T>::fluid(in, out, split ? nullptr : sweep_potential<T>(c, d), c->dt_dev,
                             geom(c), d, c->lim, c->hse != 0, c->gamma, c->alpha, c->h, c->flags,
                             fuse_cfl ? c->minbits : nullptr, c->stream, mesh_of<T>(c).get(), fused_split,
                             c->kernels),
            "fluid sweep launch");
    c->cu = 1 - c->cu;
    c->launches += 1;
    if (split && (r = op_gravity<T>(c, d))) return r;
    return FISH_OK;
}

template <class T> int op_ct(fish_ctx *c, int d)
{
    const T *b[3];
    T *bo[3];
    for (int f = 0; f < 3; ++f) {
        b[f] = (const T *)c->bf[c->cb][f];
        bo[f] = (T *)c->bf[1 - c->cb][f];
    }
    FISH_CK(c,
            Launch<T>::ct((const T *)c->fl[c->cu][0], (const T *)c->fl[c->cu][1 + d], b, bo, c->dt_dev, geom(c), d,
                          c->lim, c->h, c->flags, c->stream, mesh_of<T>(c).get()),
            "constrained-transport sweep launch");
    c->cb = 1 - c->cb;
    c->launches += 1;
    return FISH_OK;
}

int apply_op(fish_ctx *c, int op, int d, bool fuse_cfl = false)
{
    int r = set_layout(c, layout_for(d));
    if (r) return r;
    if (c->prec == FISH_PREC_FP64)
        return op == FISH_OP_FLUID ? op_fluid<double>(c, d, fuse_cfl) : op_ct<double>(c, d);
    return op == FISH_OP_FLUID ? op_fluid<float>(c, d, fuse_cfl) : op_ct<float>(c, d);
}

// Whether the last sweep of a double step (L_x) can also reduce the CFL
// minimum of the new state (FP32 two-column kernels only).
bool last_sweep_fuses_cfl(const fish_ctx *c)
{
    if (c->prec != FISH_PREC_FP32 || c->nu) return false;  // (split kicks run inside the march)
    return Launch<float>::fluid_fuses_cfl(geom_of(c, layout_for(0)), 0, c->lim, c->hse != 0);
}

// The twelve operators of one double step in time order (reading C-4);
// with fuse_cfl the final L_x also reduces the CFL minimum of the result.
int queue_sweeps(fish_ctx *c, bool fuse_cfl = false)
{
    int r;
    for (int d = 0; d < 3; ++d) {
        if ((r = apply_op(c, FISH_OP_FLUID, d))) return r;
        if ((r = apply_op(c, FISH_OP_CT, d))) return r;
    }
    for (int d = 2; d >= 0; --d) {
        if ((r = apply_op(c, FISH_OP_CT, d))) return r;
        if ((r = apply_op(c, FISH_OP_FLUID, d, fuse_cfl && d == 0))) return r;
    }
    return FISH_OK;
}

template <class T> int queue_cfl(fish_ctx *c, int k0 = 0, int nk = -1)
{
    const T *in[8];
    for (int f = 0; f < 8; ++f) in[f] = (const T *)field_ptr(c, f);
    FISH_CK(c,
            Launch<T>::cfl(in, geom(c), c->h, c->gamma, c->minbits, c->flags, c->stream, mesh_of<T>(c).get(), k0,
                           nk),
            "cfl launch");
    c->launches += 1;
    return FISH_OK;
}

// Standalone CFL reduction into minbits (reset first), over the z-planes
// k0 .. k0+nk-1 (nk < 0: all).
int queue_cfl_min(fish_ctx *c, int k0 = 0, int nk = -1)
{
    FISH_CK(c, fish::launch_reset_min(c->minbits, c->stream), "cfl reset launch");
    c->launches += 1;
    return c->prec == FISH_PREC_FP64 ? queue_cfl<double>(c, k0, nk) : queue_cfl<float>(c, k0, nk);
}

int queue_cfl_dt(fish_ctx *c, double k, double *dt_target, double *dt_copy, int k0 = 0, int nk = -1)
{
    int r = queue_cfl_min(c, k0, nk);
    if (r) return r;
    FISH_CK(c, fish::launch_cfl_finish(c->minbits, k, dt_target, dt_copy, c->stream), "cfl finish launch");
    c->launches += 1;
    return FISH_OK;
}

// Upload the cell widths of an irregular mesh (outside any capture): the
// given widths per axis, h of the axis where none were given.
int sync_mesh(fish_ctx *c)
{
    if (!c->nu || (!c->mesh_dirty && c->wdev_prec == c->prec)) return FISH_OK;
    const size_t es = esize(c);
    for (int a = 0; a < 3; ++a) {
        if (c->wdev_prec != c->prec) c->wdev[a] = nullptr;  // other precision: fresh arrays
        if (!c->wdev[a] && !(c->wdev[a] = dev_alloc(c, (size_t)c->n[a] * es)))
            return fail(c, FISH_ERR_OOM, "mesh allocation failed");
        std::vector<double> wd(c->n[a], c->h[a]);
        if (!c->wmesh[a].empty()) wd = c->wmesh[a];
        if (c->prec == FISH_PREC_FP64) {
            FISH_CK(c, cudaMemcpy(c->wdev[a], wd.data(), wd.size() * sizeof(double), cudaMemcpyHostToDevice), "mesh");
        } else {
            std::vector<float> wf(wd.begin(), wd.end());
            FISH_CK(c, cudaMemcpy(c->wdev[a], wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice), "mesh");
        }
    }
    c->wdev_prec = c->prec;
    c->mesh_dirty = false;
    return FISH_OK;
}

int ready(fish_ctx *c)
{
    if (!c) return FISH_ERR_ARG;
    if (!c->allocated) return fail(c, FISH_ERR_STATE, "no state set (call fish_set_state first)");
    return sync_mesh(c);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int fish_create(int nx, int ny, int nz, double gamma, int bc, fish_ctx **out)
{
    if (!out) return FISH_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !(gamma > 1.0) || (bc != FISH_BC_PERIODIC && bc != FISH_BC_OUTFLOW))
        return FISH_ERR_ARG;
    if ((long long)nx * ny * nz > (1ll << 33)) return FISH_ERR_ARG;
    fish_ctx *c = new (std::nothrow) fish_ctx;
    if (!c) return FISH_ERR_OOM;
    c->n[0] = nx;
    c->n[1] = ny;
    c->n[2] = nz;
    c->N = (long long)nx * ny * nz;
    c->gamma = gamma;
    c->bc = bc;
    c->h[0] = 1.0 / nx;
    c->h[1] = 1.0 / ny;
    c->h[2] = 1.0 / nz;
    cudaError_t e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return FISH_ERR_CUDA;
    }
    c->stream = c->own;
    *out = c;
    return FISH_OK;
}

int fish_set_option(fish_ctx *c, int key, double v)
{
    if (!c) return FISH_ERR_ARG;
    switch (key) {
    case FISH_OPT_PRECISION:
        if (v != FISH_PREC_FP64 && v != FISH_PREC_FP32) return fail(c, FISH_ERR_ARG, "bad precision");
        if (c->allocated && (int)v != c->prec) return fail(c, FISH_ERR_STATE, "precision fixed after set_state");
        c->prec = (int)v;
        break;
    case FISH_OPT_LIMITER:
        if (v != FISH_LIM_VANLEER && v != FISH_LIM_MINMOD && v != FISH_LIM_NONE && v != FISH_LIM_HYBRID)
            return fail(c, FISH_ERR_ARG, "bad limiter");
        c->lim = (int)v;
        break;
    case FISH_OPT_HSE:
        if (v != 0 && v != 1) return fail(c, FISH_ERR_ARG, "bad HSE switch");
        if (v == 1 && c->gsplit) return fail(c, FISH_ERR_ARG, "HSE correction needs unsplit gravity");
        c->hse = (int)v;
        break;
    case FISH_OPT_GRAVITY:
        if (v != FISH_GRAV_UNSPLIT && v != FISH_GRAV_SPLIT) return fail(c, FISH_ERR_ARG, "bad gravity mode");
        if (v == FISH_GRAV_SPLIT && c->hse) return fail(c, FISH_ERR_ARG, "HSE correction needs unsplit gravity");
        c->gsplit = (int)v;
        break;
    case FISH_OPT_KERNELS:
        if (v != FISH_KERNELS_COLUMN && v != FISH_KERNELS_RING) return fail(c, FISH_ERR_ARG, "bad kernel family");
        c->kernels = (int)v;
        break;
    case FISH_OPT_PRED_DISS:
        if (!(v >= 0.0 && v <= 1.0)) return fail(c, FISH_ERR_ARG, "predictor factor outside [0,1]");
        c->alpha = v;
        break;
    case FISH_OPT_DX:
    case FISH_OPT_DY:
    case FISH_OPT_DZ:
        if (!(v > 0.0) || !std::isfinite(v)) return fail(c, FISH_ERR_ARG, "cell width must be > 0");
        c->h[key - FISH_OPT_DX] = v;
        c->mesh_dirty = true;
        break;
    default:
        return fail(c, FISH_ERR_ARG, "unknown option key");
    }
    c->gdirty = true;
    c->cfl_pending = false;
    return FISH_OK;
}

int fish_set_stream(fish_ctx *c, void *s)
{
    if (!c) return FISH_ERR_ARG;
    c->stream = s ? (cudaStream_t)s : c->own;
    c->gdirty = true;
    return FISH_OK;
}

int fish_set_allocator(fish_ctx *c, void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *), void *user)
{
    if (!c) return FISH_ERR_ARG;
    if (c->allocated) return fail(c, FISH_ERR_STATE, "allocator must be set before set_state");
    if (alloc && !free_fn) return fail(c, FISH_ERR_ARG, "allocator needs a free function");
    c->ualloc = alloc;
    c->ufree = alloc ? free_fn : nullptr;
    c->uud = user;
    return FISH_OK;
}

int fish_set_state(fish_ctx *c, const double *state)
{
    if (!c || !state) return FISH_ERR_ARG;
    int r = ensure_alloc(c);
    if (r) return r;
    c->cfl_pending = false;
    c->layout = 0;
    if (c->prec == FISH_PREC_FP64) {
        for (int f = 0; f < 8; ++f)
            FISH_CK(c, cudaMemcpyAsync(field_ptr(c, f), state + (long long)f * c->N, c->N * sizeof(double),
                                       cudaMemcpyHostToDevice, c->stream),
                    "state upload");
    } else {
        if ((r = ensure_stage(c))) return r;
        for (int f = 0; f < 8; ++f)
            for (long long o = 0; o < c->N; o += kStageChunk) {
                const long long m = c->N - o < kStageChunk ? c->N - o : kStageChunk;
                FISH_CK(c, cudaMemcpyAsync(c->stage, state + (long long)f * c->N + o, m * sizeof(double),
                                           cudaMemcpyHostToDevice, c->stream),
                        "state upload");
                FISH_CK(c, Launch<float>::from_f64(c->stage, (float *)field_ptr(c, f) + o, m, c->stream), "convert");
                c->launches += 1;
            }
    }
    FISH_CK(c, cudaStreamSynchronize(c->stream), "state upload");
    return FISH_OK;
}

int fish_set_state_device(fish_ctx *c, const void *state, int dtype)
{
    if (!c || !state || (dtype != FISH_F64 && dtype != FISH_F32)) return FISH_ERR_ARG;
    int r = ensure_alloc(c);
    if (r) return r;
    c->cfl_pending = false;
    c->layout = 0;
    for (int f = 0; f < 8; ++f) {
        void *dst = field_ptr(c, f);
        if (dtype == FISH_F64) {
            const double *src = (const double *)state + (long long)f * c->N;
            if (c->prec == FISH_PREC_FP64)
                FISH_CK(c, cudaMemcpyAsync(dst, src, c->N * 8, cudaMemcpyDeviceToDevice, c->stream), "copy");
            else
                FISH_CK(c, Launch<float>::from_f64(src, (float *)dst, c->N, c->stream), "convert");
        } else {
            const float *src = (const float *)state + (long long)f * c->N;
            if (c->prec == FISH_PREC_FP32)
                FISH_CK(c, cudaMemcpyAsync(dst, src, c->N * 4, cudaMemcpyDeviceToDevice, c->stream), "copy");
            else
                FISH_CK(c, Launch<double>::from_f32(src, (double *)dst, c->N, c->stream), "convert");
        }
        c->launches += 1;
    }
    return FISH_OK;
}

int fish_set_state_host(fish_ctx *c, const void *state, int dtype)
{
    if (!c || !state || (dtype != FISH_F64 && dtype != FISH_F32)) return FISH_ERR_ARG;
    if (dtype == FISH_F64) return fish_set_state(c, (const double *)state);
    int r = ensure_alloc(c);
    if (r) return r;
    c->cfl_pending = false;
    c->layout = 0;
    if (c->prec == FISH_PREC_FP32) {
        for (int f = 0; f < 8; ++f)
            FISH_CK(c, cudaMemcpyAsync(field_ptr(c, f), (const float *)state + (long long)f * c->N,
                                       c->N * sizeof(float), cudaMemcpyHostToDevice, c->stream),
                    "state upload");
    } else {
        if ((r = ensure_stage(c))) return r;
        float *stage = (float *)c->stage;
        for (int f = 0; f < 8; ++f)
            for (long long o = 0; o < c->N; o += kStageChunk) {
                const long long m = c->N - o < kStageChunk ? c->N - o : kStageChunk;
                FISH_CK(c, cudaMemcpyAsync(stage, (const float *)state + (long long)f * c->N + o, m * sizeof(float),
                                           cudaMemcpyHostToDevice, c->stream),
                        "state upload");
                FISH_CK(c, Launch<double>::from_f32(stage, (double *)field_ptr(c, f) + o, m, c->stream), "convert");
                c->launches += 1;
            }
    }
    FISH_CK(c, cudaStreamSynchronize(c->stream), "state upload");
    return FISH_OK;
}

int fish_set_potential(fish_ctx *c, const double *phi)
{
    if (!c) return FISH_ERR_ARG;
    int r = ensure_alloc(c);
    if (r) return r;
    c->gdirty = true;
    if (!phi) {
        c->has_phi = false;
        return FISH_OK;
    }
    if (c->prec == FISH_PREC_FP64) {
        if (!c->phi && !(c->phi = dev_alloc(c, (size_t)c->N * sizeof(double))))
            return fail(c, FISH_ERR_OOM, "potential allocation failed");
        if (!c->phiT && !(c->phiT = dev_alloc(c, (size_t)c->N * sizeof(double))))
            return fail(c, FISH_ERR_OOM, "potential allocation failed");
        FISH_CK(c, cudaMemcpyAsync(c->phi, phi, c->N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "phi");
        // the x sweeps read the potential in the y-fastest layout
        const void *src[8] = {c->phi};
        void *dst[8] = {c->phiT};
        FISH_CK(c, Launch<double>::transpose((const double *const *)src, (double *const *)dst, 1, c->n[0], c->n[1],
                                             c->n[2], c->stream),
                "phi transpose");
        c->launches += 1;
        FISH_CK(c, cudaStreamSynchronize(c->stream), "phi upload");
        c->has_phi = true;
        return FISH_OK;
    }
    // FP32: per axis the difference to the next cell (periodic wrap or the
    // outflow copy of the boundary cell), formed in FP64 and rounded once, so
    // the hydrostatic estimate and the gravity source see no cancellation of
    // the stored potential; the x differences in the y-fastest layout
    for (int d = 0; d < 3; ++d)
        if (!c->phiD[d] && !(c->phiD[d] = dev_alloc(c, (size_t)c->N * sizeof(float))))
            return fail(c, FISH_ERR_OOM, "potential allocation failed");
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    const long long plane = (long long)nx * ny;
    std::vector<float> dx(plane), dy(plane), dz(plane);
    auto wrap = [&](int s, int n) { return c->bc == FISH_BC_PERIODIC ? (s >= n ? s - n : s) : (s >= n ? n - 1 : s); };
    for (int k = 0; k < nz; ++k) {
        const double *p0 = phi + (long long)k * plane;
        const double *p1 = phi + (long long)wrap(k + 1, nz) * plane;
        for (int j = 0; j < ny; ++j) {
            const int jp = wrap(j + 1, ny);
            for (int i = 0; i < nx; ++i) {
                const int ip = wrap(i + 1, nx);
                const double v = p0[(long long)j * nx + i];
                dx[(long long)i * ny + j] = (float)(p0[(long long)j * nx + ip] - v);
                dy[(long long)j * nx + i] = (float)(p0[(long long)jp * nx + i] - v);
                dz[(long long)j * nx + i] = (float)(p1[(long long)j * nx + i] - v);
            }
        }
        const long long off = (long long)k * plane;
        FISH_CK(c, cudaMemcpyAsync((float *)c->phiD[0] + off, dx.data(), plane * sizeof(float), cudaMemcpyHostToDevice,
                                   c->stream), "phi");
        FISH_CK(c, cudaMemcpyAsync((float *)c->phiD[1] + off, dy.data(), plane * sizeof(float), cudaMemcpyHostToDevice,
                                   c->stream), "phi");
        FISH_CK(c, cudaMemcpyAsync((float *)c->phiD[2] + off, dz.data(), plane * sizeof(float), cudaMemcpyHostToDevice,
                                   c->stream), "phi");
        FISH_CK(c, cudaStreamSynchronize(c->stream), "phi upload");
    }
    c->has_phi = true;
    return FISH_OK;
}

int fish_set_mesh(fish_ctx *c, const double *dx, const double *dy, const double *dz)
{
    if (!c) return FISH_ERR_ARG;
    const double *w[3] = {dx, dy, dz};
    for (int a = 0; a < 3; ++a)
        if (w[a])
            for (int i = 0; i < c->n[a]; ++i)
                if (!(w[a][i] > 0.0) || !std::isfinite(w[a][i]))
                    return fail(c, FISH_ERR_ARG, "cell widths must be finite and > 0");
    for (int a = 0; a < 3; ++a) {
        c->wmesh[a].clear();
        if (w[a]) c->wmesh[a].assign(w[a], w[a] + c->n[a]);
    }
    c->nu = dx || dy || dz;
    c->mesh_dirty = true;
    c->gdirty = true;
    c->cfl_pending = false;
    return FISH_OK;
}

int fish_cfl_dt(fish_ctx *c, double k, double *dt_out)
{
    int r = ready(c);
    if (r) return r;
    c->cfl_pending = false;
    if (!dt_out || !(k > 0.0)) return fail(c, FISH_ERR_ARG, "bad CFL arguments");
    if ((r = queue_cfl_dt(c, k, c->partial, nullptr))) return r;
    FISH_CK(c, cudaMemcpyAsync(dt_out, c->partial, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "dt");
    return check_flags(c);
}

int fish_cfl_dt_planes(fish_ctx *c, double k, int k0, int nk, double *dt_out)
{
    int r = ready(c);
    if (r) return r;
    c->cfl_pending = false;
    if (!dt_out || !(k > 0.0) || k0 < 0 || nk < 1 || k0 + nk > c->n[2])
        return fail(c, FISH_ERR_ARG, "bad CFL arguments");
    if ((r = queue_cfl_dt(c, k, c->partial, nullptr, k0, nk))) return r;
    FISH_CK(c, cudaMemcpyAsync(dt_out, c->partial, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "dt");
    return check_flags(c);
}

int fish_step(fish_ctx *c, double dt)
{
    int r = ready(c);
    if (r) return r;
    c->cfl_pending = false;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, FISH_ERR_ARG, "dt must be > 0");
    FISH_CK(c, fish::launch_set_scalar(c->dt_dev, dt, c->stream), "dt");
    FISH_CK(c, fish::launch_set_scalar(c->dt_last, dt, c->stream), "dt");
    c->launches += 2;
    return queue_sweeps(c);
}

// Capture one double step starting from the current buffers (the host's
// buffer bookkeeping is restored afterwards); the graph of parity p and the
// parity it ends on.
int capture_step(fish_ctx *c, double k, bool fused, int p)
{
    const int cu0 = c->cu, cb0 = c->cb, lay0 = c->layout;
    const long long l0 = c->launches;
    cudaStream_t cap = c->stream;
    cudaGraph_t graph = nullptr;
    FISH_CK(c, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int r;
    if (fused) {
        cudaError_t e0 = fish::launch_cfl_finish(c->minbits, k, c->dt_dev, c->dt_last, cap);
        r = e0 == cudaSuccess ? FISH_OK : cuda_fail(c, e0, "cfl finish launch");
        c->launches += 1;
    } else {
        r = queue_cfl_dt(c, k, c->dt_dev, c->dt_last);
    }
    if (!r) r = queue_sweeps(c, fused);
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    const int pend = c->cu * 2 + c->cb;
    const bool lay_ok = c->layout == lay0;
    c->cu = cu0;
    c->cb = cb0;
    c->layout = lay0;
    c->glaunches = c->launches - l0;
    c->launches = l0;  // captured, not launched
    if (r) {
        if (graph) cudaGraphDestroy(graph);
        return r;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    if (!lay_ok) {
        cudaGraphDestroy(graph);
        return fail(c, FISH_ERR_STATE, "double step does not end in its starting layout");
    }
    e = cudaGraphInstantiate(&c->gexec[p], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    c->gend[p] = pend;
    return FISH_OK;
}

int fish_step_cfl(fish_ctx *c, double k, int nsteps)
{
    int r = ready(c);
    if (r) return r;
    if (!(k > 0.0) || nsteps < 0) return fail(c, FISH_ERR_ARG, "bad arguments");
    if (nsteps == 0) return FISH_OK;
    // every replay starts (and ends) in the layout of the x sweeps
    if ((r = set_layout(c, layout_for(0)))) return r;
    const bool fused = last_sweep_fuses_cfl(c);
    if (c->gdirty || c->gk != k || c->gfused != fused) {
        for (auto &g : c->gexec)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        c->gk = k;
        c->gfused = fused;
        c->gdirty = false;
    }
    if (fused && !c->cfl_pending) {
        // the CFL minimum of the current state for the first replay
        if ((r = queue_cfl_min(c))) return r;
    }
    for (int s = 0; s < nsteps; ++s) {
        const int p = c->cu * 2 + c->cb;
        if (!c->gexec[p] && (r = capture_step(c, k, fused, p))) return r;
        FISH_CK(c, cudaGraphLaunch(c->gexec[p], c->stream), "graph launch");
        c->launches += c->glaunches;
        c->cu = c->gend[p] >> 1;
        c->cb = c->gend[p] & 1;
    }
    c->cfl_pending = fused;
    return FISH_OK;
}

int fish_last_dt(fish_ctx *c, double *dt_out)
{
    int r = ready(c);
    if (r) return r;
    if (!dt_out) return FISH_ERR_ARG;
    FISH_CK(c, cudaMemcpyAsync(dt_out, c->dt_last, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "dt");
    return check_flags(c);
}

int fish_apply(fish_ctx *c, int op, int dir, double dt)
{
    int r = ready(c);
    if (r) return r;
    c->cfl_pending = false;
    if ((op != FISH_OP_FLUID && op != FISH_OP_CT) || dir < 0 || dir > 2 || !(dt > 0.0))
        return fail(c, FISH_ERR_ARG, "bad operator arguments");
    FISH_CK(c, fish::launch_set_scalar(c->dt_dev, dt, c->stream), "dt");
    c->launches += 1;
    return apply_op(c, op, dir);
}

int fish_get_state(fish_ctx *c, double *state)
{
    int r = ready(c);
    if (r) return r;
    if (!state) return FISH_ERR_ARG;
    if ((r = set_layout(c, 0))) return r;
    if (c->prec == FISH_PREC_FP64) {
        for (int f = 0; f < 8; ++f)
            FISH_CK(c, cudaMemcpyAsync(state + (long long)f * c->N, field_ptr(c, f), c->N * sizeof(double),
                                       cudaMemcpyDeviceToHost, c->stream),
                    "state download");
    } else {
        if ((r = ensure_stage(c))) return r;
        for (int f = 0; f < 8; ++f)
            for (long long o = 0; o < c->N; o += kStageChunk) {
                const long long m = c->N - o < kStageChunk ? c->N - o : kStageChunk;
                FISH_CK(c, Launch<float>::to_f64((const float *)field_ptr(c, f) + o, c->stage, m, c->stream),
                        "convert");
                c->launches += 1;
                FISH_CK(c, cudaMemcpyAsync(state + (long long)f * c->N + o, c->stage, m * sizeof(double),
                                           cudaMemcpyDeviceToHost, c->stream),
                        "state download");
            }
    }
    return check_flags(c);
}

int fish_get_state_host(fish_ctx *c, void *state, int dtype)
{
    if (!c || !state || (dtype != FISH_F64 && dtype != FISH_F32)) return FISH_ERR_ARG;
    if (dtype == FISH_F64) return fish_get_state(c, (double *)state);
    int r = ready(c);
    if (r) return r;
    if ((r = set_layout(c, 0))) return r;
    if (c->prec == FISH_PREC_FP32) {
        for (int f = 0; f < 8; ++f)
            FISH_CK(c, cudaMemcpyAsync((float *)state + (long long)f * c->N, field_ptr(c, f), c->N * sizeof(float),
                                       cudaMemcpyDeviceToHost, c->stream),
                    "state download");
    } else {
        if ((r = ensure_stage(c))) return r;
        float *stage = (float *)c->stage;
        for (int f = 0; f < 8; ++f)
            for (long long o = 0; o < c->N; o += kStageChunk) {
                const long long m = c->N - o < kStageChunk ? c->N - o : kStageChunk;
                FISH_CK(c, Launch<double>::to_f32((const double *)field_ptr(c, f) + o, stage, m, c->stream),
                        "convert");
                c->launches += 1;
                FISH_CK(c, cudaMemcpyAsync((float *)state + (long long)f * c->N + o, stage, m * sizeof(float),
                                           cudaMemcpyDeviceToHost, c->stream),
                        "state download");
            }
    }
    return check_flags(c);
}

int fish_get_state_device(fish_ctx *c, void *state, int dtype)
{
    int r = ready(c);
    if (r) return r;
    if (!state || (dtype != FISH_F64 && dtype != FISH_F32)) return FISH_ERR_ARG;
    if ((r = set_layout(c, 0))) return r;
    for (int f = 0; f < 8; ++f) {
        const void *src = field_ptr(c, f);
        if (dtype == FISH_F64) {
            double *dst = (double *)state + (long long)f * c->N;
            if (c->prec == FISH_PREC_FP64)
                FISH_CK(c, cudaMemcpyAsync(dst, src, c->N * 8, cudaMemcpyDeviceToDevice, c->stream), "copy");
            else
                FISH_CK(c, Launch<float>::to_f64((const float *)src, dst, c->N, c->stream), "convert");
        } else {
            float *dst = (float *)state + (long long)f * c->N;
            if (c->prec == FISH_PREC_FP32)
                FISH_CK(c, cudaMemcpyAsync(dst, src, c->N * 4, cudaMemcpyDeviceToDevice, c->stream), "copy");
            else
                FISH_CK(c, Launch<double>::to_f32((const double *)src, dst, c->N, c->stream), "convert");
        }
        c->launches += 1;
    }
    return FISH_OK;
}

// z-planes [k0, k0+nk) of all 8 fields to / from a buffer laid out field
// by field, each field's planes contiguous (a z-plane is contiguous in both
// memory layouts: z is the slowest axis); the values stay in the context's
// precision and current layout.
int planes_check(fish_ctx *c, int k0, int nk, const void *buf)
{
    int r = ready(c);
    if (r) return r;
    if (!buf || nk < 0 || k0 < 0 || k0 + nk > c->n[2]) return fail(c, FISH_ERR_ARG, "bad plane range");
    return FISH_OK;
}

int fish_get_planes(fish_ctx *c, int k0, int nk, void *dst)
{
    int r = planes_check(c, k0, nk, dst);
    if (r) return r;
    const size_t es = esize(c), plane = (size_t)c->n[0] * c->n[1];
    for (int f = 0; f < 8; ++f)
        FISH_CK(c, cudaMemcpyAsync((char *)dst + (size_t)f * nk * plane * es,
                                   (const char *)field_ptr(c, f) + (size_t)k0 * plane * es, (size_t)nk * plane * es,
                                   cudaMemcpyDefault, c->stream),
                "plane copy");
    return FISH_OK;
}

int fish_set_planes(fish_ctx *c, int k0, int nk, const void *src)
{
    int r = planes_check(c, k0, nk, src);
    if (r) return r;
    const size_t es = esize(c), plane = (size_t)c->n[0] * c->n[1];
    for (int f = 0; f < 8; ++f)
        FISH_CK(c, cudaMemcpyAsync((char *)field_ptr(c, f) + (size_t)k0 * plane * es,
                                   (const char *)src + (size_t)f * nk * plane * es, (size_t)nk * plane * es,
                                   cudaMemcpyDefault, c->stream),
                "plane copy");
    c->cfl_pending = false;  // the state changed outside a graph replay
    return FISH_OK;
}

int fish_diagnostics(fish_ctx *c, double out[9])
{
    int r = ready(c);
    if (r) return r;
    if (!out) return FISH_ERR_ARG;
    const Geom g = geom(c);
    if (c->prec == FISH_PREC_FP64) {
        const double *in[8];
        for (int f = 0; f < 8; ++f) in[f] = (const double *)field_ptr(c, f);
        FISH_CK(c, Launch<double>::diag(in, g, c->h, c->partial, kDiagBlocks, c->stream, mesh_of<double>(c).get()),
                "diag launch");
    } else {
        const float *in[8];
        for (int f = 0; f < 8; ++f) in[f] = (const float *)field_ptr(c, f);
        FISH_CK(c, Launch<float>::diag(in, g, c->h, c->partial, kDiagBlocks, c->stream, mesh_of<float>(c).get()),
                "diag launch");
    }
    c->launches += 1;
    std::vector<double> part((size_t)9 * kDiagBlocks);
    FISH_CK(c, cudaMemcpyAsync(part.data(), c->partial, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream),
            "diag download");
    FISH_CK(c, cudaStreamSynchronize(c->stream), "diag");
    // an irregular mesh weights each cell by its volume in the kernel
    const double vol = c->nu ? 1.0 : c->h[0] * c->h[1] * c->h[2];
    for (int f = 0; f < 9; ++f) out[f] = 0.0;
    for (int b = 0; b < kDiagBlocks; ++b) {
        for (int f = 0; f < 8; ++f) out[f] += part[(size_t)b * 9 + f];
        out[8] = std::fmax(out[8], part[(size_t)b * 9 + 8]);
    }
    for (int f = 0; f < 8; ++f) out[f] *= vol;
    return check_flags(c);
}

int fish_sync(fish_ctx *c)
{
    if (!c) return FISH_ERR_ARG;
    if (!c->allocated) {
        FISH_CK(c, cudaStreamSynchronize(c->stream), "sync");
        return FISH_OK;
    }
    return check_flags(c);
}

int fish_clear_error(fish_ctx *c)
{
    if (!c) return FISH_ERR_ARG;
    c->err.clear();
    if (c->allocated) {
        FISH_CK(c, cudaMemsetAsync(c->flags, 0, sizeof(unsigned), c->stream), "clear");
        FISH_CK(c, cudaStreamSynchronize(c->stream), "clear");
    }
    return FISH_OK;
}

const char *fish_last_error(fish_ctx *c) { return c ? c->err.c_str() : "null context"; }

long long fish_launch_count(fish_ctx *c) { return c ? c->launches : -1; }

int fish_probe_fp64_fma(double *fma_per_s)
{
    if (!fma_per_s) return FISH_ERR_ARG;
    *fma_per_s = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        (void)cudaGetLastError();
        return FISH_ERR_CUDA;
    }
    const int blocks = sms * 8, iters = 4096;
    double *buf = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FISH_ERR_CUDA;
    float ms = 0.0f;
    if (cudaMalloc(&buf, (size_t)blocks * 256 * sizeof(double)) != cudaSuccess) goto done;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) goto done;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    if (fish::launch_dfma_probe(buf, blocks, iters, s) != cudaSuccess) goto done;  // warm-up
    if (cudaEventRecord(e0, s) != cudaSuccess) goto done;
    for (int r = 0; r < 3; ++r)
        if (fish::launch_dfma_probe(buf, blocks, iters, s) != cudaSuccess) goto done;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) goto done;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f)) goto done;
    *fma_per_s = 3.0 * (double)blocks * 256.0 * 8.0 * iters / (ms * 1e-3);
    rc = FISH_OK;
done:
    if (rc != FISH_OK) (void)cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (buf) cudaFree(buf);
    return rc;
}

void fish_destroy(fish_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto g : c->gexec)
        if (g) cudaGraphExecDestroy(g);
    dev_free_all(c);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
}

}  // extern "C"
