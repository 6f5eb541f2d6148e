/*
 * fish_oracle.c -- plain FP64 CPU oracle of FISH's operator-split MHD step
 * (Kaeppeli et al., "FISH: A 3D parallel MHD code for astrophysical
 * applications", arXiv:0910.2854).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path in
 * paper_0910_2854_gb300/csrc and must never be called by the product path.
 *
 * The code follows the paper's steps in the paper's order, one pencil at a
 * time, with no blocking, fusion or reordering:
 *   - state: cell averages u = (rho, rho v, E) (eq0070) and face averages of
 *     b stored as the "right" face of each cell (eq0080, eq0080a, eq0080b);
 *   - composition: Strang-symmetric palindrome of the directional fluid
 *     operators L_d and magnetic operators B_d (eq0081-eq0082, reading C-4);
 *   - L_d: relaxing-TVD fluid sweep (eq0090-eq0240), with unsplit gravity
 *     (eq0253-eq0255) and the hydrostatic-gradient correction
 *     (eq0321-eq03261);
 *   - B_d: constrained transport (eq0330-eq0364);
 *   - CFL time step (eq0083-eq0084);
 *   - irregular Cartesian meshes (Sec. 2.5, eq037, eq0420): cell widths per
 *     axis, readings C-23 .. C-27.
 * Equations are cited by the paper's LaTeX labels.
 * Where the paper is silent, garbled or inconsistent, the reading used is
 * named C-n in the comments; each is listed with its justification in the
 * design notes of the repository.
 *
 * Precision: IEEE double throughout, compiled with -ffp-contract=off so that
 * no multiply-add is fused behind the reader's back.
 *
 * Layout: 8 fields of nx*ny*nz doubles each, x fastest,
 * index = i + nx*(j + ny*k):  rho, m_x, m_y, m_z, E, b_x, b_y, b_z, where
 * b_x[i,j,k] is the face average at x_{i+1/2} (likewise b_y at y_{j+1/2},
 * b_z at z_{k+1/2}).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_NG 4 /* ghost cells gathered at each pencil end */

enum { OR_LIM_VANLEER = 0, OR_LIM_MINMOD = 1, OR_LIM_NONE = 2, OR_LIM_HYBRID = 3 };
enum { OR_BC_PERIODIC = 0, OR_BC_OUTFLOW = 1 };
enum { OR_FLAG_RHO = 1, OR_FLAG_P = 2, OR_FLAG_NAN = 4 };

/* Problem description passed from Python (ctypes mirror in oracle/__init__.py). */
typedef struct {
    int n[3];            /* nx, ny, nz (each >= 1) */
    double h[3];         /* dx, dy, dz */
    double gamma;        /* ratio of specific heats, eq0050 */
    int bc;              /* OR_BC_* */
    int limiter;         /* OR_LIM_* (eq0190, eq0200) */
    int hse;             /* 1: hydrostatic-gradient correction (eq0321-eq03261) */
    double pred_diss;    /* predictor freezing-speed factor in [0,1] (Sec. 2.2, predictor step) */
    const double *phi;   /* NULL or cell-centred potential, nx*ny*nz */
    int gravity_split;   /* 1: operator-split gravity G(dt/2) L G(dt/2) (eq025111-eq02513) */
    const double *w[3];  /* NULL (uniform h[d]) or the n[d] cell widths along axis d (eq037) */
} or_problem;

/* ------------------------------------------------------------------------ */
/* index helpers                                                             */
/* ------------------------------------------------------------------------ */

/* Ghost index map of a cell (or stored face) coordinate s along an axis of
 * n cells: periodic wrap, or zeroth-order extrapolation (clamp) for outflow
 * (Sec. 4, two-dimensional MHD Riemann problem: zeroth-order
 * extrapolation; reading C-14 for faces). */
static long or_map(long s, long n, int bc)
{
    if (bc == OR_BC_PERIODIC) {
        long r = s % n;
        return r < 0 ? r + n : r;
    }
    if (s < 0) return 0;
    if (s >= n) return n - 1;
    return s;
}

/* Width of cell s along axis d: a ghost has the width of the cell it copies
 * (the periodic image, or the boundary cell for outflow; reading C-23). */
static double or_width(const or_problem *P, int d, long s)
{
    return P->w[d] ? P->w[d][or_map(s, P->n[d], P->bc)] : P->h[d];
}

/* Distance between the centres of cells s-1 and s+1 along d (the centred
 * potential difference, eq02513, on an irregular mesh; reading C-26). */
static double or_centre_span(const or_problem *P, int d, long s)
{
    if (!P->w[d]) return 2.0 * P->h[d];
    return 0.5 * or_width(P, d, s - 1) + or_width(P, d, s) + 0.5 * or_width(P, d, s + 1);
}

static long or_index(const or_problem *P, long c0, long c1, long c2)
{
    long i = or_map(c0, P->n[0], P->bc);
    long j = or_map(c1, P->n[1], P->bc);
    long k = or_map(c2, P->n[2], P->bc);
    return i + (long)P->n[0] * (j + (long)P->n[1] * k);
}

/* Coordinate triple (x,y,z) of the point that is s along the sweep axis d
 * and (a, b) along the two transverse axes t1 = d+1, t2 = d+2 (cyclic). */
static void or_coords(int d, long s, long a, long b, long c[3])
{
    c[d] = s;
    c[(d + 1) % 3] = a;
    c[(d + 2) % 3] = b;
}

static long or_index_dir(const or_problem *P, int d, long s, long a, long b)
{
    long c[3];
    or_coords(d, s, a, b, c);
    return or_index(P, c[0], c[1], c[2]);
}

/* ------------------------------------------------------------------------ */
/* limiters eq0190-eq0200, with sign(0) = 0 (reading C-8)                    */
/* ------------------------------------------------------------------------ */

static double or_sign(double a) { return a > 0.0 ? 1.0 : (a < 0.0 ? -1.0 : 0.0); }

static double or_minmod(double a, double b)
{
    return 0.5 * (or_sign(a) + or_sign(b)) * fmin(fabs(a), fabs(b));
}

static double or_vanleer(double a, double b)
{
    /* eq0200: (1/2)(sign a + sign b) * 2ab/(a+b); the prefactor vanishes
     * unless a and b have the same (nonzero) sign, and then a+b != 0. */
    if (a * b > 0.0) return 2.0 * a * b / (a + b);
    return 0.0;
}

static double or_limit(int lim, double a, double b)
{
    if (lim == OR_LIM_MINMOD) return or_minmod(a, b);
    if (lim == OR_LIM_NONE) return 0.0;
    return or_vanleer(a, b);
}

/* ------------------------------------------------------------------------ */
/* cell quantities in the frame of the sweep: component 0 is along the sweep */
/* ------------------------------------------------------------------------ */

typedef struct {
    double u[5];   /* rho, m_n, m_t1, m_t2, E */
    double F[5];   /* flux vector, eq0100 */
    double p;      /* gas pressure, eq0050 with E = rho e + rho v^2/2 + b^2/2 */
    double cs;     /* sound speed */
    double cf;     /* fast magnetosonic speed along the sweep (reading C-1) */
    double vn;     /* velocity along the sweep */
    double d;      /* freezing speed |v_n| + c_F, label 0111 */
} or_cell;

/* Primitive quantities, flux (eq0100) and freezing speed (label 0111) of one
 * cell, given its conserved state u and its cell-centred field bb (the
 * magnetic field is held constant during L_d and interpolated to the cell
 * centre, Sec. 2.2; reading C-11). */
static void or_cell_eval(const or_problem *P, const double u[5], const double bb[3],
                         or_cell *c, int *flags)
{
    const double g = P->gamma;
    double rho = u[0];
    double v0, v1, v2, kin, mag, p, ptot, a2, bt2, bn2, B2, disc, bv;
    int k;
    for (k = 0; k < 5; ++k) c->u[k] = u[k];
    v0 = u[1] / rho;
    v1 = u[2] / rho;
    v2 = u[3] / rho;
    kin = 0.5 * (u[1] * v0 + u[2] * v1 + u[3] * v2);
    mag = 0.5 * (bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
    p = (g - 1.0) * (u[4] - kin - mag);                     /* eq0050 */
    ptot = p + mag;                                          /* P_tot = p + b^2/2 */
    a2 = g * p / rho;                                        /* c_S^2 */
    bn2 = bb[0] * bb[0] / rho;
    bt2 = (bb[1] * bb[1] + bb[2] * bb[2]) / rho;
    B2 = bn2 + bt2;
    /* c_F^2 = ((a^2 + B^2) + sqrt((a^2 + B^2)^2 - 4 a^2 b_n^2)) / 2, with the
     * discriminant written as (a^2 - B^2)^2 + 4 a^2 b_t^2 >= 0 (reading C-1). */
    disc = (a2 - B2) * (a2 - B2) + 4.0 * a2 * bt2;
    c->cf = sqrt(0.5 * (a2 + B2 + sqrt(disc)));
    c->cs = sqrt(a2);
    c->p = p;
    c->vn = v0;
    c->d = fabs(v0) + c->cf;                                 /* label 0111 */
    bv = bb[0] * v0 + bb[1] * v1 + bb[2] * v2;
    c->F[0] = u[1];                                          /* eq0100 */
    c->F[1] = u[1] * v0 + ptot - bb[0] * bb[0];
    c->F[2] = u[2] * v0 - bb[0] * bb[1];
    c->F[3] = u[3] * v0 - bb[0] * bb[2];
    c->F[4] = (u[4] + ptot) * v0 - bb[0] * bv;
    if (!(rho > 0.0)) *flags |= OR_FLAG_RHO;
    if (!(p > 0.0)) *flags |= OR_FLAG_P;
    if (rho != rho || p != p || c->cf != c->cf) *flags |= OR_FLAG_NAN;
}

/* Hydrostatic-gradient estimate g_e between cells a and b (eq0321) and the
 * HSE-corrected difference delta u (eq0323).  xi = -(rho, m, E + p)
 * (eq0320); c_S as printed (reading C-3). */
static void or_hse_delta(const or_cell *a, const or_cell *b, double phia, double phib,
                         double du[5], double ddu[5])
{
    double xa[5], xb[5], fac;
    int k;
    xa[0] = -a->u[0]; xa[1] = -a->u[1]; xa[2] = -a->u[2]; xa[3] = -a->u[3];
    xa[4] = -(a->u[4] + a->p);
    xb[0] = -b->u[0]; xb[1] = -b->u[1]; xb[2] = -b->u[2]; xb[3] = -b->u[3];
    xb[4] = -(b->u[4] + b->p);
    fac = (phib - phia) / (a->cs * b->cs);
    for (k = 0; k < 5; ++k) {
        double gk = 0.5 * (xb[k] + xa[k]) * fac;
        du[k] = b->u[k] - a->u[k];                            /* eq0323 */
        ddu[k] = or_minmod(du[k] - gk, du[k]);                /* eq0323 */
    }
}

/* First-order interface flux between cells a (left) and b (right).
 *   hse == 0: eq0140 with the freezing speed D = alpha * max(d_a, d_b)
 *             (eq0150; alpha = predictor freezing-speed factor).
 *   hse == 1: eq0324 with D_adv = max(|v_a|,|v_b|) (eq0325, reading C-3)
 *             and D_ac = max(c_F,a, c_F,b) (eq03261), both scaled by alpha. */
static void or_flux1(const or_problem *P, const or_cell *a, const or_cell *b,
                     double phia, double phib, double alpha, double F[5])
{
    int k;
    if (!P->hse) {
        double D = alpha * fmax(a->d, b->d);
        for (k = 0; k < 5; ++k)
            F[k] = 0.5 * (a->F[k] + b->F[k]) - 0.5 * D * (b->u[k] - a->u[k]);
    } else {
        double du[5], ddu[5];
        double Dadv = alpha * fmax(fabs(a->vn), fabs(b->vn));
        double Dac = alpha * fmax(a->cf, b->cf);
        or_hse_delta(a, b, phia, phib, du, ddu);
        for (k = 0; k < 5; ++k)
            F[k] = 0.5 * (a->F[k] + b->F[k]) - 0.5 * Dadv * du[k] - 0.5 * Dac * ddu[k];
    }
}

/* Second-order TVD flux at the interface between cells c1 = e and c2 = e+1
 * from the predicted cells c0..c3 = e-1 .. e+2 (eq0160-eq0230).
 *
 * Without HSE the split fluxes are F+ = (F + D u)/2 and F- = (F - D u)/2
 * (eq0130) with one freezing speed D = max(d_e, d_{e+1}) of this interface
 * for every cell of the stencil (reading C-2); the left/right differences
 * (eq0170, eq0210) are limited (eq0180, eq0220) and combined as eq0230, in which
 * the Delta x factors cancel:
 *   F = F+_e + F-_{e+1} + (1/2)[phi(F+_e - F+_{e-1}, F+_{e+1} - F+_e)
 *                              - phi(F-_{e+1} - F-_e, F-_{e+2} - F-_{e+1})].
 *
 * With HSE the dissipative part of each difference, D (u_{j+1} - u_j), is
 * replaced by its HSE-corrected form D_adv Delta u_j + D_ac delta u_j of
 * eq0324, with the speeds of this interface (reading C-19: "the second
 * order fluxes are constructed in the same way ... but with the HSE
 * corrected first order fluxes"). */
static void or_flux2(const or_problem *P, const or_cell *c0, const or_cell *c1,
                     const or_cell *c2, const or_cell *c3, const double ph[4], const double *dw,
                     double F[5])
{
    int k;
    /* irregular mesh (reading C-25): each one-sided difference is divided by
     * the distance between the centres it joins and the limited slope is
     * carried over half the width of its own cell (c1 for F+, c2 for F-);
     * uniform widths reduce this to eq0230 */
    double sp = 1.0, sm = 1.0, gl = 1.0, gc = 1.0, gr = 1.0;
    if (dw) {
        sp = dw[1];
        sm = dw[2];
        gl = 0.5 * (dw[0] + dw[1]);
        gc = 0.5 * (dw[1] + dw[2]);
        gr = 0.5 * (dw[2] + dw[3]);
    }
    /* hybrid limiter (Sec. 2.2, after eq0200): Van Leer where the flow is
     * subsonic, minmod where it is supersonic; decided per interface from the
     * two cells that share it (reading C-21) */
    int lim = P->limiter;
    if (lim == OR_LIM_HYBRID)
        lim = (fabs(c1->vn) > c1->cs || fabs(c2->vn) > c2->cs) ? OR_LIM_MINMOD : OR_LIM_VANLEER;
    if (!P->hse) {
        double D = fmax(c1->d, c2->d);
        for (k = 0; k < 5; ++k) {
            double fp0 = 0.5 * (c0->F[k] + D * c0->u[k]);
            double fp1 = 0.5 * (c1->F[k] + D * c1->u[k]);
            double fp2 = 0.5 * (c2->F[k] + D * c2->u[k]);
            double fm1 = 0.5 * (c1->F[k] - D * c1->u[k]);
            double fm2 = 0.5 * (c2->F[k] - D * c2->u[k]);
            double fm3 = 0.5 * (c3->F[k] - D * c3->u[k]);
            double slp, slm;
            if (!dw) {
                slp = or_limit(lim, fp1 - fp0, fp2 - fp1);   /* eq0180 */
                slm = or_limit(lim, fm2 - fm1, fm3 - fm2);   /* eq0220 */
            } else {
                slp = sp * or_limit(lim, (fp1 - fp0) / gl, (fp2 - fp1) / gc);
                slm = sm * or_limit(lim, (fm2 - fm1) / gc, (fm3 - fm2) / gr);
            }
            F[k] = fp1 + fm2 + 0.5 * (slp - slm);                      /* eq0230 */
        }
    } else {
        double Dadv = fmax(fabs(c1->vn), fabs(c2->vn));
        double Dac = fmax(c1->cf, c2->cf);
        double du0[5], dd0[5], du1[5], dd1[5], du2[5], dd2[5];
        or_hse_delta(c0, c1, ph[0], ph[1], du0, dd0);
        or_hse_delta(c1, c2, ph[1], ph[2], du1, dd1);
        or_hse_delta(c2, c3, ph[2], ph[3], du2, dd2);
        for (k = 0; k < 5; ++k) {
            double q0 = Dadv * du0[k] + Dac * dd0[k];
            double q1 = Dadv * du1[k] + Dac * dd1[k];
            double q2 = Dadv * du2[k] + Dac * dd2[k];
            double fp_l = 0.5 * ((c1->F[k] - c0->F[k]) + q0);  /* F+_e - F+_{e-1}    */
            double fp_r = 0.5 * ((c2->F[k] - c1->F[k]) + q1);  /* F+_{e+1} - F+_e    */
            double fm_l = 0.5 * ((c2->F[k] - c1->F[k]) - q1);  /* F-_{e+1} - F-_e    */
            double fm_r = 0.5 * ((c3->F[k] - c2->F[k]) - q2);  /* F-_{e+2} - F-_{e+1} */
            double slp, slm;
            if (!dw) {
                slp = or_limit(lim, fp_l, fp_r);
                slm = or_limit(lim, fm_l, fm_r);
            } else {
                slp = sp * or_limit(lim, fp_l / gl, fp_r / gc);
                slm = sm * or_limit(lim, fm_l / gc, fm_r / gr);
            }
            F[k] = 0.5 * (c1->F[k] + c2->F[k]) - 0.5 * q1 + 0.5 * (slp - slm);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* L_d on one pencil                                                         */
/* ------------------------------------------------------------------------ */

/* Scratch for one pencil of n cells plus OR_NG ghosts at each end. */
typedef struct {
    long cap;
    double *u, *bb, *ph;         /* [5][m], [3][m], [m] */
    or_cell *c0, *c1;            /* raw and predicted cell evaluations, [m] */
    double *F1;                  /* predictor fluxes, [5][m] */
    double *up;                  /* predicted states, [5][m] */
    double *F2;                  /* corrector fluxes, [5][m] */
    double *vt, *bf, *w, *f1, *bp, *wp, *f2, *vh; /* constrained transport, [m] each */
    double *dw;                  /* cell widths along the pencil, [m] */
} or_scratch;

static int or_scratch_init(or_scratch *s, long n)
{
    long m = n + 2 * OR_NG;
    memset(s, 0, sizeof(*s));
    s->cap = n;
    s->u = (double *)calloc(5 * m, sizeof(double));
    s->bb = (double *)calloc(3 * m, sizeof(double));
    s->ph = (double *)calloc(m, sizeof(double));
    s->c0 = (or_cell *)calloc(m, sizeof(or_cell));
    s->c1 = (or_cell *)calloc(m, sizeof(or_cell));
    s->F1 = (double *)calloc(5 * m, sizeof(double));
    s->up = (double *)calloc(5 * m, sizeof(double));
    s->F2 = (double *)calloc(5 * m, sizeof(double));
    s->vt = (double *)calloc(m, sizeof(double));
    s->bf = (double *)calloc(m, sizeof(double));
    s->w = (double *)calloc(m, sizeof(double));
    s->f1 = (double *)calloc(m, sizeof(double));
    s->bp = (double *)calloc(m, sizeof(double));
    s->wp = (double *)calloc(m, sizeof(double));
    s->f2 = (double *)calloc(m, sizeof(double));
    s->vh = (double *)calloc(m, sizeof(double));
    s->dw = (double *)calloc(m, sizeof(double));
    return (s->u && s->bb && s->ph && s->c0 && s->c1 && s->F1 && s->up && s->F2 && s->vt &&
            s->bf && s->w && s->f1 && s->bp && s->wp && s->f2 && s->vh && s->dw) ? 0 : -1;
}

static void or_scratch_free(or_scratch *s)
{
    free(s->u); free(s->bb); free(s->ph); free(s->c0); free(s->c1); free(s->F1);
    free(s->up); free(s->F2); free(s->vt); free(s->bf); free(s->w); free(s->f1);
    free(s->bp); free(s->wp); free(s->f2); free(s->vh); free(s->dw);
}

/* Fluid operator L_d(dt) for the pencil along axis d at transverse position
 * (a, b): gather with ghosts, run predictor (eq0253) and corrector
 * (eq0255), scatter the n interior cells back.  Returns flags. */
static int or_fluid_pencil(const or_problem *P, double *const *q, int d, long a, long b,
                           double dt, or_scratch *S)
{
    const long n = P->n[d];
    const long m = n + 2 * OR_NG;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const double hd = P->h[d];
    const double alpha = P->pred_diss;
    const int grav = P->phi != NULL && !P->gravity_split;  /* unsplit source terms */
    const int nu = P->w[d] != NULL;                          /* irregular mesh along d */
    int flags = 0;
    long e;
    int k;
    double *u = S->u, *bb = S->bb, *ph = S->ph, *dw = S->dw;

    for (e = 0; e < m; ++e) dw[e] = or_width(P, d, e - OR_NG);

    /* gather: conserved state in the sweep frame and the cell-centred field
     * b_bar_c = (b_c at face c-1/2 + b_c at face c+1/2)/2 along each axis c */
    for (e = 0; e < m; ++e) {
        long s = e - OR_NG, c[3], idx;
        or_coords(d, s, a, b, c);
        idx = or_index(P, c[0], c[1], c[2]);
        u[0 * m + e] = q[0][idx];
        u[1 * m + e] = q[1 + d][idx];
        u[2 * m + e] = q[1 + t1][idx];
        u[3 * m + e] = q[1 + t2][idx];
        u[4 * m + e] = q[4][idx];
        {
            /* For outflow a ghost cell copies the nearest interior cell as a
             * whole, its cell-centred field included: evaluate at the mapped
             * cell cc. */
            long cc[3], cm[3];
            double bc3[3];
            int ax, z;
            for (z = 0; z < 3; ++z) cc[z] = or_map(c[z], P->n[z], P->bc);
            for (ax = 0; ax < 3; ++ax) {
                cm[0] = cc[0]; cm[1] = cc[1]; cm[2] = cc[2];
                cm[ax] -= 1;
                bc3[ax] = 0.5 * (q[5 + ax][or_index(P, cm[0], cm[1], cm[2])] + q[5 + ax][idx]);
            }
            bb[0 * m + e] = bc3[d];
            bb[1 * m + e] = bc3[t1];
            bb[2 * m + e] = bc3[t2];
        }
        ph[e] = grav ? P->phi[idx] : 0.0;
    }

    /* raw cell evaluations */
    for (e = 0; e < m; ++e) {
        double ue[5], be[3];
        for (k = 0; k < 5; ++k) ue[k] = u[k * m + e];
        for (k = 0; k < 3; ++k) be[k] = bb[k * m + e];
        or_cell_eval(P, ue, be, &S->c0[e], &flags);
    }

    /* predictor fluxes at interfaces (e, e+1), e = 0 .. m-2 (eq0140 / eq0324) */
    for (e = 0; e + 1 < m; ++e) {
        double F[5];
        or_flux1(P, &S->c0[e], &S->c0[e + 1], ph[e], ph[e + 1], alpha, F);
        for (k = 0; k < 5; ++k) S->F1[k * m + e] = F[k];
    }

    /* predicted half-step states for cells e = 1 .. m-2 (eq0253 with the
     * source of eq0254, sign as reading C-6) */
    for (e = 1; e + 1 < m; ++e) {
        double up[5], be[3];
        const double he = nu ? dw[e] : hd;                   /* eq037: the cell's own width */
        for (k = 0; k < 5; ++k)
            up[k] = u[k * m + e] - dt / (2.0 * he) * (S->F1[k * m + e] - S->F1[k * m + e - 1]);
        if (grav) {
            double dphi = (ph[e + 1] - ph[e - 1]) / or_centre_span(P, d, e - OR_NG);
            up[1] = up[1] - 0.5 * dt * u[0 * m + e] * dphi;
            up[4] = up[4] - 0.5 * dt * u[1 * m + e] * dphi;
        }
        for (k = 0; k < 5; ++k) S->up[k * m + e] = up[k];
        for (k = 0; k < 3; ++k) be[k] = bb[k * m + e];
        or_cell_eval(P, up, be, &S->c1[e], &flags);
    }

    /* corrector fluxes at interfaces (e, e+1) for e = OR_NG-1 .. OR_NG+n-1,
     * from predicted cells e-1 .. e+2 (eq0230) */
    for (e = OR_NG - 1; e < OR_NG + n; ++e) {
        double F[5];
        or_flux2(P, &S->c1[e - 1], &S->c1[e], &S->c1[e + 1], &S->c1[e + 2], &ph[e - 1],
                 nu ? &dw[e - 1] : NULL, F);
        for (k = 0; k < 5; ++k) S->F2[k * m + e] = F[k];
    }

    /* full-step update (eq0240 / eq0255) of the interior cells, scatter */
    for (e = OR_NG; e < OR_NG + n; ++e) {
        double un[5];
        long idx = or_index_dir(P, d, e - OR_NG, a, b);
        const double he = nu ? dw[e] : hd;
        for (k = 0; k < 5; ++k)
            un[k] = u[k * m + e] - dt / he * (S->F2[k * m + e] - S->F2[k * m + e - 1]);
        if (grav) {
            double dphi = (ph[e + 1] - ph[e - 1]) / or_centre_span(P, d, e - OR_NG);
            un[1] = un[1] - dt * S->up[0 * m + e] * dphi;
            un[4] = un[4] - dt * S->up[1 * m + e] * dphi;
        }
        q[0][idx] = un[0];
        q[1 + d][idx] = un[1];
        q[1 + t1][idx] = un[2];
        q[1 + t2][idx] = un[3];
        q[4][idx] = un[4];
    }
    return flags;
}

/* ------------------------------------------------------------------------ */
/* B_d: constrained transport                                                */
/* ------------------------------------------------------------------------ */

/* Edge fluxes of the face pencil that carries the transverse component
 * b_c (c = t1 or t2) along the sweep axis d, at transverse face index fc
 * (face fc+1/2 along c) and cell index fo along the other transverse axis.
 * On return f[s + 1] is the flux at interface s' = s+1/2, s = -1 .. n-1.
 * Steps: face velocity (eq0361-eq0362), edge velocity (eq0364), upwind
 * first-order flux of the cell products (eq0363, reading C-7), predictor
 * half step, TVD corrector flux with the fluid's limiter (reading C-10). */
/* Edge velocity at the interface between pencil cells e and e+1 (eq0364):
 * the mean of the two smoothed face velocities, or on an irregular mesh
 * their linear interpolation to the interface (reading C-27). */
static double or_edge_velocity(int nu, double va, double vb, double wa, double wb)
{
    if (!nu) return 0.5 * (va + vb);
    return (wb * va + wa * vb) / (wa + wb);
}

static void or_ct_face_pencil(const or_problem *P, double *const *q, int d, int c, long fc,
                              long fo, double dt, or_scratch *S, double *f)
{
    const long n = P->n[d];
    const long m = n + 2 * OR_NG;
    const int o = 3 - d - c; /* the remaining axis */
    const double hd = P->h[d];
    const int nu = P->w[d] != NULL;
    double *vt = S->vt, *bf = S->bf, *vh = S->vh, *w = S->w, *f1 = S->f1, *bp = S->bp,
           *wp = S->wp, *f2 = S->f2, *dw = S->dw;
    /* irregular mesh along c: the face velocity is the linear interpolation
     * of the two cell velocities to the face (reading C-27) */
    const double wA = or_width(P, c, fc), wB = or_width(P, c, fc + 1);
    long e;

    for (e = 0; e < m; ++e) dw[e] = or_width(P, d, e - OR_NG);

    for (e = 0; e < m; ++e) {
        long s = e - OR_NG, cA[3], cB[3], iA, iB, iF;
        /* cells on either side of the face along c: fc and fc+1 */
        cA[d] = s; cA[c] = fc; cA[o] = fo;
        cB[d] = s; cB[c] = fc + 1; cB[o] = fo;
        iA = or_index(P, cA[0], cA[1], cA[2]);
        iB = or_index(P, cB[0], cB[1], cB[2]);
        iF = iA; /* the face fc+1/2 is stored at cell index fc (mapped) */
        if (!P->w[c])
            vt[e] = 0.5 * (q[1 + d][iA] / q[0][iA] + q[1 + d][iB] / q[0][iB]); /* eq0361 */
        else
            vt[e] = (wB * (q[1 + d][iA] / q[0][iA]) + wA * (q[1 + d][iB] / q[0][iB])) / (wA + wB);
        bf[e] = q[5 + c][iF];
    }
    for (e = 1; e + 1 < m; ++e)
        vh[e] = 0.25 * (vt[e + 1] + 2.0 * vt[e] + vt[e - 1]);   /* eq0362 */
    for (e = 1; e + 1 < m; ++e) w[e] = vh[e] * bf[e];
    /* predictor: first-order upwind fluxes at (e, e+1), e = 1 .. m-3 */
    for (e = 1; e + 2 < m; ++e) {
        double vbar = or_edge_velocity(nu, vh[e], vh[e + 1], dw[e], dw[e + 1]);  /* eq0364 */
        f1[e] = vbar > 0.0 ? w[e] : w[e + 1];                     /* eq0363 */
    }
    for (e = 2; e + 2 < m; ++e) {
        bp[e] = bf[e] - dt / (2.0 * (nu ? dw[e] : hd)) * (f1[e] - f1[e - 1]);
        wp[e] = vh[e] * bp[e];
    }
    /* corrector: piecewise-linear TVD flux about the upwind cell; the hybrid
     * limiter takes its subsonic (Van Leer) branch here: the magnetic operator
     * has no sound speed (reading C-21) */
    {
        const int lim = P->limiter == OR_LIM_HYBRID ? OR_LIM_VANLEER : P->limiter;
        for (e = OR_NG - 1; e < OR_NG + n; ++e) {
            double vbar = or_edge_velocity(nu, vh[e], vh[e + 1], dw[e], dw[e + 1]);
            if (!nu) {
                if (vbar > 0.0)
                    f2[e] = wp[e] + 0.5 * or_limit(lim, wp[e] - wp[e - 1], wp[e + 1] - wp[e]);
                else
                    f2[e] = wp[e + 1] - 0.5 * or_limit(lim, wp[e + 1] - wp[e], wp[e + 2] - wp[e + 1]);
            } else {
                /* slopes per unit length over the centre distances, carried
                 * over half the upwind cell (reading C-25) */
                const double gl = 0.5 * (dw[e - 1] + dw[e]), gc = 0.5 * (dw[e] + dw[e + 1]),
                             gr = 0.5 * (dw[e + 1] + dw[e + 2]);
                if (vbar > 0.0)
                    f2[e] = wp[e] + 0.5 * dw[e] * or_limit(lim, (wp[e] - wp[e - 1]) / gl, (wp[e + 1] - wp[e]) / gc);
                else
                    f2[e] = wp[e + 1] - 0.5 * dw[e + 1] *
                            or_limit(lim, (wp[e + 1] - wp[e]) / gc, (wp[e + 2] - wp[e + 1]) / gr);
            }
        }
    }
    for (e = -1; e < n; ++e) f[e + 1] = f2[e + OR_NG];
}

/* Magnetic operator B_d(dt) on the whole box (eq0350, eq0360 with the physical
 * signs of reading C-5): both transverse components are advected,
 *   b_c -= dt/h_d [f_c(s') - f_c((s-1)')],
 * and the normal component takes the constraint update from the same fluxes,
 *   b_d(s') += sum_c dt/h_c [f_c at face c' - f_c at face (c-1)'].
 * All non-magnetic quantities, E included, are untouched (Sec. 2.4). */
static int or_ct_sweep(const or_problem *P, double *const *q, int d, double dt)
{
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const long n = P->n[d], n1 = P->n[t1], n2 = P->n[t2];
    const long N = (long)P->n[0] * P->n[1] * P->n[2];
    const long L = n + 1; /* interfaces -1' .. (n-1)' */
    /* flux1[(a+1) + (n1+1)*b][*]: face pencil of b_t1 at face index a in [-1, n1), cell b along t2
     * flux2[a + n1*(b+1)][*]:     face pencil of b_t2 at cell a along t1, face index b in [-1, n2) */
    double *flux1 = (double *)malloc(sizeof(double) * L * (n1 + 1) * n2);
    double *flux2 = (double *)malloc(sizeof(double) * L * n1 * (n2 + 1));
    double *nb[3];
    long a, b;
    int ax, err = 0;
    if (!flux1 || !flux2) { free(flux1); free(flux2); return -1; }

#pragma omp parallel
    {
        or_scratch S;
        int ok = or_scratch_init(&S, n) == 0;
        long pid;
#pragma omp for schedule(static)
        for (pid = 0; pid < (n1 + 1) * n2; ++pid) {
            long aa = pid % (n1 + 1) - 1, bb2 = pid / (n1 + 1);
            if (ok) or_ct_face_pencil(P, q, d, t1, aa, bb2, dt, &S, flux1 + L * pid);
        }
#pragma omp for schedule(static)
        for (pid = 0; pid < n1 * (n2 + 1); ++pid) {
            long aa = pid % n1, bb2 = pid / n1 - 1;
            if (ok) or_ct_face_pencil(P, q, d, t2, bb2, aa, dt, &S, flux2 + L * pid);
        }
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
        or_scratch_free(&S);
    }
    if (err) { free(flux1); free(flux2); return -1; }

    for (ax = 0; ax < 3; ++ax) {
        nb[ax] = (double *)malloc(sizeof(double) * N);
        if (!nb[ax]) err = 1;
        else memcpy(nb[ax], q[5 + ax], sizeof(double) * N);
    }
    if (err) { for (ax = 0; ax < 3; ++ax) free(nb[ax]); free(flux1); free(flux2); return -1; }

    for (b = 0; b < n2; ++b)
        for (a = 0; a < n1; ++a) {
            const double *fa = flux1 + L * ((a + 1) + (n1 + 1) * b);   /* face a+1/2 along t1 */
            const double *fam = flux1 + L * (a + (n1 + 1) * b);        /* face a-1/2 along t1 */
            const double *fb = flux2 + L * (a + n1 * (b + 1));         /* face b+1/2 along t2 */
            const double *fbm = flux2 + L * (a + n1 * b);              /* face b-1/2 along t2 */
            long s;
            for (s = 0; s < n; ++s) {
                long idx = or_index_dir(P, d, s, a, b);
                /* f[s+1] is the flux at interface s' */
                /* eq037 on the faces: the width of the cell a face pencil
                 * crosses along d, and for b_d the widths of its cell
                 * along t1 and t2 */
                const double hs = or_width(P, d, s), ha = or_width(P, t1, a), hb = or_width(P, t2, b);
                nb[t1][idx] = q[5 + t1][idx] - dt / hs * (fa[s + 1] - fa[s]);
                nb[t2][idx] = q[5 + t2][idx] - dt / hs * (fb[s + 1] - fb[s]);
                nb[d][idx] = q[5 + d][idx] + dt / ha * (fa[s + 1] - fam[s + 1])
                                           + dt / hb * (fb[s + 1] - fbm[s + 1]);
            }
        }
    for (ax = 0; ax < 3; ++ax) {
        memcpy(q[5 + ax], nb[ax], sizeof(double) * N);
        free(nb[ax]);
    }
    free(flux1);
    free(flux2);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* public entry points                                                       */
/* ------------------------------------------------------------------------ */

static void or_fields(const or_problem *P, double *state, double *q[8])
{
    long N = (long)P->n[0] * P->n[1] * P->n[2];
    int f;
    for (f = 0; f < 8; ++f) q[f] = state + (long)f * N;
}

/* Gravity operator G_d(tau) of the operator-split form (eq02512 with the
 * centred difference eq02513): the momentum along d takes the impulse of the
 * potential, rho and the internal energy stay; the total energy changes by
 * the kinetic energy the impulse adds (the paper's code keeps internal
 * energy as its variable, Sec. 2.3; reading C-22). */
static void or_gravity(const or_problem *P, double *const *q, int d, double tau)
{
    const long N = (long)P->n[0] * P->n[1] * P->n[2];
    long idx;
#pragma omp parallel for schedule(static)
    for (idx = 0; idx < N; ++idx) {
        long c[3], cp[3], cm[3];
        double dphi, mo, mn, rho;
        int a;
        c[0] = idx % P->n[0];
        c[1] = (idx / P->n[0]) % P->n[1];
        c[2] = idx / ((long)P->n[0] * P->n[1]);
        for (a = 0; a < 3; ++a) cp[a] = cm[a] = c[a];
        cp[d] += 1;
        cm[d] -= 1;
        dphi = (P->phi[or_index(P, cp[0], cp[1], cp[2])] - P->phi[or_index(P, cm[0], cm[1], cm[2])]) /
               or_centre_span(P, d, c[d]);
        rho = q[0][idx];
        mo = q[1 + d][idx];
        mn = mo - tau * rho * dphi;
        q[1 + d][idx] = mn;
        q[4][idx] = q[4][idx] + 0.5 * (mn * mn - mo * mo) / rho;
    }
}

/* L_d(dt) on every pencil along d -- with operator-split gravity the sweep
 * G_d(dt/2) L_d(dt) G_d(dt/2) (eq025111).  Returns the OR_FLAG_* bits seen. */
int oracle_fluid(const or_problem *P, double *state, int d, double dt)
{
    double *q[8];
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const long n1 = P->n[t1], n2 = P->n[t2];
    int flags = 0, err = 0;
    const int split = P->phi != NULL && P->gravity_split;
    or_fields(P, state, q);
    if (split) or_gravity(P, q, d, 0.5 * dt);
#pragma omp parallel
    {
        or_scratch S;
        int myflags = 0;
        long pid;
        int ok = or_scratch_init(&S, P->n[d]) == 0;
#pragma omp for schedule(static)
        for (pid = 0; pid < n1 * n2; ++pid)
            if (ok) myflags |= or_fluid_pencil(P, q, d, pid % n1, pid / n1, dt, &S);
#pragma omp critical
        {
            flags |= myflags;
            if (!ok) err = 1;
        }
        or_scratch_free(&S);
    }
    if (split && !err) or_gravity(P, q, d, 0.5 * dt);
    return err ? -1 : flags;
}

/* B_d(dt) on the whole box.  Returns 0, or -1 on allocation failure. */
int oracle_ct(const or_problem *P, double *state, int d, double dt)
{
    double *q[8];
    or_fields(P, state, q);
    return or_ct_sweep(P, q, d, dt);
}

/* One full double step u^{n+2} = L_forward L_backward u^n (eq0081): every
 * operator takes the full dt, so the state advances by 2 dt.  Time order
 * (reading C-4, the Strang-symmetric palindrome):
 *   L_x B_x L_y B_y L_z B_z | B_z L_z B_y L_y B_x L_x                       */
int oracle_step(const or_problem *P, double *state, double dt, int nsteps)
{
    int s, flags = 0, r;
    for (s = 0; s < nsteps; ++s) {
        int d;
        for (d = 0; d < 3; ++d) {
            r = oracle_fluid(P, state, d, dt); if (r < 0) return r; flags |= r;
            r = oracle_ct(P, state, d, dt); if (r < 0) return r;
        }
        for (d = 2; d >= 0; --d) {
            r = oracle_ct(P, state, d, dt); if (r < 0) return r;
            r = oracle_fluid(P, state, d, dt); if (r < 0) return r; flags |= r;
        }
    }
    return flags;
}

/* CFL time step (eq0083-eq0084, reading C-15):
 *   dt = k * min over cells and d of h_d / (|v_d| + c_F,d),
 * c_F,d the fast speed along d with the cell-centred field. */
/* eq0083-eq0084 with the minimum taken over the z-planes k0 .. k0+nk-1 only
 * (cells of other planes still serve as lower neighbours for the
 * cell-centred field). */
double oracle_cfl_planes(const or_problem *P, const double *state, double k, long k0, long nk)
{
    const long plane = (long)P->n[0] * P->n[1];
    double *q[8];
    double best = INFINITY;
    long idx;
    or_fields(P, (double *)state, q);
#pragma omp parallel for reduction(min : best) schedule(static)
    for (idx = k0 * plane; idx < (k0 + nk) * plane; ++idx) {
        long i = idx % P->n[0], j = (idx / P->n[0]) % P->n[1], kk = idx / ((long)P->n[0] * P->n[1]);
        double bcc[3];
        int ax, d, fl = 0;
        long c[3] = {i, j, kk};
        for (ax = 0; ax < 3; ++ax) {
            long cm[3] = {c[0], c[1], c[2]};
            cm[ax] -= 1;
            bcc[ax] = 0.5 * (q[5 + ax][or_index(P, cm[0], cm[1], cm[2])] + q[5 + ax][idx]);
        }
        for (d = 0; d < 3; ++d) {
            int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            double ue[5] = {q[0][idx], q[1 + d][idx], q[1 + t1][idx], q[1 + t2][idx], q[4][idx]};
            double be[3] = {bcc[d], bcc[t1], bcc[t2]};
            or_cell ce;
            double r;
            or_cell_eval(P, ue, be, &ce, &fl);
            r = or_width(P, d, c[d]) / (fabs(ce.vn) + ce.cf);   /* eq0420 */
            if (r < best) best = r;
        }
    }
    return k * best;
}

double oracle_cfl(const or_problem *P, const double *state, double k)
{
    return oracle_cfl_planes(P, state, k, 0, P->n[2]);
}

/* Diagnostics: out[0..7] = sum over cells of each field times the cell
 * volume; out[8] = max over cells of |div b| (eq0341).  For outflow
 * boxes the low boundary faces are ghosts, so the divergence is taken over
 * cells whose six faces are all stored (i, j, k >= 1 along axes with n > 1). */
void oracle_diag(const or_problem *P, const double *state, double *out)
{
    const long nx = P->n[0], ny = P->n[1], nz = P->n[2];
    const long N = nx * ny * nz;
    const double vol = P->h[0] * P->h[1] * P->h[2];
    const int nu = P->w[0] || P->w[1] || P->w[2];
    const double *q[8];
    double mx = 0.0;
    long f, i, j, k;
    for (f = 0; f < 8; ++f) q[f] = state + f * N;
    for (f = 0; f < 8; ++f) {
        double s = 0.0;
        long idx;
        if (!nu) {
            for (idx = 0; idx < N; ++idx) s += q[f][idx];
            out[f] = s * vol;
        } else {
            /* irregular mesh: each cell weighted by its own volume */
            for (idx = 0; idx < N; ++idx) {
                long ii = idx % nx, jj = (idx / nx) % ny, kk = idx / (nx * ny);
                s += q[f][idx] * (or_width(P, 0, ii) * or_width(P, 1, jj) * or_width(P, 2, kk));
            }
            out[f] = s;
        }
    }
    for (k = 0; k < nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 0; i < nx; ++i) {
                double dv;
                long idx = i + nx * (j + ny * k);
                if (P->bc == OR_BC_OUTFLOW &&
                    ((nx > 1 && i == 0) || (ny > 1 && j == 0) || (nz > 1 && k == 0)))
                    continue;
                dv = (q[5][idx] - q[5][or_index(P, i - 1, j, k)]) / or_width(P, 0, i)
                   + (q[6][idx] - q[6][or_index(P, i, j - 1, k)]) / or_width(P, 1, j)
                   + (q[7][idx] - q[7][or_index(P, i, j, k - 1)]) / or_width(P, 2, k);
                if (fabs(dv) > mx) mx = fabs(dv);
            }
    out[8] = mx;
}
