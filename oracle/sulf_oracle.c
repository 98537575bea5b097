/*
 * sulf_oracle.c -- plain, single-threaded FP64 CPU oracle for the Newton-multigrid
 * solve of one Crank-Nicolson step of the marble-sulfation system on a
 * level-set-masked Cartesian grid (Coco, Semplice, Serra Capizzano,
 * "A level-set multigrid technique for nonlinear diffusion in the numerical
 * simulation of marble degradation under chemical pollutants", arXiv:1902.07029).
 *
 * TEST INFRASTRUCTURE.  This file exists only to check the CUDA library.  Only
 * the test suite, the package smoke check and the benchmark's CPU-baseline and
 * reference legs may load it; the product path never does.  It shares no code,
 * header, table or helper with the CUDA implementation.
 *
 * Style: every routine restates the passage it cites in the most direct form --
 * explicit Jacobian entries per row, loops in box order, a textbook dense LU at
 * the coarsest level -- so that it can be checked against the paper by eye.
 *
 * Readings taken where the paper is silent, ambiguous or garbled (each is also
 * used by the CUDA path, so iterates can be compared stage by stage):
 *   R1  the flux sum of L^s_h carries 1/h^2 (Sec. 3.3, L^s_h below Eq. FDc).
 *   R2  the Jacobian is the exact derivative of F (Eqs. JssI, JscI, JcsI, JccI
 *       are printed with typos: a stray d/2, missing 1/2 factors, a shared sum).
 *   R3  the boundary row is F^s_g = s~(B_g) - s_b (Eq. BCs written with the sign
 *       that makes the diagonal positive, as the Newton update W -= dW needs).
 *   R4  theta_a = m_a (B_a - x_{i_a - m_a}) / h (Eq. JssD; the printed reference
 *       point (x_{i+1}, y_{j-1}) is a typo), second component of Eq. nij is n_y.
 *   R5  bisection on [P,G] is run until the bracket is below 1e-14 (at most 60
 *       halvings) instead of 1e-6, so B is reproducible to rounding.
 *   R6  the row of a ghost needs every stencil node that carries a nonzero
 *       weight to be active; phi~ itself may use any grid node (phi is known on
 *       the whole grid).  B comes from the quadratic phi~ (3^d stencil in the
 *       box, phi~(P) < 0), else from the linear phi~ with P = G - h n.  Per-axis
 *       interpolation orders are then tried (the construction is dimension by
 *       dimension, Eq. JssD): all 2 (the paper's row), all 1, then order 0 on
 *       the axis of smallest |n_a| (the others 2, then 1), then on the two
 *       smallest; else the identity row, which is refused on the finest level
 *       (domain rejected).  theta_a = 1 - m_a (G_a - B_a) / h, so a zero normal
 *       component gives the weights [1, 0, 0] exactly.
 *   R7  smoother: red-black collective Gauss-Seidel on the inside nodes (colour =
 *       parity of the index sum; Sec. 3.5.1 allows red-black), then the ghost
 *       rows of Eq. RelGhost relaxed ghost_sweeps times (default 4): each pass
 *       steps every ghost s from the previous pass's values, then relaxes each
 *       ghost c row by its diagonal with the fresh s.  One pass per sweep leaves
 *       the boundary rows as the bottleneck (measured factor ~0.6 per cycle);
 *       four passes give ~0.05-0.15.
 *   R8  coarse operator by rediscretisation (Sec. 3.5.3): phi and (s,c) injected;
 *       a coarse ghost whose fine twin is not active takes the mean (s,c) of the
 *       active fine nodes of its 3^d neighbourhood.
 *   R9  restriction: per-axis mirrored full weighting ([1,2,1], [2,2,0], [0,2,2],
 *       [0,4,0]) over inside fine nodes at coarse inside nodes and over outside
 *       fine nodes (ghost or band) at coarse ghosts; a tensor weight that lands
 *       on an invalid diagonal node moves to the centre.  Both components.
 *   R10 ghost-defect extension: band = inactive nodes within Chebyshev distance
 *       2 of a ghost, zero start, K = 4 explicit upwind Euler steps of
 *       dr/dtau + n.grad r = 0 with dtau = h/2 (2-D) or h/3 (3-D).
 *   R11 prolongation: (bi/tri)linear, weights renormalised over coarse active
 *       nodes (no correction where none is active).
 *   R12 coarsest level: dense LU with partial pivoting of the assembled Jacobian.
 *   R13 Newton stops on min{||F||, ||dW||/||W||} < tol; if ||F(W^n)|| < tol
 *       already, the step takes no Newton iteration.  Linear solve: cycles until
 *       ||r|| <= rtol ||F|| or the cycle cap.
 *   R16 Neumann rows (Sec. 3.6): n~ . grad s~ at B with n~ the unit gradient of
 *       the quadratic phi~ at B (linear where the 3^d stencil leaves the box);
 *       per axis the first-derivative weights of Eq. intcoeffsN times m_a / h,
 *       the other axes' value weights (Eq. JccN dimension by dimension), with
 *       the orders of R6 (checked on the members these weights reach); the
 *       identity fallback is s_g / h; tau = tau_s * 4 h / (3 sqrt(d)), the
 *       bound 2 sqrt(2) h / 3 of Eq. CFLcondN in 2-D.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ENOTCONV (-3)
#define OR_EGEOM (-4)

#define OR_MAXLEV 20
#define OR_RHOMAX 65536

enum { T_OUT = 0, T_IN = 1, T_GHOST = 2, T_BAND = 3 };


typedef struct {
    int dim, N, n;
    long nn;
    long st[3];
    double lo, h;
    double *phi;
    signed char *type;
    int ng;
    long *gidx;
    int *gpos;          /* node -> ghost index, -1 elsewhere */
    signed char *gkind; /* 0 quadratic row, 1 linear row, 2 identity row */
    signed char *gm;    /* ng*dim */
    double *gw;         /* ng*dim*3, offsets 0,1,2 */
    double *gB;         /* ng*dim */
    signed char *gord;  /* ng*dim per-axis interpolation orders of the row */
    double *gth;        /* ng*dim theta per axis at B */
    double *gnt;        /* ng*dim unit normal of phi~ at B (Neumann rows) */
    double *gwk;        /* ng*3^dim weights of the row's stencil members */
    int nb;
    long *bidx;
    long *bup;          /* nb*dim, -1 when there is no upwind value */
    double *ban;        /* nb*dim, |n_a| */
    double *Wc, *rhs, *x, *res;
    int nact;
    long *act;
    long *pos;
    double *A;
    int *piv;
} OLevel;

typedef struct {
    int dim, N, L;
    OLevel lev[OR_MAXLEV];
    /* model, Eq. maineq and Eq. dataeq */
    double a, d, m_s, m_c, alpha, beta, s_ext, s0, c0;
    /* solver */
    int bc; /* 0 Dirichlet (Eq. BCs), 1 Neumann for s (Eq. BCsN) */
    int nu1, nu2, cycle, max_newton, max_cycles, smoother, ext_steps, ghost_sweeps;
    double newton_tol, lin_rtol, tau_s;
    double t, dt;
    double *Wn;  /* state at t_n, interleaved */
    double *F;   /* Newton residual */
    const double *f1o, *f1n, *f2o, *f2n, *sbg;
    double *src_store; /* owned copies of the optional sources */
    double *sbg_store;
    /* statistics */
    long newton_total, cycles_total, steps_total;
    int newton_last, cycles_last;
    double last_rho, last_fnorm;
    int nrho;
    double *rho;
    signed char *rho_first;
    char err[256];
} Oracle;

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */

static void coords(const OLevel *L, long idx, int *ii)
{
    ii[0] = (int)(idx % L->n);
    ii[1] = L->dim > 1 ? (int)((idx / L->n) % L->n) : 0;
    ii[2] = L->dim > 2 ? (int)(idx / ((long)L->n * L->n)) : 0;
}

static int active(signed char t) { return t == T_IN || t == T_GHOST; }

static double phi_of(const Oracle *O, double c) { return O->alpha * c + O->beta; } /* Sec. 2 */

static double maxabs_active(const OLevel *L, const double *v)
{
    double m = 0.0;
    for (long i = 0; i < L->nn; i++) {
        if (!active(L->type[i])) continue;
        double a0 = fabs(v[2 * i]), a1 = fabs(v[2 * i + 1]);
        if (a0 > m || a0 != a0) m = a0;
        if (a1 > m || a1 != a1) m = a1;
        if (m != m) return m;
    }
    return m;
}

static int ipow3(int d) { return d == 2 ? 9 : 27; }

/* ------------------------------------------------------------------ */
/* geometry: Sec. 3.2, Sec. 3.3 (Eq. ghostdef, Eq. nij, ST, Fig.       */
/* closestpoint), Eq. intcoeffsD, Eq. JssD                              */
/* ------------------------------------------------------------------ */

/* central differences of the level set (Eq. nij); one-sided at the box edge */
static void grad_phi(const OLevel *L, long idx, const int *ii, double *g)
{
    for (int a = 0; a < L->dim; a++) {
        int hm = ii[a] > 0, hp = ii[a] < L->N;
        if (hm && hp)
            g[a] = (L->phi[idx + L->st[a]] - L->phi[idx - L->st[a]]) / (2.0 * L->h);
        else if (hp)
            g[a] = (L->phi[idx + L->st[a]] - L->phi[idx]) / L->h;
        else
            g[a] = (L->phi[idx] - L->phi[idx - L->st[a]]) / L->h;
    }
}

/* 1-D Lagrange basis on the upwind nodes of a ghost, in the local coordinate
   xi = m (X - x_{i-m}) / h that puts offset 0 (the ghost) at xi = +1, offset 1
   at 0 and offset 2 at -1.  Quadratic: Eq. intcoeffsD with theta = xi.
   Linear and constant (fallbacks, R6): offsets 0,1 and offset 0 only. */
static double lag(int order, int k, double xi)
{
    if (order == 0) return k == 0 ? 1.0 : 0.0;
    if (order == 2) {
        if (k == 0) return xi * (1.0 + xi) / 2.0;
        if (k == 1) return (1.0 - xi) * (1.0 + xi);
        return xi * (xi - 1.0) / 2.0;
    }
    if (k == 0) return xi;
    if (k == 1) return 1.0 - xi;
    return 0.0;
}

/* derivative of lag with respect to xi: the 1-D first-derivative weights of
   Eq. intcoeffsN (times h) for the quadratic, (1, -1) for the linear, 0 for
   the constant */
static double dlag(int order, int k, double xi)
{
    if (order == 0) return 0.0;
    if (order == 2) {
        if (k == 0) return xi + 0.5;
        if (k == 1) return -2.0 * xi;
        return xi - 0.5;
    }
    if (k == 0) return 1.0;
    if (k == 1) return -1.0;
    return 0.0;
}

/* gradient of the tensor interpolant phi~ of the given order on the upwind
   stencil of ghost g, at the local coordinates xi (Eq. Neumanntilde: n~* =
   grad phi~); d/dX_a = (m_a / h) d/dxi_a */
static void grad_phi_tilde(const OLevel *L, int order, long g, const int *m, const double *xi, double *gr)
{
    int nk = ipow3(L->dim);
    for (int a = 0; a < L->dim; a++) gr[a] = 0.0;
    for (int kk = 0; kk < nk; kk++) {
        int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
        long node = g;
        int skip = 0;
        for (int a = 0; a < L->dim; a++) {
            if (order == 1 && k[a] == 2) skip = 1;
            node -= (long)m[a] * k[a] * L->st[a];
        }
        if (skip) continue;
        for (int a = 0; a < L->dim; a++) {
            double t = (m[a] / L->h) * dlag(order, k[a], xi[a]);
            for (int b = 0; b < L->dim; b++)
                if (b != a) t *= lag(order, k[b], xi[b]);
            gr[a] += t * L->phi[node];
        }
    }
}

/* weight of stencil member kk in a ghost's row.  Dirichlet (Eq. JssD): the
   tensor product of the 1-D value weights.  Neumann (Eq. JccN, built
   dimension by dimension): n~ . grad s~ at B, i.e. sum over axes a of
   n~_a (m_a / h) dlag_a prod_{b != a} lag_b. */
static double member_weight(int bc, int D, double h, const int *m, const int *ord, const double *th,
                            const double *nt, int kk)
{
    int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
    if (bc == 0) {
        double w = 1.0;
        for (int a = 0; a < D; a++) w *= lag(ord[a], k[a], th[a]);
        return w;
    }
    double w = 0.0;
    for (int a = 0; a < D; a++) {
        double t = nt[a] * (m[a] / h) * dlag(ord[a], k[a], th[a]);
        for (int b = 0; b < D; b++)
            if (b != a) t *= lag(ord[b], k[b], th[b]);
        w += t;
    }
    return w;
}

/* tensor-product interpolant (Eq. JssD built dimension by dimension) of phi on
   the upwind stencil of the ghost at box index g (coordinates ii, signs m),
   evaluated at X.  The local coordinate xi_a = 1 - m_a (G_a - X_a) / h equals
   m_a (X_a - x_{i_a - m_a}) / h. */
static double phi_tilde(const OLevel *L, int order, long g, const int *ii, const int *m, const double *X)
{
    double xi[3] = {0, 0, 0};
    for (int a = 0; a < L->dim; a++)
        xi[a] = 1.0 - m[a] * ((L->lo + ii[a] * L->h) - X[a]) / L->h;
    double sum = 0.0;
    int nk = ipow3(L->dim);
    for (int kk = 0; kk < nk; kk++) {
        int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
        double w = 1.0;
        long node = g;
        int skip = 0;
        for (int a = 0; a < L->dim; a++) {
            if (order == 1 && k[a] == 2) skip = 1;
            w *= lag(order, k[a], xi[a]);
            node -= (long)m[a] * k[a] * L->st[a];
        }
        if (skip) continue;
        sum += w * L->phi[node];
    }
    return sum;
}

/* is the upwind stencil with offsets 0..order per axis inside the box? */
static int stencil_in_box(const OLevel *L, const int *ii, const int *m, int order)
{
    for (int a = 0; a < L->dim; a++) {
        int ia = ii[a] - m[a] * order;
        if (ia < 0 || ia > L->N) return 0;
    }
    return 1;
}

/* does every stencil node with a nonzero member weight belong to the active set? */
static int weighted_nodes_active(const OLevel *L, long g, const int *m, const double *wk)
{
    int nk = ipow3(L->dim);
    for (int kk = 0; kk < nk; kk++) {
        int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
        long node = g;
        for (int a = 0; a < L->dim; a++) node -= (long)m[a] * k[a] * L->st[a];
        if (wk[kk] != 0.0 && !active(L->type[node])) return 0;
    }
    return 1;
}

/* Ghost geometry (Sec. 3.3): outward normal by Eq. nij, upwind stencil ST,
   closest boundary point B by bisection on phi~ along P->G, then the 1-D
   weights at B (Eq. intcoeffsD), built dimension by dimension.
   B comes from the quadratic phi~ on the 3^d stencil with P = G - 2 h n, else
   from the linear phi~ on the 2^d stencil with P = G - h n (phi~ may use any
   grid node: the level set is known on the whole grid).  The row needs every
   node it weights to be active; the per-axis interpolation orders tried are
   all 2 (the paper's row), all 1, then order 0 on the axis with the smallest
   |n_a| (others 2, then 1), then on the two smallest (3-D); else the identity
   row (R6).  Returns 0 (all axes quadratic), 1 (reduced order) or 2 (identity).
   Also returns the per-axis orders and theta of the row, the unit normal of
   phi~ at B (the quadratic interpolant where its stencil fits in the box, else
   the linear one, else the node normal), and the member weights for the
   boundary condition bc.  The activity test uses the member weights, so a
   Neumann row (whose derivative weights reach members that a value weight
   misses when theta = 0) is checked on the nodes it actually uses.  The
   identity row is s_g for Dirichlet and s_g / h for Neumann (the scale of a
   derivative row). */
static int ghost_geometry(const OLevel *L, long g, int bc, signed char *m_out, double *w_out, double *B_out,
                          signed char *ord_out, double *th_out, double *nt_out, double *wk_out)
{
    int ii[3];
    coords(L, g, ii);
    int D = L->dim;
    int nk = ipow3(D);
    double gr[3] = {0, 0, 0}, n[3] = {0, 0, 0};
    grad_phi(L, g, ii, gr);
    double nrm = 0.0;
    for (int a = 0; a < D; a++) nrm += gr[a] * gr[a];
    nrm = sqrt(nrm);
    int m[3] = {1, 1, 1};
    if (nrm > 0.0)
        for (int a = 0; a < D; a++) {
            n[a] = gr[a] / nrm;
            m[a] = n[a] >= 0.0 ? 1 : -1; /* SIGN(0) = 1 */
        }
    for (int a = 0; a < D; a++) m_out[a] = (signed char)m[a];
    int border = 0; /* order of the interpolant that located B (0: none) */
    double B[3] = {0, 0, 0};
    if (nrm > 0.0) {
        for (int order = 2; order >= 1 && !border; order--) {
            if (!stencil_in_box(L, ii, m, order)) continue;
            double G[3] = {0, 0, 0}, P[3] = {0, 0, 0}, X[3] = {0, 0, 0};
            for (int a = 0; a < D; a++) {
                G[a] = L->lo + ii[a] * L->h;
                P[a] = G[a] - order * L->h * n[a];
            }
            if (!(phi_tilde(L, order, g, ii, m, P) < 0.0)) continue;
            double alo = 0.0, ahi = 1.0;
            for (int it = 0; it < 60 && ahi - alo >= 1e-14; it++) {
                double am = 0.5 * (alo + ahi);
                for (int a = 0; a < D; a++) X[a] = P[a] + am * (G[a] - P[a]);
                if (phi_tilde(L, order, g, ii, m, X) < 0.0)
                    alo = am;
                else
                    ahi = am;
            }
            double al = 0.5 * (alo + ahi);
            for (int a = 0; a < D; a++) B[a] = P[a] + al * (G[a] - P[a]);
            border = order;
        }
    }
    double nt[3] = {n[0], n[1], n[2]};
    if (border) {
        /* axes by increasing |n_a| (ties: lower axis first) */
        int ax[3] = {0, 1, 2};
        for (int i = 0; i < D; i++)
            for (int j = i + 1; j < D; j++)
                if (fabs(n[ax[j]]) < fabs(n[ax[i]])) {
                    int t = ax[i];
                    ax[i] = ax[j];
                    ax[j] = t;
                }
        double th[3] = {0, 0, 0};
        for (int a = 0; a < D; a++) th[a] = 1.0 - m[a] * ((L->lo + ii[a] * L->h) - B[a]) / L->h;
        int q = stencil_in_box(L, ii, m, 2) ? 2 : (stencil_in_box(L, ii, m, 1) ? 1 : 0);
        if (q) {
            double gt[3] = {0, 0, 0}, gn = 0.0;
            grad_phi_tilde(L, q, g, m, th, gt);
            for (int a = 0; a < D; a++) gn += gt[a] * gt[a];
            gn = sqrt(gn);
            if (gn > 0.0)
                for (int a = 0; a < D; a++) nt[a] = gt[a] / gn;
        }
        for (int nzero = 0; nzero < D; nzero++) {
            for (int top = border; top >= 1; top--) {
                int ord[3] = {top, top, top};
                for (int z = 0; z < nzero; z++) ord[ax[z]] = 0;
                for (int kk = 0; kk < nk; kk++) wk_out[kk] = member_weight(bc, D, L->h, m, ord, th, nt, kk);
                if (weighted_nodes_active(L, g, m, wk_out)) {
                    for (int a = 0; a < D; a++) {
                        for (int k = 0; k < 3; k++) w_out[3 * a + k] = lag(ord[a], k, th[a]);
                        B_out[a] = B[a];
                        ord_out[a] = (signed char)ord[a];
                        th_out[a] = th[a];
                        nt_out[a] = nt[a];
                    }
                    return (nzero == 0 && top == 2) ? 0 : 1;
                }
            }
        }
    }
    for (int a = 0; a < D; a++) {
        w_out[3 * a + 0] = 1.0;
        w_out[3 * a + 1] = 0.0;
        w_out[3 * a + 2] = 0.0;
        B_out[a] = L->lo + ii[a] * L->h;
        ord_out[a] = 0;
        th_out[a] = 1.0;
        nt_out[a] = nt[a];
    }
    for (int kk = 0; kk < nk; kk++) wk_out[kk] = 0.0;
    wk_out[0] = bc == 0 ? 1.0 : 1.0 / L->h;
    return 2;
}

/* (re)build the boundary rows of every ghost of a level for the boundary
   condition bc; the finest level refuses identity rows */
static int build_ghost_rows(Oracle *O, OLevel *L, int finest, int bc)
{
    int D = L->dim, nk = ipow3(D);
    for (int gi = 0; gi < L->ng; gi++) {
        long g = L->gidx[gi];
        int kind = ghost_geometry(L, g, bc, L->gm + (size_t)D * gi, L->gw + (size_t)3 * D * gi,
                                  L->gB + (size_t)D * gi, L->gord + (size_t)D * gi, L->gth + (size_t)D * gi,
                                  L->gnt + (size_t)D * gi, L->gwk + (size_t)nk * gi);
        L->gkind[gi] = (signed char)kind;
        if (kind == 2 && finest) {
            snprintf(O->err, sizeof O->err, "ghost %ld has no valid boundary stencil", g);
            return OR_EGEOM;
        }
    }
    return OR_OK;
}

static int build_level_geometry(Oracle *O, OLevel *L, int finest)
{
    long nn = L->nn;
    /* Eq. ghostdef: inside = phi < 0; ghost = not inside with an inside axis neighbour */
    for (long i = 0; i < nn; i++) L->type[i] = L->phi[i] < 0.0 ? T_IN : T_OUT;
    int ii[3];
    for (long i = 0; i < nn; i++) {
        if (L->type[i] != T_OUT) continue;
        coords(L, i, ii);
        for (int a = 0; a < L->dim; a++) {
            if (ii[a] > 0 && L->type[i - L->st[a]] == T_IN) L->type[i] = T_GHOST;
            if (ii[a] < L->N && L->type[i + L->st[a]] == T_IN) L->type[i] = T_GHOST;
        }
    }
    int nin = 0, ng = 0;
    for (long i = 0; i < nn; i++) {
        if (L->type[i] == T_IN) nin++;
        if (L->type[i] == T_GHOST) ng++;
        if (finest && active(L->type[i])) {
            coords(L, i, ii);
            for (int a = 0; a < L->dim; a++)
                if (ii[a] == 0 || ii[a] == L->N) {
                    snprintf(O->err, sizeof O->err, "active node on the box edge");
                    return OR_EINVAL;
                }
        }
    }
    if (nin == 0) {
        snprintf(O->err, sizeof O->err, "no inside node at level N=%d", L->N);
        return OR_EINVAL;
    }
    /* ghost list in box order */
    L->ng = ng;
    L->gidx = (long *)malloc(sizeof(long) * (ng + 1));
    L->gkind = (signed char *)malloc(ng + 1);
    L->gm = (signed char *)malloc((size_t)L->dim * (ng + 1));
    L->gw = (double *)malloc(sizeof(double) * 3 * L->dim * (ng + 1));
    L->gB = (double *)malloc(sizeof(double) * L->dim * (ng + 1));
    L->gord = (signed char *)malloc((size_t)L->dim * (ng + 1));
    L->gth = (double *)malloc(sizeof(double) * L->dim * (ng + 1));
    L->gnt = (double *)malloc(sizeof(double) * L->dim * (ng + 1));
    L->gwk = (double *)malloc(sizeof(double) * ipow3(L->dim) * (ng + 1));
    if (!L->gidx || !L->gkind || !L->gm || !L->gw || !L->gB || !L->gord || !L->gth || !L->gnt || !L->gwk)
        return OR_ENOMEM;
    int k = 0;
    for (long i = 0; i < nn; i++)
        if (L->type[i] == T_GHOST) L->gidx[k++] = i;
    L->gpos = (int *)malloc(sizeof(int) * nn);
    if (!L->gpos) return OR_ENOMEM;
    for (long i = 0; i < nn; i++) L->gpos[i] = -1;
    for (int gi = 0; gi < ng; gi++) L->gpos[L->gidx[gi]] = gi;
    int rc = build_ghost_rows(O, L, finest, O->bc);
    if (rc) return rc;
    /* band for the ghost-defect extension (R10) */
    signed char *layer = (signed char *)calloc(nn, 1);
    if (!layer) return OR_ENOMEM;
    int nk = ipow3(L->dim);
    for (int pass = 1; pass <= 2; pass++) {
        for (long i = 0; i < nn; i++) {
            if (L->type[i] != T_OUT || layer[i]) continue;
            coords(L, i, ii);
            int hit = 0;
            for (int kk = 0; kk < nk && !hit; kk++) {
                int kd[3] = {kk % 3 - 1, (kk / 3) % 3 - 1, kk / 9 - 1};
                long node = i;
                int ok = 1;
                for (int a = 0; a < L->dim; a++) {
                    int ia = ii[a] + kd[a];
                    if (ia < 0 || ia > L->N) ok = 0;
                    node += (long)kd[a] * L->st[a];
                }
                if (!ok || node == i) continue;
                if (pass == 1 && L->type[node] == T_GHOST) hit = 1;
                if (pass == 2 && layer[node] == 1) hit = 1;
            }
            if (hit) layer[i] = (signed char)pass;
        }
    }
    int nb = 0;
    for (long i = 0; i < nn; i++)
        if (layer[i]) {
            L->type[i] = T_BAND;
            nb++;
        }
    L->nb = nb;
    L->bidx = (long *)malloc(sizeof(long) * (nb + 1));
    L->bup = (long *)malloc(sizeof(long) * L->dim * (nb + 1));
    L->ban = (double *)malloc(sizeof(double) * L->dim * (nb + 1));
    if (!L->bidx || !L->bup || !L->ban) {
        free(layer);
        return OR_ENOMEM;
    }
    int b = 0;
    for (long i = 0; i < nn; i++) {
        if (!layer[i]) continue;
        L->bidx[b] = i;
        coords(L, i, ii);
        double gr[3] = {0, 0, 0};
        grad_phi(L, i, ii, gr);
        double nrm = 0.0;
        for (int a = 0; a < L->dim; a++) nrm += gr[a] * gr[a];
        nrm = sqrt(nrm);
        for (int a = 0; a < L->dim; a++) {
            double na = nrm > 0.0 ? gr[a] / nrm : 0.0;
            int m = na >= 0.0 ? 1 : -1;
            int ia = ii[a] - m;
            long up = -1;
            if (ia >= 0 && ia <= L->N) {
                long node = i - (long)m * L->st[a];
                if (L->type[node] == T_GHOST || L->type[node] == T_BAND) up = node;
            }
            L->bup[(size_t)L->dim * b + a] = up;
            L->ban[(size_t)L->dim * b + a] = fabs(na);
        }
        b++;
    }
    free(layer);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Jacobian rows (exact derivative of F, R2; structure of Eqs. JssI,    */
/* JssD, JscI, JcsI, JccI)                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    double ss_pp, sc_pp, cs_pp, cc_pp;
    double ss_q[6], sc_q[6];
    long q[6];
    int nq;
} JRow;

static void jrow_inside(const Oracle *O, const OLevel *L, long p, JRow *J)
{
    const double *W = L->Wc;
    double s = W[2 * p], c = W[2 * p + 1];
    double ph = phi_of(O, c);
    double kap = O->d / (4.0 * L->h * L->h);
    double dt = O->dt;
    J->ss_pp = ph / dt + (O->a / (2.0 * O->m_c)) * ph * c;
    J->sc_pp = O->alpha * s / dt + (O->a / (2.0 * O->m_c)) * (O->alpha * s * c + ph * s);
    J->nq = 0;
    for (int a = 0; a < L->dim; a++)
        for (int sg = -1; sg <= 1; sg += 2) {
            long q = p + sg * L->st[a];
            double sq = W[2 * q], cq = W[2 * q + 1];
            double phq = phi_of(O, cq);
            J->q[J->nq] = q;
            J->ss_q[J->nq] = -kap * (phq + ph);
            J->sc_q[J->nq] = kap * O->alpha * (s - sq);
            J->ss_pp += kap * (phq + ph);
            J->sc_pp += kap * O->alpha * (s - sq);
            J->nq++;
        }
    J->cs_pp = (O->a / (2.0 * O->m_s)) * ph * c;
    J->cc_pp = 1.0 / dt + (O->a / (2.0 * O->m_s)) * (O->alpha * s * c + ph * s);
}

static void jrow_c(const Oracle *O, const OLevel *L, long p, double *cs, double *cc)
{
    double s = L->Wc[2 * p], c = L->Wc[2 * p + 1];
    double ph = phi_of(O, c);
    *cs = (O->a / (2.0 * O->m_s)) * ph * c;
    *cc = 1.0 / O->dt + (O->a / (2.0 * O->m_s)) * (O->alpha * s * c + ph * s);
}

/* the weight of stencil node kk (k_a in {0,1,2}) of ghost gi, and the node */
static double ghost_w(const OLevel *L, int gi, int kk, long *node)
{
    int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
    long nd = L->gidx[gi];
    for (int a = 0; a < L->dim; a++) nd -= (long)L->gm[(size_t)L->dim * gi + a] * k[a] * L->st[a];
    *node = nd;
    return L->gwk[(size_t)ipow3(L->dim) * gi + kk];
}

static double ghost_row_dot(const OLevel *L, int gi, const double *v)
{
    double sum = 0.0;
    int nk = ipow3(L->dim);
    for (int kk = 0; kk < nk; kk++) {
        long node;
        double w = ghost_w(L, gi, kk, &node);
        if (w == 0.0) continue;
        sum += w * v[2 * node];
    }
    return sum;
}

/* out = J x on every active node of the level; zero elsewhere */
static void apply_J(const Oracle *O, const OLevel *L, const double *x, double *out)
{
    for (long i = 0; i < 2 * L->nn; i++) out[i] = 0.0;
    for (long p = 0; p < L->nn; p++) {
        if (L->type[p] != T_IN) continue;
        JRow J;
        jrow_inside(O, L, p, &J);
        double vs = J.ss_pp * x[2 * p] + J.sc_pp * x[2 * p + 1];
        for (int k = 0; k < J.nq; k++) vs += J.ss_q[k] * x[2 * J.q[k]] + J.sc_q[k] * x[2 * J.q[k] + 1];
        out[2 * p] = vs;
        out[2 * p + 1] = J.cs_pp * x[2 * p] + J.cc_pp * x[2 * p + 1];
    }
    for (int gi = 0; gi < L->ng; gi++) {
        long g = L->gidx[gi];
        double cs, cc;
        jrow_c(O, L, g, &cs, &cc);
        out[2 * g] = ghost_row_dot(L, gi, x);
        out[2 * g + 1] = cs * x[2 * g] + cc * x[2 * g + 1];
    }
}

/* ------------------------------------------------------------------ */
/* Newton residual F: Eqs. FDs, FDc (inside; FDc also at ghosts) and    */
/* Eq. BCs (ghost s rows, sign of R3)                                   */
/* ------------------------------------------------------------------ */

static double Ls_h(const Oracle *O, const OLevel *L, const double *W, long p)
{
    double s = W[2 * p], c = W[2 * p + 1], ph = phi_of(O, c);
    double flux = 0.0;
    for (int a = 0; a < L->dim; a++)
        for (int sg = -1; sg <= 1; sg += 2) {
            long q = p + sg * L->st[a];
            flux += (phi_of(O, W[2 * q + 1]) + ph) * (W[2 * q] - s);
        }
    return -(O->a / O->m_c) * ph * s * c + (O->d / (2.0 * L->h * L->h)) * flux;
}

static double Lc_h(const Oracle *O, const double *W, long p)
{
    double s = W[2 * p], c = W[2 * p + 1];
    return -(O->a / O->m_s) * phi_of(O, c) * s * c;
}

static void eval_F(const Oracle *O, const double *W, const double *Wn, double *F)
{
    const OLevel *L = &O->lev[0];
    double dt = O->dt;
    for (long i = 0; i < 2 * L->nn; i++) F[i] = 0.0;
    for (long p = 0; p < L->nn; p++) {
        if (!active(L->type[p])) continue;
        if (L->type[p] == T_IN) {
            double fs = (phi_of(O, W[2 * p + 1]) * W[2 * p] - phi_of(O, Wn[2 * p + 1]) * Wn[2 * p]) / dt -
                        0.5 * (Ls_h(O, L, Wn, p) + Ls_h(O, L, W, p));
            if (O->f1o) fs -= 0.5 * (O->f1o[p] + O->f1n[p]);
            F[2 * p] = fs;
        }
        double fc = (W[2 * p + 1] - Wn[2 * p + 1]) / dt - 0.5 * (Lc_h(O, Wn, p) + Lc_h(O, W, p));
        if (O->f2o) fc -= 0.5 * (O->f2o[p] + O->f2n[p]);
        F[2 * p + 1] = fc;
    }
    for (int gi = 0; gi < L->ng; gi++) {
        long g = L->gidx[gi];
        double sb = O->sbg ? O->sbg[gi] : O->s_ext;
        F[2 * g] = ghost_row_dot(L, gi, W) - sb;
    }
}

/* ------------------------------------------------------------------ */
/* multigrid: Sec. 3.5                                                   */
/* ------------------------------------------------------------------ */

/* collective (2x2 block) update of inside node p: Eq. matrixP, or its diagonal
   (Eq. matrixPclassical) for the pointwise variant */
static void relax_inside(const Oracle *O, OLevel *L, long p, int pointwise)
{
    double *x = L->x;
    const double *rhs = L->rhs;
    JRow J;
    jrow_inside(O, L, p, &J);
    double rs = rhs[2 * p] - (J.ss_pp * x[2 * p] + J.sc_pp * x[2 * p + 1]);
    for (int k = 0; k < J.nq; k++) rs -= J.ss_q[k] * x[2 * J.q[k]] + J.sc_q[k] * x[2 * J.q[k] + 1];
    double rc = rhs[2 * p + 1] - (J.cs_pp * x[2 * p] + J.cc_pp * x[2 * p + 1]);
    if (pointwise) {
        x[2 * p] += rs / J.ss_pp;
        x[2 * p + 1] += rc / J.cc_pp;
    } else {
        double det = J.ss_pp * J.cc_pp - J.sc_pp * J.cs_pp;
        x[2 * p] += (J.cc_pp * rs - J.sc_pp * rc) / det;
        x[2 * p + 1] += (J.ss_pp * rc - J.cs_pp * rs) / det;
    }
}

/* ghost relaxation of Eq. RelGhost, repeated ghost_sweeps times (R7): in each
   pass every ghost s row takes the fictitious-time step s_g += tau (r_g - row.x)
   from the values of the previous pass, then each ghost c row is relaxed by its
   diagonal with the fresh s_g */
static void relax_ghosts(const Oracle *O, OLevel *L)
{
    double *x = L->x;
    const double *rhs = L->rhs;
    double *ns = (double *)malloc(sizeof(double) * (L->ng + 1));
    /* Neumann rows have a diagonal of order 1/h: tau_s scales the bound of
       Eq. CFLcondN, 2 sqrt(2) h / 3 in 2-D, i.e. 4 h / (3 sqrt(d)) */
    const double tau = O->bc ? O->tau_s * 4.0 * L->h / (3.0 * sqrt((double)L->dim)) : O->tau_s;
    for (int rep = 0; rep < O->ghost_sweeps; rep++) {
        for (int gi = 0; gi < L->ng; gi++) {
            long g = L->gidx[gi];
            ns[gi] = x[2 * g] + tau * (rhs[2 * g] - ghost_row_dot(L, gi, x));
        }
        for (int gi = 0; gi < L->ng; gi++) {
            long g = L->gidx[gi];
            double cs, cc;
            jrow_c(O, L, g, &cs, &cc);
            x[2 * g] = ns[gi];
            x[2 * g + 1] += (rhs[2 * g + 1] - (cs * x[2 * g] + cc * x[2 * g + 1])) / cc;
        }
    }
    free(ns);
}

/* one relaxation sweep (Sec. 3.5.1): the inside nodes first, then the ghosts,
   following the map M that lists inside nodes before ghosts.  smoother 0/1:
   red-black order of the inside nodes (colour = parity of the index sum),
   collective or pointwise; smoother 2: lexicographic (box) order. */
static void smooth(const Oracle *O, OLevel *L)
{
    int ii[3];
    if (O->smoother == 2) {
        for (long p = 0; p < L->nn; p++)
            if (L->type[p] == T_IN) relax_inside(O, L, p, 0);
    } else {
        for (int colour = 0; colour < 2; colour++)
            for (long p = 0; p < L->nn; p++) {
                if (L->type[p] != T_IN) continue;
                coords(L, p, ii);
                if (((ii[0] + ii[1] + ii[2]) & 1) != colour) continue;
                relax_inside(O, L, p, O->smoother == 1);
            }
    }
    relax_ghosts(O, L);
}

/* defect r = rhs - J x on active nodes, zero elsewhere */
static void residual(const Oracle *O, OLevel *L)
{
    apply_J(O, L, L->x, L->res);
    for (long p = 0; p < L->nn; p++) {
        if (!active(L->type[p])) {
            L->res[2 * p] = L->res[2 * p + 1] = 0.0;
            continue;
        }
        L->res[2 * p] = L->rhs[2 * p] - L->res[2 * p];
        L->res[2 * p + 1] = L->rhs[2 * p + 1] - L->res[2 * p + 1];
    }
}

/* extend the ghost defect into the band along the normal (Sec. 3.5.2, R10) */
static void extend_defect(const Oracle *O, OLevel *L)
{
    if (L->nb == 0) return;
    double cfl = L->dim == 2 ? 0.5 : 1.0 / 3.0;
    double *nv = (double *)malloc(sizeof(double) * 2 * L->nb);
    for (int b = 0; b < L->nb; b++) L->res[2 * L->bidx[b]] = L->res[2 * L->bidx[b] + 1] = 0.0;
    for (int it = 0; it < O->ext_steps; it++) {
        for (int b = 0; b < L->nb; b++) {
            long i = L->bidx[b];
            for (int comp = 0; comp < 2; comp++) {
                double v = L->res[2 * i + comp], acc = 0.0;
                for (int a = 0; a < L->dim; a++) {
                    long up = L->bup[(size_t)L->dim * b + a];
                    if (up < 0) continue;
                    acc += L->ban[(size_t)L->dim * b + a] * (v - L->res[2 * up + comp]);
                }
                nv[2 * b + comp] = v - cfl * acc;
            }
        }
        for (int b = 0; b < L->nb; b++) {
            L->res[2 * L->bidx[b]] = nv[2 * b];
            L->res[2 * L->bidx[b] + 1] = nv[2 * b + 1];
        }
    }
    free(nv);
}

/* boundary-aware full weighting (Eqs. Fstencil, Fstencilgen, Fig. Neigh, R9) */
static void restrict_defect(const OLevel *Lf, OLevel *Lc)
{
    int ii[3];
    int nk = ipow3(Lf->dim);
    for (long i = 0; i < 2 * Lc->nn; i++) Lc->rhs[i] = 0.0;
    for (long I = 0; I < Lc->nn; I++) {
        signed char tc = Lc->type[I];
        if (!active(tc)) continue;
        coords(Lc, I, ii);
        long f = 0;
        int fi[3] = {0, 0, 0};
        for (int a = 0; a < Lf->dim; a++) {
            fi[a] = 2 * ii[a];
            f += (long)fi[a] * Lf->st[a];
        }
        double w1[3][3];
        for (int a = 0; a < Lf->dim; a++) {
            int vl = 0, vr = 0;
            if (fi[a] > 0) {
                signed char t = Lf->type[f - Lf->st[a]];
                vl = tc == T_IN ? t == T_IN : (t == T_GHOST || t == T_BAND);
            }
            if (fi[a] < Lf->N) {
                signed char t = Lf->type[f + Lf->st[a]];
                vr = tc == T_IN ? t == T_IN : (t == T_GHOST || t == T_BAND);
            }
            double l = 1, c = 2, r = 1;
            if (vl && !vr) { l = 2; c = 2; r = 0; }
            if (!vl && vr) { l = 0; c = 2; r = 2; }
            if (!vl && !vr) { l = 0; c = 4; r = 0; }
            w1[a][0] = l / 4.0;
            w1[a][1] = c / 4.0;
            w1[a][2] = r / 4.0;
        }
        double acc_s = 0.0, acc_c = 0.0, wcentre = 0.0;
        for (int kk = 0; kk < nk; kk++) {
            int k[3] = {kk % 3 - 1, (kk / 3) % 3 - 1, kk / 9 - 1};
            double w = 1.0;
            long node = f;
            int centre = 1;
            for (int a = 0; a < Lf->dim; a++) {
                w *= w1[a][k[a] + 1];
                node += (long)k[a] * Lf->st[a];
                if (k[a] != 0) centre = 0;
            }
            if (w == 0.0) continue;
            if (centre) {
                wcentre += w;
                continue;
            }
            signed char t = Lf->type[node];
            int valid = tc == T_IN ? t == T_IN : (t == T_GHOST || t == T_BAND);
            if (!valid) {
                wcentre += w;
                continue;
            }
            acc_s += w * Lf->res[2 * node];
            acc_c += w * Lf->res[2 * node + 1];
        }
        acc_s += wcentre * Lf->res[2 * f];
        acc_c += wcentre * Lf->res[2 * f + 1];
        Lc->rhs[2 * I] = acc_s;
        Lc->rhs[2 * I + 1] = acc_c;
    }
}

/* linear interpolation of the coarse correction to every fine active node
   (Sec. 3.5.3, R11) */
static void prolong_add(const OLevel *Lc, OLevel *Lf)
{
    int ii[3];
    for (long i = 0; i < Lf->nn; i++) {
        if (!active(Lf->type[i])) continue;
        coords(Lf, i, ii);
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < Lf->dim; a++) {
            lo[a] = ii[a] / 2;
            hi[a] = (ii[a] + 1) / 2;
        }
        double ws = 0.0, as = 0.0, ac = 0.0;
        int nc = 1 << Lf->dim;
        for (int cc = 0; cc < nc; cc++) {
            long node = 0;
            double w = 1.0;
            int dup = 0;
            for (int a = 0; a < Lf->dim; a++) {
                int pick = (cc >> a) & 1;
                if (lo[a] == hi[a]) {
                    if (pick) dup = 1;
                    node += (long)lo[a] * Lc->st[a];
                } else {
                    w *= 0.5;
                    node += (long)(pick ? hi[a] : lo[a]) * Lc->st[a];
                }
            }
            if (dup) continue;
            if (!active(Lc->type[node])) continue;
            ws += w;
            as += w * Lc->x[2 * node];
            ac += w * Lc->x[2 * node + 1];
        }
        if (ws > 0.0) {
            Lf->x[2 * i] += as / ws;
            Lf->x[2 * i + 1] += ac / ws;
        }
    }
}

/* coefficients of the coarse Jacobian by injection of (s,c) (R8) */
static void inject_Wc(const OLevel *Lf, OLevel *Lc)
{
    int ii[3];
    int nk = ipow3(Lf->dim);
    for (long I = 0; I < Lc->nn; I++) {
        Lc->Wc[2 * I] = Lc->Wc[2 * I + 1] = 0.0;
        if (!active(Lc->type[I])) continue;
        coords(Lc, I, ii);
        long f = 0;
        for (int a = 0; a < Lf->dim; a++) f += (long)(2 * ii[a]) * Lf->st[a];
        if (active(Lf->type[f])) {
            Lc->Wc[2 * I] = Lf->Wc[2 * f];
            Lc->Wc[2 * I + 1] = Lf->Wc[2 * f + 1];
            continue;
        }
        double ss = 0.0, sc = 0.0;
        int cnt = 0;
        for (int kk = 0; kk < nk; kk++) {
            int k[3] = {kk % 3 - 1, (kk / 3) % 3 - 1, kk / 9 - 1};
            long node = f;
            int ok = 1;
            for (int a = 0; a < Lf->dim; a++) {
                int ia = 2 * ii[a] + k[a];
                if (ia < 0 || ia > Lf->N) ok = 0;
                node += (long)k[a] * Lf->st[a];
            }
            if (!ok || !active(Lf->type[node])) continue;
            ss += Lf->Wc[2 * node];
            sc += Lf->Wc[2 * node + 1];
            cnt++;
        }
        if (cnt > 0) {
            Lc->Wc[2 * I] = ss / cnt;
            Lc->Wc[2 * I + 1] = sc / cnt;
        }
    }
}

/* dense LU of the assembled coarsest Jacobian (R12) */
static int assemble_dense(const Oracle *O, OLevel *L)
{
    int m = 2 * L->nact;
    double *A = L->A;
    for (long i = 0; i < (long)m * m; i++) A[i] = 0.0;
    for (int r = 0; r < L->nact; r++) {
        long p = L->act[r];
        if (L->type[p] == T_IN) {
            JRow J;
            jrow_inside(O, L, p, &J);
            A[(long)(2 * r) * m + 2 * r] += J.ss_pp;
            A[(long)(2 * r) * m + 2 * r + 1] += J.sc_pp;
            for (int k = 0; k < J.nq; k++) {
                long qc = L->pos[J.q[k]];
                A[(long)(2 * r) * m + 2 * qc] += J.ss_q[k];
                A[(long)(2 * r) * m + 2 * qc + 1] += J.sc_q[k];
            }
            A[(long)(2 * r + 1) * m + 2 * r] += J.cs_pp;
            A[(long)(2 * r + 1) * m + 2 * r + 1] += J.cc_pp;
        } else {
            int gi = L->gpos[p];
            int nk = ipow3(L->dim);
            for (int kk = 0; kk < nk; kk++) {
                long node;
                double w = ghost_w(L, gi, kk, &node);
                if (w == 0.0) continue;
                A[(long)(2 * r) * m + 2 * L->pos[node]] += w;
            }
            double cs, cc;
            jrow_c(O, L, p, &cs, &cc);
            A[(long)(2 * r + 1) * m + 2 * r] += cs;
            A[(long)(2 * r + 1) * m + 2 * r + 1] += cc;
        }
    }
    return OR_OK;
}

static int lu_factor(double *A, int *piv, int m)
{
    for (int k = 0; k < m; k++) {
        int pr = k;
        double best = fabs(A[(long)k * m + k]);
        for (int i = k + 1; i < m; i++)
            if (fabs(A[(long)i * m + k]) > best) {
                best = fabs(A[(long)i * m + k]);
                pr = i;
            }
        piv[k] = pr;
        if (!(best > 0.0)) return OR_ENOTCONV;
        if (pr != k)
            for (int j = 0; j < m; j++) {
                double tmp = A[(long)k * m + j];
                A[(long)k * m + j] = A[(long)pr * m + j];
                A[(long)pr * m + j] = tmp;
            }
        for (int i = k + 1; i < m; i++) {
            double l = A[(long)i * m + k] / A[(long)k * m + k];
            A[(long)i * m + k] = l;
            for (int j = k + 1; j < m; j++) A[(long)i * m + j] -= l * A[(long)k * m + j];
        }
    }
    return OR_OK;
}

/* solve A x = b from the factors of lu_factor: the factorisation swapped whole
   rows, so P A = L U with P the product of the interchanges; apply them all to
   b in order, then forward substitution with the unit lower L and back
   substitution with U */
static void lu_solve(const double *A, const int *piv, int m, double *b)
{
    for (int k = 0; k < m; k++)
        if (piv[k] != k) {
            double t = b[k];
            b[k] = b[piv[k]];
            b[piv[k]] = t;
        }
    for (int i = 1; i < m; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= A[(long)i * m + k] * b[k];
        b[i] = s;
    }
    for (int i = m - 1; i >= 0; i--) {
        double s = b[i];
        for (int j = i + 1; j < m; j++) s -= A[(long)i * m + j] * b[j];
        b[i] = s / A[(long)i * m + i];
    }
}

static void coarsest_solve(OLevel *L)
{
    int m = 2 * L->nact;
    double *b = (double *)malloc(sizeof(double) * (m + 1));
    for (int r = 0; r < L->nact; r++) {
        b[2 * r] = L->rhs[2 * L->act[r]];
        b[2 * r + 1] = L->rhs[2 * L->act[r] + 1];
    }
    lu_solve(L->A, L->piv, m, b);
    for (long i = 0; i < 2 * L->nn; i++) L->x[i] = 0.0;
    for (int r = 0; r < L->nact; r++) {
        L->x[2 * L->act[r]] = b[2 * r];
        L->x[2 * L->act[r] + 1] = b[2 * r + 1];
    }
    free(b);
}

/* one V- (gamma = 1) or W- (gamma = 2) cycle on level l (Sec. 3.5) */
static void cycle(Oracle *O, int l)
{
    OLevel *L = &O->lev[l];
    if (l == O->L - 1) {
        coarsest_solve(L);
        return;
    }
    OLevel *C = &O->lev[l + 1];
    for (int k = 0; k < O->nu1; k++) smooth(O, L);
    residual(O, L);
    extend_defect(O, L);
    restrict_defect(L, C);
    for (long i = 0; i < 2 * C->nn; i++) C->x[i] = 0.0;
    int gam = O->cycle == 2 ? 2 : 1;
    for (int g = 0; g < gam; g++) cycle(O, l + 1);
    prolong_add(C, L);
    for (int k = 0; k < O->nu2; k++) smooth(O, L);
}

/* Full multigrid (cycle type 3, the first cycle of every linear solve): the
   right-hand side is carried down the hierarchy with the same boundary-aware
   restriction the cycles use (defect of x = 0 is the right-hand side itself,
   ghost defects extended into the band first), the coarsest system is solved
   directly, and on the way up each level starts from the interpolated coarse
   solution and takes one V-cycle (Sec. 3.5's transfers and smoother). */
static void fmg(Oracle *O)
{
    for (int l = 0; l + 1 < O->L; l++) {
        OLevel *L = &O->lev[l];
        for (long i = 0; i < 2 * L->nn; i++) L->x[i] = 0.0;
        residual(O, L);
        extend_defect(O, L);
        restrict_defect(L, &O->lev[l + 1]);
    }
    OLevel *C = &O->lev[O->L - 1];
    for (long i = 0; i < 2 * C->nn; i++) C->x[i] = 0.0;
    coarsest_solve(C);
    int saved = O->cycle;
    O->cycle = 1;
    for (int l = O->L - 2; l >= 0; l--) {
        OLevel *L = &O->lev[l];
        for (long i = 0; i < 2 * L->nn; i++) L->x[i] = 0.0;
        prolong_add(&O->lev[l + 1], L);
        cycle(O, l);
    }
    O->cycle = saved;
}

/* prepare coarse coefficients and the coarsest factorisation from lev[0].Wc */
static int prepare_hierarchy(Oracle *O)
{
    for (int l = 1; l < O->L; l++) inject_Wc(&O->lev[l - 1], &O->lev[l]);
    OLevel *C = &O->lev[O->L - 1];
    assemble_dense(O, C);
    if (lu_factor(C->A, C->piv, 2 * C->nact) != OR_OK) {
        snprintf(O->err, sizeof O->err, "singular coarsest Jacobian");
        return OR_ENOTCONV;
    }
    return OR_OK;
}

/* solve J x = rhs on the finest level by multigrid cycles; returns cycles used */
static int linear_solve(Oracle *O, double rnorm0)
{
    OLevel *L = &O->lev[0];
    for (long i = 0; i < 2 * L->nn; i++) L->x[i] = 0.0;
    if (O->L == 1) {
        coarsest_solve(L);
        return 1;
    }
    double rprev = rnorm0;
    int cyc;
    for (cyc = 1; cyc <= O->max_cycles; cyc++) {
        if (O->cycle == 3 && cyc == 1) {
            fmg(O);
        } else {
            int saved = O->cycle;
            if (O->cycle == 3) O->cycle = 1;
            cycle(O, 0);
            O->cycle = saved;
        }
        residual(O, L);
        double rn = maxabs_active(L, L->res);
        double rho = rprev > 0.0 ? rn / rprev : 0.0;
        if (O->nrho < OR_RHOMAX) {
            O->rho[O->nrho] = rho;
            O->rho_first[O->nrho] = (signed char)(cyc == 1);
            O->nrho++;
        }
        O->last_rho = rho;
        rprev = rn;
        if (rn <= O->lin_rtol * rnorm0 || rn != rn) break;
    }
    return cyc > O->max_cycles ? O->max_cycles : cyc;
}

/* one Crank-Nicolson step by Newton-Raphson (Sec. 3.1, Sec. 3.4, R13) */
static int cn_step(Oracle *O)
{
    OLevel *L = &O->lev[0];
    double *W = L->Wc;
    memcpy(O->Wn, W, sizeof(double) * 2 * L->nn);
    eval_F(O, W, O->Wn, O->F);
    double fn = maxabs_active(L, O->F);
    O->newton_last = 0;
    O->cycles_last = 0;
    if (fn < O->newton_tol) {
        O->t += O->dt;
        O->last_fnorm = fn;
        return OR_OK;
    }
    for (int k = 1; k <= O->max_newton; k++) {
        int rc = prepare_hierarchy(O);
        if (rc) return rc;
        memcpy(L->rhs, O->F, sizeof(double) * 2 * L->nn);
        int nc = linear_solve(O, fn);
        O->cycles_last += nc;
        O->cycles_total += nc;
        double wn = maxabs_active(L, W);
        for (long p = 0; p < L->nn; p++) {
            if (!active(L->type[p])) continue;
            W[2 * p] -= L->x[2 * p];
            W[2 * p + 1] -= L->x[2 * p + 1];
        }
        double dn = maxabs_active(L, L->x);
        eval_F(O, W, O->Wn, O->F);
        fn = maxabs_active(L, O->F);
        O->newton_last = k;
        O->newton_total++;
        O->last_fnorm = fn;
        if (fn != fn || dn != dn) break;
        double rel = wn > 0.0 ? dn / wn : dn;
        if ((fn < rel ? fn : rel) < O->newton_tol) {
            O->t += O->dt;
            O->steps_total++;
            return OR_OK;
        }
    }
    snprintf(O->err, sizeof O->err, "Newton did not converge (||F||=%g)", fn);
    return OR_ENOTCONV;
}

/* ------------------------------------------------------------------ */
/* public entry points (used from Python through ctypes)                */
/* ------------------------------------------------------------------ */

static void free_level(OLevel *L)
{
    free(L->phi); free(L->type); free(L->gidx); free(L->gpos); free(L->gkind); free(L->gm); free(L->gw); free(L->gB);
    free(L->gord); free(L->gth); free(L->gnt); free(L->gwk);
    free(L->bidx); free(L->bup); free(L->ban); free(L->Wc); free(L->rhs); free(L->x); free(L->res);
    free(L->act); free(L->pos); free(L->A); free(L->piv);
    memset(L, 0, sizeof *L);
}

void oracle_destroy(void *h)
{
    Oracle *O = (Oracle *)h;
    if (!O) return;
    for (int l = 0; l < O->L; l++) free_level(&O->lev[l]);
    free(O->Wn); free(O->F); free(O->rho); free(O->rho_first); free(O->src_store); free(O->sbg_store);
    free(O);
}

static char g_err[256];
const char *oracle_last_error(void) { return g_err; }

/* phi: (N+1)^dim node values, x fastest.  Box [lo,hi]^dim, h = (hi-lo)/N. */
void *oracle_create(const double *phi, int dim, double lo, double hi, int N, int coarsest_N, int *status)
{
    *status = OR_EINVAL;
    if (dim < 2 || dim > 3 || N < 2 || !(hi > lo) || coarsest_N < 2 || !phi) {
        snprintf(g_err, sizeof g_err, "invalid arguments");
        return NULL;
    }
    int nl = 1, Nl = N;
    while (Nl > coarsest_N) {
        if (Nl % 2) break;
        Nl /= 2;
        nl++;
    }
    if (Nl != coarsest_N || nl > OR_MAXLEV) {
        snprintf(g_err, sizeof g_err, "N must be coarsest_N times a power of two");
        return NULL;
    }
    Oracle *O = (Oracle *)calloc(1, sizeof(Oracle));
    if (!O) { *status = OR_ENOMEM; return NULL; }
    O->dim = dim;
    O->N = N;
    O->L = nl;
    /* defaults: model of Eq. dataeq with ICs/BC of Eq. BCnumtests, V(2,2) */
    O->a = 1e4; O->d = 0.1; O->m_s = 64.06; O->m_c = 100.09; O->alpha = 0.01; O->beta = 0.1;
    O->s_ext = 1.0; O->s0 = 0.0; O->c0 = 10.0;
    O->nu1 = 2; O->nu2 = 2; O->cycle = 1; O->max_newton = 20; O->max_cycles = 30; O->smoother = 0;
    O->ext_steps = 4;
    O->ghost_sweeps = 4;
    O->newton_tol = 1e-10; O->lin_rtol = 1e-10; O->tau_s = 0.9;
    O->rho = (double *)malloc(sizeof(double) * OR_RHOMAX);
    O->rho_first = (signed char *)malloc(OR_RHOMAX);
    for (int l = 0; l < nl; l++) {
        OLevel *L = &O->lev[l];
        L->dim = dim;
        L->N = N >> l;
        L->n = L->N + 1;
        L->nn = 1;
        for (int a = 0; a < dim; a++) L->nn *= L->n;
        L->st[0] = 1;
        L->st[1] = L->n;
        L->st[2] = (long)L->n * L->n;
        L->lo = lo;
        L->h = (hi - lo) / L->N;
        L->phi = (double *)malloc(sizeof(double) * L->nn);
        L->type = (signed char *)malloc(L->nn);
        L->Wc = (double *)calloc(2 * L->nn, sizeof(double));
        L->rhs = (double *)calloc(2 * L->nn, sizeof(double));
        L->x = (double *)calloc(2 * L->nn, sizeof(double));
        L->res = (double *)calloc(2 * L->nn, sizeof(double));
        if (!L->phi || !L->type || !L->Wc || !L->rhs || !L->x || !L->res) {
            oracle_destroy(O);
            *status = OR_ENOMEM;
            return NULL;
        }
        /* level-set coarsening by injection: phi_2h(I) = phi_h(2I) */
        if (l == 0) {
            memcpy(L->phi, phi, sizeof(double) * L->nn);
        } else {
            OLevel *F = &O->lev[l - 1];
            int ii[3];
            for (long I = 0; I < L->nn; I++) {
                coords(L, I, ii);
                long f = 0;
                for (int a = 0; a < dim; a++) f += (long)(2 * ii[a]) * F->st[a];
                L->phi[I] = F->phi[f];
            }
        }
        int rc = build_level_geometry(O, L, l == 0);
        if (rc != OR_OK) {
            snprintf(g_err, sizeof g_err, "%s", O->err);
            oracle_destroy(O);
            *status = rc;
            return NULL;
        }
    }
    OLevel *C = &O->lev[nl - 1];
    C->nact = 0;
    C->pos = (long *)malloc(sizeof(long) * C->nn);
    for (long i = 0; i < C->nn; i++) C->pos[i] = active(C->type[i]) ? C->nact++ : -1;
    C->act = (long *)malloc(sizeof(long) * (C->nact + 1));
    for (long i = 0; i < C->nn; i++)
        if (C->pos[i] >= 0) C->act[C->pos[i]] = i;
    C->A = (double *)malloc(sizeof(double) * 4 * (size_t)C->nact * C->nact + 8);
    C->piv = (int *)malloc(sizeof(int) * (2 * C->nact + 1));
    O->Wn = (double *)calloc(2 * O->lev[0].nn, sizeof(double));
    O->F = (double *)calloc(2 * O->lev[0].nn, sizeof(double));
    if (!C->A || !C->piv || !O->Wn || !O->F) {
        oracle_destroy(O);
        *status = OR_ENOMEM;
        return NULL;
    }
    O->dt = 1.0;
    *status = OR_OK;
    return O;
}

static void reset_state(Oracle *O)
{
    OLevel *L = &O->lev[0];
    for (long p = 0; p < L->nn; p++) {
        int act = active(L->type[p]);
        L->Wc[2 * p] = act ? O->s0 : 0.0;
        L->Wc[2 * p + 1] = act ? O->c0 : 0.0;
    }
    O->t = 0.0;
}

/* params: a, d, m_s, m_c, alpha, beta, s_ext, s0, c0 (Eq. maineq, Eq. dataeq);
   resets the state to the uniform initial condition, ghosts included (ICs are
   extrapolated exactly when they are uniform) */
int oracle_set_model(void *h, const double *p)
{
    Oracle *O = (Oracle *)h;
    O->a = p[0]; O->d = p[1]; O->m_s = p[2]; O->m_c = p[3]; O->alpha = p[4]; O->beta = p[5];
    O->s_ext = p[6]; O->s0 = p[7]; O->c0 = p[8];
    reset_state(O);
    return OR_OK;
}

/* smoother: 0 red-black collective GS, 1 red-black pointwise GS, 2 lexicographic collective GS;
   cycle_type: 1 V, 2 W, 3 full multigrid first, then V-cycles */
int oracle_set_solver(void *h, int nu1, int nu2, int cycle_type, int max_newton, int max_cycles,
                      double newton_tol, double lin_rtol, double tau_s, int smoother, int ghost_sweeps)
{
    Oracle *O = (Oracle *)h;
    if (nu1 < 0 || nu2 < 0 || cycle_type < 1 || cycle_type > 3 || max_newton < 1 || max_cycles < 1 ||
        !(tau_s > 0.0 && tau_s < 1.0) || smoother < 0 || smoother > 2 || ghost_sweeps < 1)
        return OR_EINVAL;
    O->ghost_sweeps = ghost_sweeps;
    O->nu1 = nu1; O->nu2 = nu2; O->cycle = cycle_type; O->max_newton = max_newton; O->max_cycles = max_cycles;
    O->newton_tol = newton_tol; O->lin_rtol = lin_rtol; O->tau_s = tau_s; O->smoother = smoother;
    return OR_OK;
}

int oracle_step(void *h, double dt, int nsteps)
{
    Oracle *O = (Oracle *)h;
    if (!(dt > 0.0) || nsteps < 0) return OR_EINVAL;
    O->dt = dt;
    for (int k = 0; k < nsteps; k++) {
        int rc = cn_step(O);
        if (rc) {
            snprintf(g_err, sizeof g_err, "%s", O->err);
            return rc;
        }
    }
    return OR_OK;
}

int oracle_get_state(void *h, double *s, double *c, signed char *type)
{
    Oracle *O = (Oracle *)h;
    OLevel *L = &O->lev[0];
    for (long p = 0; p < L->nn; p++) {
        int act = active(L->type[p]);
        if (s) s[p] = act ? L->Wc[2 * p] : 0.0;
        if (c) c[p] = act ? L->Wc[2 * p + 1] : 0.0;
        if (type) type[p] = act ? L->type[p] : 0;
    }
    return OR_OK;
}

int oracle_set_state(void *h, const double *s, const double *c, double t)
{
    Oracle *O = (Oracle *)h;
    OLevel *L = &O->lev[0];
    for (long p = 0; p < L->nn; p++) {
        int act = active(L->type[p]);
        L->Wc[2 * p] = act ? s[p] : 0.0;
        L->Wc[2 * p + 1] = act ? c[p] : 0.0;
    }
    O->t = t;
    return OR_OK;
}

/* stats: [newton_last, cycles_last, newton_total, cycles_total, nrho] and
   [t, last_rho, last_fnorm] */
int oracle_get_stats(void *h, long *istats, double *dstats)
{
    Oracle *O = (Oracle *)h;
    istats[0] = O->newton_last;
    istats[1] = O->cycles_last;
    istats[2] = O->newton_total;
    istats[3] = O->cycles_total;
    istats[4] = O->nrho;
    dstats[0] = O->t;
    dstats[1] = O->last_rho;
    dstats[2] = O->last_fnorm;
    return OR_OK;
}

int oracle_get_rho(void *h, double *rho, signed char *first, int maxn)
{
    Oracle *O = (Oracle *)h;
    int n = O->nrho < maxn ? O->nrho : maxn;
    memcpy(rho, O->rho, sizeof(double) * n);
    memcpy(first, O->rho_first, n);
    return n;
}

void oracle_clear_rho(void *h) { ((Oracle *)h)->nrho = 0; }

/* ---------------- test hooks ---------------- */

int oracle_num_levels(void *h) { return ((Oracle *)h)->L; }

/* info: [N, n, ng, nb, nact (coarsest only, else 0), quadratic, linear, identity ghost rows] */
int oracle_level_info(void *h, int l, long *info)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    OLevel *L = &O->lev[l];
    info[0] = L->N;
    info[1] = L->n;
    info[2] = L->ng;
    info[3] = L->nb;
    info[4] = l == O->L - 1 ? L->nact : 0;
    info[5] = info[6] = info[7] = 0;
    for (int gi = 0; gi < L->ng; gi++) info[5 + L->gkind[gi]]++;
    return OR_OK;
}

int oracle_level_type(void *h, int l, signed char *type)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    memcpy(type, O->lev[l].type, O->lev[l].nn);
    return OR_OK;
}

int oracle_level_phi(void *h, int l, double *phi)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    memcpy(phi, O->lev[l].phi, sizeof(double) * O->lev[l].nn);
    return OR_OK;
}

/* ghosts in box order: idx[ng], kind[ng], m[ng*dim], w[ng*dim*3], B[ng*dim] */
int oracle_level_ghosts(void *h, int l, long *idx, signed char *kind, signed char *m, double *w, double *B)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    OLevel *L = &O->lev[l];
    memcpy(idx, L->gidx, sizeof(long) * L->ng);
    memcpy(kind, L->gkind, L->ng);
    memcpy(m, L->gm, (size_t)L->ng * L->dim);
    memcpy(w, L->gw, sizeof(double) * 3 * L->dim * L->ng);
    memcpy(B, L->gB, sizeof(double) * L->dim * L->ng);
    return OR_OK;
}

/* per-ghost member weights (ng x 3^dim, member kk = k0 + 3 k1 + 9 k2 at node
   g - sum_a m_a k_a e_a) and the unit normal of phi~ at B (ng x dim) */
int oracle_level_rows(void *h, int l, double *wk, double *nt)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    OLevel *L = &O->lev[l];
    memcpy(wk, L->gwk, sizeof(double) * ipow3(L->dim) * L->ng);
    memcpy(nt, L->gnt, sizeof(double) * L->dim * L->ng);
    return OR_OK;
}

int oracle_level_band(void *h, int l, long *idx, long *up, double *an)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    OLevel *L = &O->lev[l];
    memcpy(idx, L->bidx, sizeof(long) * L->nb);
    memcpy(up, L->bup, sizeof(long) * L->dim * L->nb);
    memcpy(an, L->ban, sizeof(double) * L->dim * L->nb);
    return OR_OK;
}

/* per-ghost boundary values s_b(B_g) of the finest level (NULL: constant s_ext) */
int oracle_set_ghost_sb(void *h, const double *sb)
{
    Oracle *O = (Oracle *)h;
    free(O->sbg_store);
    O->sbg_store = NULL;
    O->sbg = NULL;
    if (!sb) return OR_OK;
    int ng = O->lev[0].ng;
    O->sbg_store = (double *)malloc(sizeof(double) * (ng + 1));
    memcpy(O->sbg_store, sb, sizeof(double) * ng);
    O->sbg = O->sbg_store;
    return OR_OK;
}

/* source terms of the manufactured-solution tests (Sec. 4.1) at t_n and t_{n+1},
   node values of the finest level; NULL clears them */
/* boundary condition for s: 0 Dirichlet (Eq. BCs), 1 Neumann (Eq. BCsN, Sec.
   3.6) with s_b the prescribed normal derivative; rebuilds the ghost rows of
   every level */
int oracle_set_bc(void *h, int bc)
{
    Oracle *O = (Oracle *)h;
    if (bc != 0 && bc != 1) return OR_EINVAL;
    O->bc = bc;
    for (int l = 0; l < O->L; l++) {
        int rc = build_ghost_rows(O, &O->lev[l], l == 0, bc);
        if (rc) return rc;
    }
    return OR_OK;
}

int oracle_set_sources(void *h, const double *f1o, const double *f1n, const double *f2o, const double *f2n)
{
    Oracle *O = (Oracle *)h;
    free(O->src_store);
    O->src_store = NULL;
    O->f1o = O->f1n = O->f2o = O->f2n = NULL;
    if (!f1o) return OR_OK;
    long nn = O->lev[0].nn;
    O->src_store = (double *)malloc(sizeof(double) * 4 * nn);
    memcpy(O->src_store, f1o, sizeof(double) * nn);
    memcpy(O->src_store + nn, f1n, sizeof(double) * nn);
    memcpy(O->src_store + 2 * nn, f2o, sizeof(double) * nn);
    memcpy(O->src_store + 3 * nn, f2n, sizeof(double) * nn);
    O->f1o = O->src_store;
    O->f1n = O->src_store + nn;
    O->f2o = O->src_store + 2 * nn;
    O->f2n = O->src_store + 3 * nn;
    return OR_OK;
}

/* F(W; W^n) on the finest level with time step dt; arrays interleaved (s,c) */
int oracle_eval_F(void *h, double dt, const double *W, const double *Wn, double *F)
{
    Oracle *O = (Oracle *)h;
    O->dt = dt;
    eval_F(O, W, Wn, F);
    return OR_OK;
}

/* J(Wc) x on level l with time step dt */
int oracle_apply_J(void *h, int l, double dt, const double *Wc, const double *x, double *out)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    OLevel *L = &O->lev[l];
    O->dt = dt;
    memcpy(L->Wc, Wc, sizeof(double) * 2 * L->nn);
    apply_J(O, L, x, out);
    return OR_OK;
}

/* dense Jacobian of the finest level (rows/cols: active nodes in box order,
   (s,c) interleaved), m = 2 * number of active nodes, caller allocates m*m */
int oracle_dense_J(void *h, double dt, const double *Wc, double *dense, long *act)
{
    Oracle *O = (Oracle *)h;
    OLevel *L = &O->lev[0];
    O->dt = dt;
    memcpy(L->Wc, Wc, sizeof(double) * 2 * L->nn);
    int na = 0;
    for (long i = 0; i < L->nn; i++)
        if (active(L->type[i])) na++;
    OLevel tmp = *L;
    tmp.nact = na;
    tmp.act = act;
    tmp.pos = (long *)malloc(sizeof(long) * L->nn);
    int k = 0;
    for (long i = 0; i < L->nn; i++) {
        tmp.pos[i] = active(L->type[i]) ? k : -1;
        if (tmp.pos[i] >= 0) act[k++] = i;
    }
    tmp.A = dense;
    assemble_dense(O, &tmp);
    free(tmp.pos);
    return na;
}

/* sweeps of the relaxation of Sec. 3.5.1 on level l: x updated in place */
int oracle_smooth(void *h, int l, double dt, const double *Wc, const double *rhs, double *x, int sweeps)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    OLevel *L = &O->lev[l];
    O->dt = dt;
    memcpy(L->Wc, Wc, sizeof(double) * 2 * L->nn);
    memcpy(L->rhs, rhs, sizeof(double) * 2 * L->nn);
    memcpy(L->x, x, sizeof(double) * 2 * L->nn);
    for (int k = 0; k < sweeps; k++) smooth(O, L);
    memcpy(x, L->x, sizeof(double) * 2 * L->nn);
    return OR_OK;
}

/* restriction of the defect of level l (res given on active nodes) to level
   l+1, with the band extension; also returns the extended fine defect */
int oracle_restrict(void *h, int l, double *res, double *rhs_coarse)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l + 1 >= O->L) return OR_EINVAL;
    OLevel *L = &O->lev[l], *C = &O->lev[l + 1];
    memcpy(L->res, res, sizeof(double) * 2 * L->nn);
    extend_defect(O, L);
    restrict_defect(L, C);
    memcpy(res, L->res, sizeof(double) * 2 * L->nn);
    memcpy(rhs_coarse, C->rhs, sizeof(double) * 2 * C->nn);
    return OR_OK;
}

/* x_fine += P x_coarse (level l+1 to level l) */
int oracle_prolong(void *h, int l, const double *xc, double *xf)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l + 1 >= O->L) return OR_EINVAL;
    OLevel *L = &O->lev[l], *C = &O->lev[l + 1];
    memcpy(C->x, xc, sizeof(double) * 2 * C->nn);
    memcpy(L->x, xf, sizeof(double) * 2 * L->nn);
    prolong_add(C, L);
    memcpy(xf, L->x, sizeof(double) * 2 * L->nn);
    return OR_OK;
}

/* coarse coefficients from the finest Wc (returns level l's Wc) */
int oracle_inject(void *h, const double *Wc0, int l, double *Wc_out)
{
    Oracle *O = (Oracle *)h;
    if (l < 0 || l >= O->L) return OR_EINVAL;
    memcpy(O->lev[0].Wc, Wc0, sizeof(double) * 2 * O->lev[0].nn);
    for (int k = 1; k <= l; k++) inject_Wc(&O->lev[k - 1], &O->lev[k]);
    memcpy(Wc_out, O->lev[l].Wc, sizeof(double) * 2 * O->lev[l].nn);
    return OR_OK;
}

/* ncycles multigrid cycles for J(Wc0) x = rhs on the finest level from x (in/out);
   residual max-norms after each cycle in rnorms.  The finest Wc is overwritten. */
int oracle_cycles(void *h, double dt, const double *Wc0, const double *rhs, double *x, int ncycles, double *rnorms)
{
    Oracle *O = (Oracle *)h;
    OLevel *L = &O->lev[0];
    O->dt = dt;
    memcpy(L->Wc, Wc0, sizeof(double) * 2 * L->nn);
    int rc = prepare_hierarchy(O);
    if (rc) return rc;
    memcpy(L->rhs, rhs, sizeof(double) * 2 * L->nn);
    memcpy(L->x, x, sizeof(double) * 2 * L->nn);
    for (int k = 0; k < ncycles; k++) {
        if (O->L == 1)
            coarsest_solve(L);
        else if (O->cycle == 3 && k == 0)
            fmg(O); /* full multigrid starts from x = 0 */
        else
            cycle(O, 0);
        residual(O, L);
        rnorms[k] = maxabs_active(L, L->res);
    }
    memcpy(x, L->x, sizeof(double) * 2 * L->nn);
    return OR_OK;
}

/* the assembled Jacobian of the coarsest level after injecting the finest Wc0
   (2*nact rows, active nodes in box order, (s,c) interleaved); returns nact */
int oracle_coarsest_matrix(void *h, double dt, const double *Wc0, double *A_out)
{
    Oracle *O = (Oracle *)h;
    O->dt = dt;
    memcpy(O->lev[0].Wc, Wc0, sizeof(double) * 2 * O->lev[0].nn);
    for (int l = 1; l < O->L; l++) inject_Wc(&O->lev[l - 1], &O->lev[l]);
    OLevel *C = &O->lev[O->L - 1];
    assemble_dense(O, C);
    memcpy(A_out, C->A, sizeof(double) * 4 * (size_t)C->nact * C->nact);
    return C->nact;
}

/* solve the coarsest level's system for a given right-hand side (level-sized,
   interleaved), after injecting the finest Wc0 and factoring */
int oracle_coarsest_solve(void *h, double dt, const double *Wc0, const double *rhs_c, double *x_c)
{
    Oracle *O = (Oracle *)h;
    O->dt = dt;
    memcpy(O->lev[0].Wc, Wc0, sizeof(double) * 2 * O->lev[0].nn);
    int rc = prepare_hierarchy(O);
    if (rc) return rc;
    OLevel *C = &O->lev[O->L - 1];
    memcpy(C->rhs, rhs_c, sizeof(double) * 2 * C->nn);
    coarsest_solve(C);
    memcpy(x_c, C->x, sizeof(double) * 2 * C->nn);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* level-set preprocessing (Sec. 2)                                     */
/* ------------------------------------------------------------------ */

/* one-sided differences of v at box node i along axis a; a missing neighbour
   (box edge) gives a zero difference on that side */
static void one_sided(const double *v, long i, const int *ii, int a, int N, const long *st, double h, double *dm,
                      double *dp)
{
    *dm = ii[a] > 0 ? (v[i] - v[i - st[a]]) / h : 0.0;
    *dp = ii[a] < N ? (v[i + st[a]] - v[i]) / h : 0.0;
}

/* Reinitialization (Sec. 2): the PDE d phi_d / d mu = sgn(phi)(1 - |grad phi_d|)
   with phi_d = phi at mu = 0, marched `steps` explicit Euler steps of
   d mu = h / dim.  sgn is the smoothed sign phi / sqrt(phi^2 + h^2) of the
   initial phi; |grad phi_d| is Godunov's upwind approximation from the
   one-sided differences (first order), chosen by the sign of phi: where
   phi > 0, sqrt(sum_a max(max(D-_a,0)^2, min(D+_a,0)^2)); where phi < 0,
   sqrt(sum_a max(min(D-_a,0)^2, max(D+_a,0)^2)).  phi_out may alias nothing. */
int oracle_reinit(const double *phi0, int dim, int N, double h, int steps, double *phi_out)
{
    if ((dim != 2 && dim != 3) || N < 2 || !(h > 0) || steps < 0) return OR_EINVAL;
    long n = N + 1, nn = dim == 2 ? n * n : n * n * n;
    long st[3] = {1, n, n * n};
    double *a = (double *)malloc(sizeof(double) * nn), *b = (double *)malloc(sizeof(double) * nn);
    if (!a || !b) {
        free(a);
        free(b);
        return OR_ENOMEM;
    }
    memcpy(a, phi0, sizeof(double) * nn);
    const double dmu = h / dim;
    for (int k = 0; k < steps; k++) {
        for (long i = 0; i < nn; i++) {
            int ii[3] = {(int)(i % n), (int)((i / n) % n), (int)(i / (n * n))};
            double p0 = phi0[i];
            double sg = p0 / sqrt(p0 * p0 + h * h);
            double g2 = 0.0;
            for (int ax = 0; ax < dim; ax++) {
                double dm, dp;
                one_sided(a, i, ii, ax, N, st, h, &dm, &dp);
                double l, r;
                if (p0 > 0.0) {
                    l = dm > 0.0 ? dm : 0.0;
                    r = dp < 0.0 ? dp : 0.0;
                } else {
                    l = dm < 0.0 ? dm : 0.0;
                    r = dp > 0.0 ? dp : 0.0;
                }
                g2 += l * l > r * r ? l * l : r * r;
            }
            b[i] = p0 == 0.0 ? a[i] : a[i] - dmu * sg * (sqrt(g2) - 1.0);
        }
        double *t = a;
        a = b;
        b = t;
    }
    memcpy(phi_out, a, sizeof(double) * nn);
    free(a);
    free(b);
    return OR_OK;
}

/* A provisional level set from a binary mask (Sec. 2): phi = -1 inside
   (mask != 0), +1 outside, then `steps` explicit steps of the heat equation
   phi += lambda sum_q (phi_q - phi) over the axis neighbours present in the
   box, lambda = 1 / (4 dim) (half the stability limit). */
int oracle_mask_levelset(const unsigned char *mask, int dim, int N, int steps, double *phi_out)
{
    if ((dim != 2 && dim != 3) || N < 2 || steps < 0) return OR_EINVAL;
    long n = N + 1, nn = dim == 2 ? n * n : n * n * n;
    long st[3] = {1, n, n * n};
    double *a = (double *)malloc(sizeof(double) * nn), *b = (double *)malloc(sizeof(double) * nn);
    if (!a || !b) {
        free(a);
        free(b);
        return OR_ENOMEM;
    }
    for (long i = 0; i < nn; i++) a[i] = mask[i] ? -1.0 : 1.0;
    const double lam = 1.0 / (4.0 * dim);
    for (int k = 0; k < steps; k++) {
        for (long i = 0; i < nn; i++) {
            int ii[3] = {(int)(i % n), (int)((i / n) % n), (int)(i / (n * n))};
            double acc = 0.0;
            for (int ax = 0; ax < dim; ax++) {
                if (ii[ax] > 0) acc += a[i - st[ax]] - a[i];
                if (ii[ax] < N) acc += a[i + st[ax]] - a[i];
            }
            b[i] = a[i] + lam * acc;
        }
        double *t = a;
        a = b;
        b = t;
    }
    memcpy(phi_out, a, sizeof(double) * nn);
    free(a);
    free(b);
    return OR_OK;
}

/* Extrapolation of initial data to the ghosts (Sec. 3.3: the ICs of s and c
   are extrapolated outside the domain with second order, by the PDE approach
   of the cited extrapolation technique).  For a field u known at the inside
   nodes (phi < 0) of the finest level:
     1. u_n = n . grad u by central differences where all axis neighbours are
        inside, n = grad phi / |grad phi| (Eq. ncurv, central differences);
     2. u_n extended to the other nodes by `iters` Jacobi steps of
        d q / d tau + n . grad q = 0, i.e. q <- q - (dtau / h) sum_a |n_a|
        (q - q_up(a)), with q_up(a) the neighbour toward the inside along axis
        a (index i - sign(n_a)), dtau = h / 2;
     3. u extended linearly to the non-inside nodes by `iters` Jacobi steps of
        d u / d tau + n . grad u = u_n, i.e. u <- u - dtau ((1/h) sum_a |n_a|
        (u - u_up(a)) - u_n).
   Known values never change; unknown ones start at 0.  u is overwritten at
   the non-inside nodes (all of the box: callers read the ghosts). */
int oracle_extrapolate(const double *phi, const signed char *type, int dim, int N, double h, int iters, double *u)
{
    if ((dim != 2 && dim != 3) || N < 2 || !(h > 0) || iters < 0) return OR_EINVAL;
    long n = N + 1, nn = dim == 2 ? n * n : n * n * n;
    long st[3] = {1, n, n * n};
    double *nv = (double *)calloc((size_t)dim * nn, sizeof(double));
    double *q = (double *)calloc(nn, sizeof(double)), *q2 = (double *)calloc(nn, sizeof(double));
    double *v2 = (double *)malloc(sizeof(double) * nn);
    signed char *kn = (signed char *)calloc(nn, 1);
    if (!nv || !q || !q2 || !v2 || !kn) {
        free(nv); free(q); free(q2); free(v2); free(kn);
        return OR_ENOMEM;
    }
    /* normals and u_n where the central stencil is inside */
    for (long i = 0; i < nn; i++) {
        int ii[3] = {(int)(i % n), (int)((i / n) % n), (int)(i / (n * n))};
        double g[3] = {0, 0, 0}, gn = 0.0;
        for (int a = 0; a < dim; a++) {
            int lo = ii[a] > 0, hi = ii[a] < N;
            if (lo && hi) g[a] = (phi[i + st[a]] - phi[i - st[a]]) / (2.0 * h);
            else if (hi) g[a] = (phi[i + st[a]] - phi[i]) / h;
            else g[a] = (phi[i] - phi[i - st[a]]) / h;
            gn += g[a] * g[a];
        }
        gn = sqrt(gn);
        for (int a = 0; a < dim; a++) nv[(size_t)dim * i + a] = gn > 0.0 ? g[a] / gn : 0.0;
        if (type[i] != T_IN) continue;
        int ok = 1;
        for (int a = 0; a < dim; a++) {
            if (ii[a] == 0 || ii[a] == N || type[i - st[a]] != T_IN || type[i + st[a]] != T_IN) ok = 0;
        }
        if (!ok) continue;
        double un = 0.0;
        for (int a = 0; a < dim; a++) un += nv[(size_t)dim * i + a] * (u[i + st[a]] - u[i - st[a]]) / (2.0 * h);
        q[i] = un;
        kn[i] = 1;
    }
    const double dtau = 0.5 * h;
    /* the upwind neighbour of node i along axis a, or -1 */
#define UPW(i, a)                                                                                          \
    (nv[(size_t)dim * (i) + (a)] == 0.0                                                                    \
         ? -1L                                                                                             \
         : ((nv[(size_t)dim * (i) + (a)] > 0.0) ? ((((i) / st[a]) % n) > 0 ? (i) - st[a] : -1L)             \
                                                 : ((((i) / st[a]) % n) < N ? (i) + st[a] : -1L)))
    for (int it = 0; it < iters; it++) {
        for (long i = 0; i < nn; i++) {
            if (kn[i]) {
                q2[i] = q[i];
                continue;
            }
            double acc = 0.0;
            for (int a = 0; a < dim; a++) {
                long up = UPW(i, a);
                if (up < 0) continue;
                acc += fabs(nv[(size_t)dim * i + a]) * (q[i] - q[up]);
            }
            q2[i] = q[i] - (dtau / h) * acc;
        }
        double *t = q; q = q2; q2 = t;
    }
    for (long i = 0; i < nn; i++)
        if (type[i] != T_IN) u[i] = 0.0;
    for (int it = 0; it < iters; it++) {
        for (long i = 0; i < nn; i++) {
            if (type[i] == T_IN) {
                v2[i] = u[i];
                continue;
            }
            double acc = 0.0;
            for (int a = 0; a < dim; a++) {
                long up = UPW(i, a);
                if (up < 0) continue;
                acc += fabs(nv[(size_t)dim * i + a]) * (u[i] - u[up]);
            }
            v2[i] = u[i] - dtau * (acc / h - q[i]);
        }
        memcpy(u, v2, sizeof(double) * nn);
    }
#undef UPW
    free(nv); free(q); free(q2); free(v2); free(kn);
    return OR_OK;
}
