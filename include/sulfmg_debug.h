/*
 * sulfmg_debug.h -- stage-level entry points of the sulfmg library, for
 * checking each stage of the method on its own (arXiv:1902.07029, Sec. 3).
 *
 * Each call runs the library's CUDA kernels for one stage on caller-supplied
 * host inputs and copies the result back; the host arrays are only marshalled.
 * Vectors are interleaved (s, c) pairs per node, 2*(n^dim) doubles for a level
 * with n nodes per axis.  The calls use the handle's work arrays and OVERWRITE
 * its state: use a dedicated handle.  Errors as in sulfmg.h.
 */
#ifndef SULFMG_DEBUG_H
#define SULFMG_DEBUG_H

#include <stdint.h>
#include "sulfmg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* info (11 entries): N, n, ghosts, band nodes, active nodes of the coarsest
   level (0 on other levels), inside nodes, then the ghost-row kinds:
   quadratic, linear, identity (Sec. 3.3 and its fallbacks), then the entries
   of the level's composed ghost relaxation (Eq. RelGhost, all passes of a
   sweep as one affine map; -1 when the level relaxes pass by pass) and the
   passes it composes (0 when none). */
int sulf_dbg_level_info(sulf_handle h, int level, int64_t* info);

/* node types of a level: 0 inactive, 1 inside, 2 ghost, 3 band (inactive nodes
   that receive the extended boundary defect, Sec. 3.5.2) */
int sulf_dbg_level_type(sulf_handle h, int level, int8_t* type);

/* ghost rows of a level in box order: node index, kind (0 quadratic, 1 linear,
   2 identity), upwind signs m_a (dim per ghost), 1-D weights at offsets 0,1,2
   (3*dim per ghost, Eq. intcoeffsD), boundary point B (dim per ghost) */
int sulf_dbg_level_ghosts(sulf_handle h, int level, int64_t* idx, int8_t* kind, int8_t* m, double* w,
                          double* B);

/* the boundary rows of a level as member weights, ghost-major: wk holds
   3^dim weights per ghost (member kk = k0 + 3 k1 + 9 k2 at node
   g - sum_a m_a k_a e_a; Eq. JssD for Dirichlet, Eq. JccN for Neumann), nt the
   unit normal of the interpolated level set at B (dim per ghost, Eq.
   Neumanntilde) */
int sulf_dbg_level_rows(sulf_handle h, int level, double* wk, double* nt);

/* Newton residual F(W; W^n) of Eqs. FDs, FDc, BCs on the finest level */
int sulf_dbg_eval_F(sulf_handle h, double dt, const double* W, const double* Wn, double* F);

/* J(Wc) x on a level (Eqs. JssI-JccI, exact derivative) */
int sulf_dbg_apply_J(sulf_handle h, int level, double dt, const double* Wc, const double* x, double* out);

/* sweeps of the relaxation of Sec. 3.5.1 on a level; x in/out */
int sulf_dbg_smooth(sulf_handle h, int level, double dt, const double* Wc, const double* rhs, double* x,
                    int sweeps);

/* restriction of a defect from level to level+1 (Sec. 3.5.2): res in/out (the
   band entries are filled by the normal extension), rhs_coarse out */
int sulf_dbg_restrict(sulf_handle h, int level, double* res, double* rhs_coarse);

/* x_fine += interpolated x_coarse, level+1 to level (Sec. 3.5.3) */
int sulf_dbg_prolong(sulf_handle h, int level, const double* xc, double* xf);

/* coefficients (s, c) of level l injected from the finest-level Wc0 */
int sulf_dbg_inject(sulf_handle h, const double* Wc0, int level, double* Wc_out);

/* direct solve on the coarsest level (Sec. 3.5, dense LU of the assembled
   Jacobian) after injecting the finest-level Wc0: rhs_c and x_c are
   coarsest-level vectors */
int sulf_dbg_coarsest_solve(sulf_handle h, double dt, const double* Wc0, const double* rhs_c, double* x_c);

/* ncycles multigrid cycles for J(Wc0) x = rhs on the finest level, x in/out;
   |r|_inf after each cycle in rnorms.  Uses the handle's solver controls. */
int sulf_dbg_cycles(sulf_handle h, double dt, const double* Wc0, const double* rhs, double* x, int ncycles,
                    double* rnorms);

#ifdef __cplusplus
}
#endif
#endif /* SULFMG_DEBUG_H */
