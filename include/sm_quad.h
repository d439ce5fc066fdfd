/* sm_quad.h -- C ABI of the 2-D and axisymmetric variants of the library
 * (arXiv:1708.08434, Sec. 1 and 2.1.1: 2-D, axisymmetric and 3-D runs on
 * quadtree / octree grids):
 *
 *   - quadtree of fixed 8^2-cell boxes with proper nesting    (Sec. 2.1.1)
 *   - geometric multigrid for Poisson's equation, FAS V-cycle and FMG with
 *     red-black Gauss-Seidel smoothing                         (Sec. 2.1.2, Eq. 1, 5)
 *   - cell-centred field, Koren-limited drift-diffusion-reaction step with
 *     refinement-boundary fluxes, Heun time stepping and its limits
 *                                                               (Sec. 2.2-2.4, Eq. 2-3, 6-7)
 *
 * in Cartesian (x, y) or cylindrical (r, z) coordinates.  The paper states
 * no 2-D or cylindrical formulas; the library implements the finite-volume
 * forms of the 3-D rules: the 5-point operator, and in cylindrical
 * coordinates (1/r) d/dr (r d/dr) + d2/dz2 with radial face fluxes weighted
 * by the face radius over the cell-centre radius (no flux through the axis),
 * restriction and refinement-face flux means weighted by volume and area;
 * coarse-fine potential ghost phi_f/3 + 2 phihat/3, phihat = 3/4 c + 1/4 c_t;
 * prolongation (2c + c_x + c_y)/4.
 *
 * Conventions are those of sm_streamer.h (status codes, stream ordering, one
 * caller-owned arena, no CPU fallback), with 2-D fields: each variable is an
 * array of [max_boxes][64] doubles, box b the b-th table entry (boxes sorted
 * by level, then 2-D Morton key with x in bit 0), cell (i,j) at i + 8 j.
 * Faces are numbered 0..3 = -x,+x,-y,+y.  In the axisymmetric geometry x is
 * the radius r (the axis is face -x, origin[0] must be 0, and its boundary
 * setting is ignored) and y is the axial coordinate z.
 */
#ifndef SM_QUAD_H
#define SM_QUAD_H

#include <stddef.h>
#include <stdint.h>

#include "sm_streamer.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sm_quad sm_quad;  /* opaque, owned by the library */

typedef enum { SM_CARTESIAN = 0, SM_AXISYMMETRIC = 1 } sm_geometry;

/* Domain [origin, origin + length]^2 on a base grid of nb^2 boxes (nb a
 * power of two: levels 0 .. log2(nb) are uniform multigrid levels with 2^l
 * boxes per side), refined up to max_level levels above the base.
 * bc_type per face: 0 = Neumann zero, 1 = Dirichlet with value bc_val
 * (potential).  Densities use Neumann zero walls.  At least one face must
 * be Dirichlet. */
typedef struct {
  double length;
  double origin[2];
  int nb;
  int max_level;
  int geometry;            /* sm_geometry */
  int bc_type[4];
  double bc_val[4];
} sm_quad_domain;

/* Create a context for at most max_boxes boxes with V(nu1,nu2) cycles on
 * `stream` (cudaStream_t as void*).  The uniform levels 0 .. log2(nb) are
 * built when the arena is bound.  Errors: SM_EINVAL (bad domain, nu < 1,
 * max_boxes below the uniform levels), SM_ECUDA (no device). */
int sm_quad_create(sm_quad **out, const sm_quad_domain *dom, int max_boxes, int nu1, int nu2,
                   void *stream);
int sm_quad_destroy(sm_quad *q);
/* bytes of the device arena the caller must allocate (256-byte aligned) */
int sm_quad_arena_size(const sm_quad *q, size_t *bytes);
/* hand over the arena; zeroes every field and uploads the uniform levels'
 * tables.  SM_ENOMEM if too small, SM_EINVAL if misaligned. */
int sm_quad_bind_arena(sm_quad *q, void *dev_ptr, size_t bytes);

/* Refine the flagged boxes (host int8 per box of `level`, > 0 = refine) of
 * the finest level.  Proper nesting: a box is refined only if all 8
 * neighbour positions of its level hold a box or lie outside the domain;
 * other requests are counted in *n_dropped.  Out: boxes added.  New boxes'
 * fields are zero.  SM_ESTATE unless `level` is the finest level below the
 * maximum; SM_ENOMEM past max_boxes. */
int sm_quad_refine_level(sm_quad *q, int level, const int8_t *flags, int *n_new, int *n_dropped);

/* Table copies into host arrays (any may be NULL): level_offset
 * [n_levels+1], level [n], ij [2n], morton [n], parent [n] (-1 at level 0),
 * child [4n] (-1: leaf; child c at (2i + (c&1), 2j + (c>>1))), nbr [8n]
 * (directions (dx,dy) in x-fastest order without (0,0); -1 outside the
 * domain, -2 no box of that level). */
int sm_quad_get_tables(const sm_quad *q, int *n_boxes, int *n_levels, int32_t *level_offset,
                       int32_t *level, int32_t *ij, uint64_t *morton, int32_t *parent,
                       int32_t *child, int32_t *nbr);

/* Device pointer of a field (sm_var numbering; [max_boxes][64] doubles). */
int sm_quad_var_ptr(sm_quad *q, int var, double **dev);
/* Synchronous copies of the first n_boxes boxes of a field from / to host
 * memory ([n_boxes][64] doubles). */
int sm_quad_upload(sm_quad *q, int var, const double *host);
int sm_quad_download(sm_quad *q, int var, double *host);

/* Transport coefficients sampled at E_k = k e_max/(n-1), k = 0..n-1 (host
 * arrays; linear interpolation, clamped at the ends; Sec. 2.3).
 * 2 <= n <= 4096. */
int sm_quad_set_table(sm_quad *q, int n, double e_max, const double *mu, const double *diff,
                      const double *alpha);

/* Eq. 5 right-hand side on leaf cells: f = -charge (n_i - n_e)/eps, or
 * f = -rho/eps when use_rho != 0. */
int sm_quad_charge_rhs(sm_quad *q, double charge, double eps, int use_rho);

/* Full multigrid (restrict f, exact level-0 solve, per level prolongation
 * and one V-cycle), then V-cycles until max_leaf |f - L phi| /
 * max_leaf |f - L 0| <= tol or max_cycles cycles.  Out (may be NULL):
 * cycles, final relative residual.  Synchronises.  SM_ENOCONV if tol was
 * not reached. */
int sm_quad_fmg(sm_quad *q, double tol, int max_cycles, int *cycles, double *rel);
/* V-cycles from the current potential, same stopping rule. */
int sm_quad_solve(sm_quad *q, double tol, int max_cycles, int *cycles, double *rel);

/* n V-cycles from the current potential with no residual evaluation
 * (enqueue only; for timing and fixed schedules). */
int sm_quad_vcycles(sm_quad *q, int n);

/* |E| on leaf cells from the current potential (zero on refined boxes). */
int sm_quad_compute_field(sm_quad *q);
/* Time-step limits of Sec. 2.4 in two dimensions: 0.9 min(0.5 /
 * max sum|v_d|/dx, 1 / max(sum|v_d|/dx + 4 D/dx^2), eps/(charge mu n_e)).
 * Needs a table and the field.  Synchronises. */
int sm_quad_dt_limit(sm_quad *q, double charge, double eps, double *dt);
/* One forward Euler stage n += dt F(n) on the current field (Eq. 2-3). */
int sm_quad_fluid_stage(sm_quad *q, double dt);
/* One Heun step (Sec. 2.4): Euler stage, solve, field, Euler stage,
 * average, solve, field; dt_next from the second stage's field.  cycles
 * (host int[2], may be NULL): V-cycles of the two solves.  Synchronises. */
int sm_quad_advance(sm_quad *q, double dt, double charge, double eps, double tol, int max_cycles,
                    double *dt_next, int *cycles);

/* Refinement criterion (Sec. 2.5, Eq. 8) per leaf box from the stored |E|,
 * the rules of sm_refine_flags on the quadtree: +1 where a cell has
 * alpha(c1 |E|) dx >= c0 c1 (alpha from the table, each operation rounded
 * on its own) or a needing cell of a same-level leaf neighbour (one of the
 * 8) lies within `buffer` cells (Chebyshev distance), below the maximum
 * level; -1 for a leaf above the base grid whose cells all have
 * alpha(c1 |E|) dx < c0_deref c1 and dx < dx_deref; 0 otherwise.
 * flags: host int8 [n_boxes] out.  0 <= buffer <= 8.  Synchronises.
 * Errors: SM_EINVAL, SM_ESTATE (no table). */
int sm_quad_refine_flags(sm_quad *q, double c0, double c1, double c0_deref, double dx_deref, int buffer,
                         int8_t *flags);
/* Regrid with per-box flags (host int8 [n_boxes], leaves only; the layout
 * of sm_quad_refine_flags), the rules of sm_regrid: densities restricted
 * first; a +1 leaf below the maximum level gets 4 children when all 8
 * neighbour positions of its level are covered or outside the domain (else
 * dropped); a box whose 4 children are all -1 leaves loses them unless a
 * non-sibling neighbour of a child has children or is refined in the same
 * call.  Boxes are renumbered in (level, Morton) order; kept boxes keep phi,
 * f, n_e, n_i, |E| and rho; new children get phi, n_e, n_i by the
 * prolongation (2c + c_x + c_y)/4 of their parent's cells (wall ghosts for
 * phi; mirrors and the 2c limit for densities), the rest zero.  Out (may be
 * NULL): refined boxes, derefined boxes, dropped requests.  The decisions,
 * the new box set and its tables are formed on the device (scratch in the
 * arena's per-call work fields); the host reads the counts once and then
 * the new tables for sm_quad_get_tables and sm_quad_refine_flags.
 * Synchronises.  Errors: SM_EINVAL, SM_ENOMEM (past max_boxes; the mesh is
 * unchanged), SM_ESTATE. */
int sm_quad_regrid(sm_quad *q, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped);

/* on != 0 (the default): each V-cycle runs as a CUDA graph, captured per
 * top level on first use and dropped when the mesh or the arena changes;
 * 0: the same launches are issued from the host.  Results are identical. */
int sm_quad_set_graphs(sm_quad *q, int on);
/* on != 0 (the default): the V-cycle kernels are launched with programmatic
 * dependent launch (each loads its box's tables while its predecessor
 * drains, and waits for it before reading a field); 0: plain stream
 * order.  Results are identical. */
int sm_quad_set_pdl(sm_quad *q, int on);
/* Kernel launches issued by this context so far (a graph counts its
 * kernels). */
int sm_quad_launch_count(const sm_quad *q, long long *n);
/* One-line reason of the last error of this context ("" if none). */
const char *sm_quad_last_error(const sm_quad *q);

#ifdef __cplusplus
}
#endif
#endif
