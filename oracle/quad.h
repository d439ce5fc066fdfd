/* quad.h -- plain CPU oracle of the 2-D and axisymmetric variants of the
 * octree path of arXiv:1708.08434 (Sec. 1: "2D, axisymmetric and 3D
 * simulations are supported"; Sec. 2.1.1 quadtree grids): the multigrid
 * Poisson solve on a quadtree of 8^2-cell boxes (Sec. 2.1.2) and the explicit
 * drift-diffusion-reaction step (Sec. 2.2-2.4), in Cartesian (x, y) or
 * cylindrical (r, z) coordinates.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the package smoke check and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Field arrays exchanged through q2_set/q2_get are [n_boxes][64] doubles,
 * box order = table order (level, then Morton key), cell order x fastest.
 * Axisymmetric: x is the radius r (the axis r = 0 is face -x, where no
 * boundary condition applies) and y is the axial coordinate z.
 */
#ifndef ORACLE_QUAD_H
#define ORACLE_QUAD_H
#include <stdint.h>

typedef struct q2 q2;

enum { Q2_PHI = 0, Q2_RHS = 1, Q2_RES = 2, Q2_NE = 3, Q2_NI = 4, Q2_EMAG = 5, Q2_RHO = 6 };
enum { Q2_CARTESIAN = 0, Q2_AXISYMMETRIC = 1 };

/* bc per face -x,+x,-y,+y: type 0 Neumann zero, 1 Dirichlet with value */
q2 *q2_create(double length, const double *origin, int nb, int max_level, int geom,
              const int *bc_type, const double *bc_val);
void q2_destroy(q2 *o);
/* OpenMP threads for the per-box loops (n < 1 only queries); results do
 * not depend on it */
int q2_set_threads(int n);
int q2_n_boxes(const q2 *o);
int q2_n_levels(const q2 *o);
int q2_level_offset(const q2 *o, int level);
int q2_refine_level(q2 *o, int level, const int8_t *flags, int *n_dropped);
void q2_get_tables(const q2 *o, int32_t *level, int32_t *ij, uint64_t *morton, int32_t *parent,
                   int32_t *child, int32_t *nbr);
void q2_set(q2 *o, int var, const double *src);
void q2_get(const q2 *o, int var, double *dst);
void q2_set_table(q2 *o, int n, double e_max, const double *mu, const double *diff,
                  const double *alpha);
double q2_lookup(const q2 *o, int which, double e);
/* psi(a/b) b of the Koren limiter (Eq. 7), division-free */
double q2_koren(double a, double b);
void q2_charge_rhs(q2 *o, double q, double eps, int use_rho);
int q2_fmg(q2 *o, double tol, int max_cycles, int nu1, int nu2, double *rel, int *cycles);
int q2_vcycles(q2 *o, int n, int nu1, int nu2, double *rel);
int q2_solve(q2 *o, double tol, int max_cycles, int nu1, int nu2, double *rel, int *cycles);
double q2_rel_residual(q2 *o);
void q2_composite_residual(q2 *o);
void q2_restrict_all(q2 *o, int var);
void q2_compute_field(q2 *o);
double q2_dt_limit(q2 *o, double q, double eps);
void q2_fluid_stage(q2 *o, double dt);
int q2_advance(q2 *o, double dt, double q, double eps, double tol, int max_cycles, int nu1,
               int nu2, double *dt_next, int *cycles1, int *cycles2);
void q2_coarse_solve(q2 *o);
void q2_refine_flags(q2 *o, double c0, double c1, double c0_deref, double dx_deref, int buffer,
                     int8_t *flags);
int q2_regrid(q2 *o, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped);
#endif
