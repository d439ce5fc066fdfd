/* oracle.h -- plain CPU oracle of the octree multigrid Poisson solve and the
 * drift-diffusion-reaction step of arXiv:1708.08434 (Sec. 2.1.1, 2.1.2, 2.3,
 * 2.4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the package smoke check and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Field arrays exchanged through orc_set/orc_get are [n_boxes][512] doubles,
 * box order = table order (level, then Morton key), cell order x fastest.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

typedef struct orc orc;

/* public variable ids */
enum { ORC_PHI = 0, ORC_RHS = 1, ORC_RES = 2, ORC_NE = 3, ORC_NI = 4,
       ORC_EMAG = 5, ORC_RHO = 6 };

orc *orc_create(double length, const double *origin, int nb, int max_level,
                const int *bc_type, const double *bc_val);
void orc_destroy(orc *o);
/* OpenMP threads for the per-box loops (n >= 1; n < 1 only queries).
 * Returns the count in effect; 1 when the library was built without
 * OpenMP.  Results do not depend on it. */
int orc_set_threads(int n);
int orc_n_boxes(const orc *o);
int orc_n_levels(const orc *o);
int orc_level_offset(const orc *o, int level);
int orc_refine_level(orc *o, int level, const int8_t *flags, int *n_dropped);
void orc_get_tables(const orc *o, int32_t *level, int32_t *ijk, uint64_t *morton,
                    int32_t *parent, int32_t *child, int32_t *nbr);
void orc_set(orc *o, int var, const double *src);
void orc_get(const orc *o, int var, double *dst);
void orc_set_table(orc *o, int n, double e_max, const double *mu,
                   const double *diff, const double *alpha);

void orc_charge_rhs(orc *o, double q, double eps, int use_rho);
int orc_fmg(orc *o, double tol, int max_cycles, int nu1, int nu2,
            double *rel, int *cycles);
int orc_vcycles(orc *o, int n, int nu1, int nu2, double *rel);
int orc_solve(orc *o, double tol, int max_cycles, int nu1, int nu2,
              double *rel, int *cycles);
double orc_rel_residual(orc *o);
void orc_composite_residual(orc *o);
void orc_compute_field(orc *o);
double orc_dt_limit(orc *o, double q, double eps);
int orc_advance(orc *o, double dt, double q, double eps, double tol,
                int max_cycles, int nu1, int nu2, double *dt_next,
                int *cycles1, int *cycles2);
void orc_fluid_stage(orc *o, double dt);
double orc_koren(double a, double b);
double orc_lookup(const orc *o, int which, double e);
void orc_coarse_solve(orc *o);
void orc_refine_flags(orc *o, double c0, double c1, double c0_deref, double dx_deref,
                      int buffer, int8_t *flags);
int orc_regrid(orc *o, const int8_t *flags, int *n_refined, int *n_derefined,
               int *n_dropped);
#endif
