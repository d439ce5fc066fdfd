/* sm_streamer.h -- C ABI of the GB300 (sm_103a) library for the per-time-step
 * path of the streamer fluid model of arXiv:1708.08434 (Afivo-streamer):
 *
 *   - octree of fixed 8^3-cell boxes with proper nesting   (Sec. 2.1.1)
 *   - geometric multigrid for Poisson's equation, FAS V-cycle and FMG with
 *     red-black Gauss-Seidel smoothing                      (Sec. 2.1.2, Eq. 1, 5)
 *   - cell-centred field from the potential                 (Sec. 2.3)
 *   - drift-diffusion-reaction step with Koren-limited upwind fluxes,
 *     transport-coefficient lookup table, refinement-boundary fluxes and
 *     Heun time stepping with CFL/diffusion/relaxation limits
 *                                                            (Sec. 2.2-2.4, Eq. 2-3, 6-7)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns an sm_status; SM_OK is 0, errors are negative.  After
 *   an error, sm_last_error() gives a one-line reason.
 * - Work is ordered on the CUDA stream given to sm_create (a cudaStream_t
 *   passed as void*; NULL = the legacy default stream).  Calls that return a
 *   scalar to the host (residuals, counts, time steps) synchronise that
 *   stream before returning; the others only enqueue work.
 * - Device memory: the caller allocates one device buffer ("arena") of the
 *   size reported by sm_arena_size and hands it over with sm_bind_arena.  The
 *   library carves every table and field out of it, never frees it and
 *   never allocates device memory itself.  The arena must outlive the
 *   context.
 * - Field layout in the arena: each variable is an array of
 *   [max_boxes][512] doubles; box b is the b-th entry of the box tables
 *   (boxes sorted by level, then Morton key); inside a box cell (i,j,k),
 *   0 <= i,j,k < 8, sits at i + 8 j + 64 k.
 * - Faces are numbered 0..5 = -x,+x,-y,+y,-z,+z everywhere.
 * - There is no CPU fallback: without a usable CUDA device sm_create returns
 *   SM_ECUDA.
 */
#ifndef SM_STREAMER_H
#define SM_STREAMER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SM_BOX 8            /* cells per box side (Sec. 2.1.1, N = 8) */
#define SM_MAX_LEVELS 24    /* levels 0 .. SM_MAX_LEVELS-1 */

typedef struct sm_ctx sm_ctx;   /* opaque, owned by the library */

typedef enum {
  SM_OK = 0,
  SM_EINVAL = -1,     /* bad argument or unsupported domain */
  SM_ENOMEM = -2,     /* arena too small / box capacity exceeded */
  SM_ECUDA = -3,      /* a CUDA runtime call failed */
  SM_ENOCONV = -4,    /* tolerance not reached within max_cycles */
  SM_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
  SM_ESTATE = -6      /* call out of order (e.g. no arena, no table) or a
                         device-side consistency check failed */
} sm_status;

typedef enum { SM_FP64 = 0, SM_MIXED = 1 } sm_precision;

typedef enum {
  SM_PHI = 0,   /* electric potential phi                       */
  SM_RHS = 1,   /* right-hand side f of L phi = f (Eq. 5)       */
  SM_RES = 2,   /* scratch: residual / correction               */
  SM_NE = 3,    /* electron density n_e (current)               */
  SM_NI = 4,    /* positive-ion density n_i (current)           */
  SM_EMAG = 5,  /* cell-centred field strength |E| (leaf boxes) */
  SM_RHO = 6    /* external charge density rho (optional)       */
} sm_var;

/* Domain [origin, origin + length]^3 on a base grid of nb^3 boxes (nb a
 * power of two, so levels 0 .. log2(nb) are uniform multigrid levels with
 * 2^l boxes per side), refined up to max_level levels above the base.
 * bc_type: 0 = Neumann zero, 1 = Dirichlet with value bc_val (potential).
 * Densities always use Neumann zero walls (Sec. 3.1).  At least one face
 * must be Dirichlet. */
typedef struct {
  double length;
  double origin[3];
  int nb;
  int max_level;
  int bc_type[6];
  double bc_val[6];
} sm_domain;

typedef struct {
  int max_boxes;   /* capacity of box tables and fields */
  int nu1, nu2;    /* pre/post smoothing sweeps per level (2, 2) */
  int precision;   /* sm_precision */
} sm_config;

/* Box tables (device pointers, borrowed: valid until the next
 * sm_refine_level).  -1 in child[] = no children; nbr[b*26+d] for
 * d = (dx+1) + 3(dy+1) + 9(dz+1) with the centre skipped (d > 13 shifted
 * down by one): box index, -1 = outside the domain, -2 = no box of this
 * level there (the parent's neighbour covers it).  level_offset[l] ..
 * level_offset[l+1]-1 are the boxes of level l (host array). */
typedef struct {
  int n_boxes;
  int n_levels;
  int n_leaves;
  int level_offset[SM_MAX_LEVELS + 1];
  const int32_t *level;    /* [n_boxes]    */
  const int32_t *ijk;      /* [n_boxes][3] box coordinates at its level */
  const uint64_t *morton;  /* [n_boxes]    x -> bit 0, y -> bit 1, z -> bit 2 */
  const int32_t *parent;   /* [n_boxes]    -1 on level 0 */
  const int32_t *child;    /* [n_boxes][8] child c = cx + 2 cy + 4 cz */
  const int32_t *nbr;      /* [n_boxes][26] */
  const int32_t *leaf;     /* [n_leaves]   leaf box indices, table order */
} sm_tables;

/* ---- lifetime and memory ------------------------------------------------ */

/* Create a context on the current CUDA device.  cfg and dom are copied.
 * stream: cudaStream_t (as void*) all work is ordered on.
 * Errors: SM_EINVAL (nb not a power of two, too many levels, no Dirichlet
 * face, nu < 1, max_boxes too small for the uniform levels), SM_ECUDA. */
int sm_create(sm_ctx **out, const sm_config *cfg, const sm_domain *dom, void *stream);

/* Destroy the context (does not free the arena). NULL is accepted. */
int sm_destroy(sm_ctx *ctx);

/* Bytes of device memory the context needs (depends on cfg.max_boxes). */
int sm_arena_size(const sm_ctx *ctx, size_t *bytes);

/* Hand over a device buffer of at least sm_arena_size bytes, 256-byte
 * aligned.  Zero-fills it on the stream.  Errors: SM_EINVAL, SM_ENOMEM. */
int sm_bind_arena(sm_ctx *ctx, void *dev_ptr, size_t bytes);

/* ---- octree (Sec. 2.1.1) ------------------------------------------------ */

/* Build the uniform levels 0 .. log2(nb) (the base grid and the coarse
 * multigrid levels below it) and their tables on the device.
 * Out: *n_boxes.  Errors: SM_ESTATE (no arena), SM_ENOMEM. */
int sm_build_octree(sm_ctx *ctx, int *n_boxes);

/* Refine boxes of `level`, which must be the finest existing level and
 * below the domain's maximum.  flags: HOST array, one int8 per box of the
 * level in table order; > 0 requests refinement.  Proper nesting: a request
 * is dropped when one of the box's 26 neighbour positions at its level
 * holds no box (inside the domain).  Children are appended as level+1 in
 * Morton order and all tables (neighbours, leaf list) are rebuilt on the
 * device.  Out: *n_new boxes created, *n_dropped requests dropped (either
 * may be NULL).  Errors: SM_EINVAL, SM_ESTATE, SM_ENOMEM (capacity). */
int sm_refine_level(sm_ctx *ctx, int level, const int8_t *flags, int *n_new, int *n_dropped);

/* Borrowed device pointers to the tables (see sm_tables). */
int sm_get_tables(const sm_ctx *ctx, sm_tables *out);

/* ---- fields -------------------------------------------------------------- */

/* Device pointer of a variable's [max_boxes][512] double array (borrowed;
 * SM_NE/SM_NI move between buffers in sm_advance_fluid). */
int sm_var_ptr(const sm_ctx *ctx, int var, void **dev_ptr);
/* The same pointer with its layout: *ld = 512 doubles per box (cell
 * i + 8j + 64k of box b at b * ld + cell), *n_boxes = boxes in use (either
 * may be NULL).  Errors: SM_EINVAL (unknown var, no arena). */
int sm_var_layout(const sm_ctx *ctx, int var, void **dev_ptr, int *ld, int *n_boxes);

/* Copy boxes [0, n_boxes) of a variable from / to HOST memory (pinned
 * memory gives asynchronous uploads; sm_download synchronises the stream).
 * Errors: SM_EINVAL (var, n_boxes > current box count). */
int sm_upload(sm_ctx *ctx, int var, const double *host, int n_boxes);
int sm_download(sm_ctx *ctx, int var, double *host, int n_boxes);

/* Transport-coefficient table (Sec. 2.3): HOST arrays of n samples of the
 * mobility, diffusion coefficient and effective ionization coefficient at
 * E_k = k e_max/(n-1); looked up by linear interpolation, clamped at the
 * ends.  2 <= n <= 4096. */
int sm_set_table(sm_ctx *ctx, int n, double e_max, const double *mu,
                 const double *diff, const double *alpha);

/* Right-hand side of Eq. 5 on every leaf cell:
 * f = -q (n_i - n_e) / eps, or f = -rho / eps when use_rho != 0. */
int sm_charge_rhs(sm_ctx *ctx, double q, double eps, int use_rho);

/* Refined boxes of n_e and n_i get the average of their 8 children,
 * finest level first (the 8-child restriction of the multigrid hierarchy,
 * Sec. 2.1.2, applied to the densities). */
int sm_restrict_densities(sm_ctx *ctx);

/* Coarse-to-fine interpolation values at refinement boundaries of `level`
 * for variable var (SM_PHI): for each ghost cell of a face with no box of
 * the same level, phihat = c/2 + c_t1/4 + c_t2/4 from the coarse cell c
 * containing the ghost and its two tangential neighbours on the ghost's
 * side; the ghost value is then phi_f/3 + 2 phihat/3 (Sec. 2.1.1). */
int sm_fill_ghosts(sm_ctx *ctx, int var, int level);
/* The same for every level in [level_lo, level_hi] (each from the one
 * below).  Errors: SM_EINVAL (var other than SM_PHI, empty or bad range). */
int sm_fill_ghosts_range(sm_ctx *ctx, int var, int level_lo, int level_hi);
/* The stored interpolation values phihat of boxes [0, n_boxes) into HOST
 * memory, [n_boxes][6 faces][64] (face f = 2 axis + side; face cell
 * u + 8 w with u along axis (a+1)%3 and w along (a+2)%3 of the face axis
 * a; entries of faces that are not refinement faces are unspecified).
 * Synchronises.  Errors: SM_EINVAL. */
int sm_get_ghosts(sm_ctx *ctx, int var, double *host, int n_boxes);

/* ---- multigrid (Sec. 2.1.2) ---------------------------------------------- */

/* n_cycles FAS V(nu1,nu2) cycles (Sec. 2.1.2) on the full hierarchy
 * starting from the current potential.  Out: relative residual max_leaf|f - L phi| /
 * max_leaf|f - L 0| after the last cycle (may be NULL). */
int sm_mg_vcycle(sm_ctx *ctx, int n_cycles, double *rel_res);

/* V-cycles from the current potential (warm start, Sec. 2.1.2) until the
 * relative residual is <= tol (at least one cycle).  Errors: SM_ENOCONV
 * when max_cycles is reached (the potential is still updated). */
int sm_mg_solve(sm_ctx *ctx, double tol, int max_cycles, int *cycles, double *rel_res);

/* Full multigrid from scratch (Sec. 2.1.2, the initial potential of a
 * run: restrict f, exact level-0 solve, prolong and one V-cycle per
 * level), then V-cycles to tol.  *cycles counts the
 * top-level V-cycles including the last FMG one. */
int sm_mg_fmg(sm_ctx *ctx, double tol, int max_cycles, int *cycles, double *rel_res);

/* ---- refinement criterion and regridding (Sec. 2.5, Eq. 8) -------------- */

/* Per-box flags from the stored |E| of the leaf cells (call after
 * sm_compute_field).  Eq. 8 asks dx < c0 c1 / alpha(c1 |E|) of every cell,
 * alpha from the coefficient table (linear interpolation, every operation
 * rounded separately); a cell needs refinement where
 * alpha(c1 |E|) dx >= c0 c1.  A leaf box gets +1 when one of its cells
 * needs refinement, or a cell of a same-level leaf neighbour within
 * `buffer` cells of it (Chebyshev distance) does, and its level is below
 * the maximum; -1 (derefinable) when nothing marks it, every cell meets
 * alpha(c1 |E|) dx < c0_deref c1, dx < dx_deref and it lies above the base
 * grid; every other box 0.  The paper uses c0 = 1, c1 = 1.2, a buffer of 3
 * cells, c0_deref = 1/8 and dx_deref = 30 um.
 *   flags: HOST int8 [n_boxes] out, table order.  Synchronises.
 * Errors: SM_EINVAL (buffer outside 0..8), SM_ESTATE (no octree, no table). */
int sm_refine_flags(sm_ctx *ctx, double c0, double c1, double c0_deref, double dx_deref, int buffer,
                    int8_t *flags);

/* Regrid with per-box flags (HOST int8 [n_boxes], the layout of
 * sm_refine_flags; only leaves and their parents are read; NULL: the flags
 * the last sm_refine_flags call left on the device).  Refinement:
 * a leaf flagged > 0 below the maximum level gets 8 children when all 26
 * neighbour positions of its level hold a box or lie outside the domain;
 * other requests are dropped.  Derefinement: a box whose 8 children are
 * leaves flagged < 0 loses them unless a non-sibling neighbour of a child
 * has children or is refined in the same call.  Densities are restricted
 * first; boxes are renumbered in (level, Morton) order; potential,
 * right-hand side, |E|, rho and the current densities move with their
 * boxes; new boxes get the potential and densities by the linear
 * prolongation (c + c_sx + c_sy + c_sz)/4 of the parent's cells (densities
 * limited to 2c, mirror ghosts at walls), other variables zero.  Tables,
 * device pointers of sm_get_tables and captured solves are replaced; the
 * SM_RES array is used as scratch.  The decisions, the new numbering and
 * the tables are formed on the device (scans and binary searches over the
 * Morton-sorted levels).  Out (may be NULL): refined boxes, derefined
 * boxes, dropped requests.  Synchronises.  Errors: SM_ESTATE (no octree),
 * SM_ENOMEM (max_boxes). */
int sm_regrid(sm_ctx *ctx, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped);
/* sm_regrid with the new box count as its only output. */
int sm_refine(sm_ctx *ctx, const int8_t *flags, int *n_boxes);

/* ---- field and fluid step (Sec. 2.3, 2.4) --------------------------------- */

/* |E| on every leaf cell (Sec. 2.3): face fields E = (phi_i - phi_{i+1})/dx,
 * cell components = mean of the two faces, |E| = Euclidean norm. */
int sm_compute_field(sm_ctx *ctx);

/* Next time step (Sec. 2.4) from the current field and n_e: 0.9 x min of
 * the CFL 0.5 limit, the advection+diffusion limit and the dielectric
 * relaxation time eps/(q mu n_e).  Synchronises. */
int sm_dt_limit(sm_ctx *ctx, double q, double eps, double *dt);

/* One forward-Euler stage n <- n + dt F(n) with the current field (Sec.
 * 2.2-2.3, Eq. 2-3 with the fluxes of Eq. 6-7; for tests); densities of
 * refined boxes are restricted afterwards. */
int sm_fluid_stage(sm_ctx *ctx, double dt);

/* One explicit trapezoidal (Heun) step over dt (Sec. 2.4): stage 1, charge
 * rhs, V-cycles to tol, field; stage 2 averaged with the stored densities,
 * charge rhs, V-cycles to tol, field.  Out: *dt_next from the limits
 * evaluated at stage 2, cycles[0..1] V-cycles of the two solves (either may
 * be NULL).  Errors: SM_ENOCONV (a solve did not reach tol), SM_ESTATE (no
 * table). */
int sm_advance_fluid(sm_ctx *ctx, double dt, double q, double eps, double tol,
                     int max_cycles, double *dt_next, int *cycles);
/* The same with its constants in one struct. */
typedef struct {
  double q;        /* elementary charge */
  double eps;      /* permittivity */
  double tol;      /* relative residual of the two solves */
  int max_cycles;  /* V-cycle limit of each solve */
} sm_fluid_coeffs;
int sm_advance_fluid_coeffs(sm_ctx *ctx, double dt, const sm_fluid_coeffs *c, double *dt_next, int *cycles);

/* ---- diagnostics ----------------------------------------------------------- */

/* Average device time of one launch of a kernel class, timed on the context
 * stream between two CUDA events after one untimed warm-up.
 *   class 0 (red-black smoother): one CUDA graph of `reps` repetitions of
 *     both colour passes over every level 1..top, the launch mix of a
 *     V-cycle; algorithmic bytes 16 per cell of the level (phi read, f and
 *     phi of the colour), FP64 instructions 3.5 per cell (5 adds, 1 fused
 *     multiply-add and 1 multiply per updated cell).
 *   class 1 (persistent V-cycle, Sec. 2.1.2): `reps` cooperative launches of
 *     the persistent kernel, each one whole FP64 FAS V-cycle; algorithmic
 *     bytes and FP64 instructions per V-cycle from the per-level model:
 *     smoothing 16 B and 3.5 per cell and colour pass; residual with
 *     restriction 18 B and 9 per fine cell; FAS completion 16 B per cell of
 *     the level below plus 16 B and 7 per cell of its refined boxes;
 *     prolongation 18 B and 3 per fine cell; level-0 solve 16 B and 60 per
 *     cell.  Ghost-value arithmetic is not counted.
 *   class 2 (V-cycle as per-level launches): one CUDA graph of `reps` FP64
 *     V-cycles launched level by level; the unit is one V-cycle, bytes and
 *     instructions as for class 1.
 *   class 3 (FP32 V-cycle of the mixed-precision form, mixed contexts only):
 *     one CUDA graph of `reps` FP32 V-cycles on the error equation; bytes
 *     half those of class 1, no FP64 instructions.
 * Out (each may be NULL): microseconds per launch, launches timed,
 * algorithmic bytes and FP64 instructions per launch.  Side effect: the
 * potential receives the extra sweeps or cycles.  Errors: SM_EINVAL for an
 * unknown class, reps < 1 or a single-level octree. */
int sm_kernel_bench(sm_ctx *ctx, int kclass, int reps, double *us_per_launch, long long *launches,
                    double *bytes_per_launch, double *fp64_per_launch);

/* Per-solve metrics log (no paper passage): with a path, every
 * sm_mg_solve and sm_mg_fmg (also those inside sm_advance_fluid) appends one
 * JSON line to that file (opened for appending; path NULL or "" closes it):
 *   seq, call ("fmg" | "solve"), precision ("fp64" | "mixed"), path
 *   ("graph" | "host" | "persistent"), boxes, levels, leaf_cells, tol,
 *   status (the call's return code), cycles, rel (final relative residual),
 *   residual_history (relative residual after each cycle, the first 64;
 *   an FMG ladder is cycle 1; empty for the persistent kernel), ms (CUDA
 *   events around the call, retries of a widened fixed-point scale
 *   included), vcycle_bytes (the per-level algorithmic model of
 *   sm_kernel_bench class 2, FP32 arrays for the mixed form's cycles being
 *   counted as FP64), bytes (vcycle_bytes x cycles), gbs (bytes / ms),
 *   hbm_frac (gbs / hbm_peak_gbs, null when hbm_peak_gbs <= 0).
 * Logging synchronises the stream after each solve (the solves do anyway).
 * Errors: SM_EINVAL (file cannot be opened), SM_ECUDA. */
int sm_set_metrics_log(sm_ctx *ctx, const char *path, double hbm_peak_gbs);

/* Levels of at least min_boxes boxes (default 2048; 0: every level) run
 * the fixed-point smoother, residual-restriction and prolongation kernels
 * with one thread per x row of a box (16-byte row loads, fewer
 * instructions per cell); smaller levels run the kernels with one
 * 128-thread group per box (more warps per box for latency).  Both give bit-identical results; the
 * choice is performance only.  Errors: SM_EINVAL for min_boxes < 0. */
int sm_set_row_kernels(sm_ctx *ctx, int min_boxes);

/* Solves run as CUDA graphs (captured on first use per octree, with the
 * cycle loop and its stopping test on the device) when enabled (default),
 * or as individually launched kernels with a host loop when disabled.
 * Both paths launch the same kernels in the same order. */
int sm_set_graphs(sm_ctx *ctx, int enable);

/* V-cycles run as one persistent cooperative launch when enabled (default
 * off: on GB300 a software grid barrier between phases costs more than a
 * kernel boundary inside a CUDA graph):
 * every block stays resident, each level operation is one phase over all
 * boxes of the level with a grid barrier after it, and the FP64 solves keep
 * their residual test and cycle loop inside the same launch.  Disabled, the
 * same per-box operations run as one launch per level and phase.  Both give
 * bit-identical results.  A barrier wait that runs out (about a second)
 * ends the launch and the solve returns SM_ETIMEOUT.  Captured graphs are
 * dropped on a change. */
int sm_set_persistent(sm_ctx *ctx, int enable);

/* Self-test of the bounded grid-barrier wait of the persistent kernel: one
 * launch whose barriers wait for one block more than the grid holds, so
 * every block's wait runs out (about a second), sets the error flag and
 * returns.  Expected result SM_ETIMEOUT; the flag is cleared afterwards and
 * the context stays usable (the potential may have received part of a
 * V-cycle).  Errors: SM_ESTATE (no octree or a pending device error),
 * SM_EINVAL (single-level octree). */
int sm_persist_barrier_selftest(sm_ctx *ctx);

/* Kernels of the multigrid solve are launched with programmatic dependent
 * launch when enabled (default): a kernel may be scheduled while its
 * predecessor on the stream drains, and waits for that predecessor's
 * completion and memory before its first access, so results are identical
 * with the switch on or off.  Captured graphs are dropped on a change. */
int sm_set_pdl(sm_ctx *ctx, int enable);

/* Number of kernels this context has launched since it was created
 * (diagnostics: lets a caller count device launches inside a region). */
int sm_launch_count(const sm_ctx *ctx, long long *n);

/* ---- batched form: many independent uniform solves ------------------------ */

/* Build form (not in the paper): n_solves independent Poisson problems
 * L phi = f with the 7-point operator and ghost rules of the octree solve,
 * each on a uniform grid of cells_per_side[s]^3 cells covering a cube of
 * side `length`, all with the same boundary types/values (bc_type, bc_val
 * as in sm_domain).  Each grid is coarsened by halving its side while it is
 * even and larger than 8; the coarsest side must be <= 16 (SM_EINVAL
 * otherwise); it is solved exactly in FP64.  Cycles are FP32
 * correction-scheme V(nu1,nu2) cycles on the error equation inside a
 * per-solve FP64 defect-correction loop; every level of all solves is one
 * grid-stride launch per phase over a work list (32x16-cell z-marching
 * columns for a whole red-black sweep, the prolongation and the FP64
 * residual; the same columns or small 3-D tiles for the restriction, as
 * the schedule below chooses); the exact coarse solves of each level run
 * on a stream of their own, forked from the cycle and joined before the
 * prolongation from that level.  A batched solve is one CUDA graph whose
 * loop runs on the device; converged solves are masked out.
 * Memory: sm_batch_arena_size / sm_batch_bind_arena as for sm_ctx.
 * Arrays (device, through sm_batch_ptrs): phi and rhs, FP64, the grids of
 * all solves one after another at the returned offsets (each a multiple of
 * 32 elements; the arrays end at offsets[n-1] + N^3 of the last solve),
 * cell (x,y,z) of solve s at offsets[s] + x + N (y + N z). */
typedef struct sm_batch sm_batch;
int sm_batch_create(sm_batch **out, int n_solves, const int *cells_per_side, double length, const int *bc_type,
                    const double *bc_val, int nu1, int nu2, void *stream);
int sm_batch_destroy(sm_batch *b);
int sm_batch_arena_size(const sm_batch *b, size_t *bytes);
int sm_batch_bind_arena(sm_batch *b, void *dev_ptr, size_t bytes);
/* device pointers of phi and rhs and the per-solve offsets (host array of
 * n_solves, may be NULL) */
int sm_batch_ptrs(const sm_batch *b, double **phi, double **rhs, long long *offsets);
/* Solve every problem from its current phi until its relative residual
 * max|f - L phi| / max|f - L 0| <= tol or max_cycles corrections.  Out
 * (host arrays of n_solves, may be NULL): corrections and final relative
 * residual per solve.  SM_ENOCONV if a solve missed tol. Synchronises.
 * A solve whose phi is all +0 on entry reuses the residual of phi = 0
 * (computed for the denominator) as its first residual. */
int sm_batch_solve(sm_batch *b, double tol, int max_cycles, int *cycles, double *rel_res);
/* Autotuner: times `iters` corrections from phi = 0 for every candidate
 * restriction schedule (shape index 0..3: one thread per coarse cell over
 * tiles of 8x8x8, 16x8x4, 32x4x4, 32x8x2 coarse cells; 4: one block per
 * 32x16-cell fine column marching the fine planes, the sweep's columns, on
 * levels with at least four columns per SM, 8x8x8 tiles on the others) and
 * grid size (2, 4, 8, 16, 32 blocks per SM), keeps the fastest; leaves phi = 0.
 * Out: the chosen shape index, blocks per SM and its time in ms.
 * sm_batch_set_schedule sets both directly (SM_EINVAL outside 0..4 and
 * 1..64). */
int sm_batch_tune(sm_batch *b, int iters, int *shape, int *grid_mult, double *best_ms);
int sm_batch_set_schedule(sm_batch *b, int shape, int grid_mult);
/* Time one kernel class of the batched cycle over all solves: `reps`
 * back-to-back launches between CUDA events on the batch stream, after one
 * warm-up launch.  kclass: 0 level-0 red-black sweep, 1 FP64 outer
 * residual, 2 level-0 prolongation, 3 level-0 -> 1 restriction in the
 * current schedule (fine columns under schedule 4 when level 0 has at
 * least four columns per SM, else coarse-cell tiles).  Out (may be NULL):
 * microseconds per launch, algorithmic bytes per launch (compulsory
 * traffic: 12, 20, 8.5, 8.5 B per cell of the level) and FP64-pipe
 * operations per launch (2 per cell for class 1: the multiply-add and the
 * int64 -> binary64 conversion of the fixed-point stencil sum; else 0).
 * Overwrites the error arrays and may leave phi changed (class 1 leaves it
 * as it is).  Errors: SM_EINVAL, SM_ESTATE (no arena; no level below the
 * finest). */
int sm_batch_kernel_bench(sm_batch *b, int kclass, int reps, double *us_per_launch, double *bytes_per_launch,
                          double *fp64_per_launch);
/* Solves as one CUDA graph with the loop on the device (default) or as the
 * same launches driven from the host (for profilers that cannot see into
 * conditional graph nodes). */
int sm_batch_set_graphs(sm_batch *b, int enable);
/* total cells (finest grids), deepest level count, kernels launched so far */
int sm_batch_info(const sm_batch *b, long long *cells, int *levels_max, long long *launches);
const char *sm_batch_last_error(const sm_batch *b);

/* ---- learned warm start ---------------------------------------------------- */

/* Build form (not in the paper): a per-box 3D convolutional network
 * predicts the change of the potential of an 8^3 box from its right-hand
 * side and previous potential; it warm-starts the two warm-started solves
 * of sm_advance_fluid, and the multigrid residual judges each prediction.
 *   input: 2 channels on the box and its ghost layer (10^3; positions
 *          outside the box repeat the nearest interior cell): the FP64
 *          residual h^2 (f - L phi) of the plain warm start divided by the
 *          box scale s = max |h^2 (f - L phi)|, and h^2 f divided by its box
 *          maximum; output delta on 8^3; phi += s * delta.  Training target:
 *          (phi_solved - phi_prev)/s clipped to [-8, 8].
 *   layers: conv 3^3 valid 2->16 + ReLU, conv 3^3 same 16->16 + ReLU (BF16
 *          tensor-core GEMM, its data and weight gradients too), conv 3^3
 *          same 16->1.  Weights BF16, operands rounded to BF16, FP32
 *          accumulation, biases FP32; gradients at FP32 accuracy.
 *   parameters (FP32, SM_CNN_PARAMS): W1[16][2][27], b1[16], W2[16][16][27],
 *          b2[16], W3[16][27], b3 with tap t = (dx+1) + 3(dy+1) + 9(dz+1).
 * Samples and inputs are kept in the network's own arena
 * (sm_cnn_arena_size / sm_cnn_bind_arena); max_samples >= 16 training
 * pairs, max_boxes boxes per prediction. */
#define SM_CNN_PARAMS 8241
typedef struct sm_cnn sm_cnn;
int sm_cnn_create(sm_cnn **out, int max_samples, int max_boxes, void *stream);
int sm_cnn_destroy(sm_cnn *c);
int sm_cnn_arena_size(const sm_cnn *c, size_t *bytes);
int sm_cnn_bind_arena(sm_cnn *c, void *dev_ptr, size_t bytes);
/* FP32 parameters from / to HOST memory (n = SM_CNN_PARAMS); setting them
 * resets the Adam moments. */
int sm_cnn_set_params(sm_cnn *c, const float *host, int n);
int sm_cnn_get_params(sm_cnn *c, float *host, int n);
/* Forward pass of n explicit inputs (HOST [n][1000][2] floats, position
 * index x + 10 y + 100 z, rounded to BF16): out HOST [n][512]; acts (HOST,
 * may be NULL) [min(n,16)][4][16][512] = z1, relu'd BF16 a1, z2, a2. */
int sm_cnn_forward(sm_cnn *c, const float *x_host, int n, float *out_host, float *acts_host);
/* Gradient of the mean squared error over n explicit (input, target)
 * pairs (HOST [n][1000][2], [n][512]); grad HOST [SM_CNN_PARAMS].
 * Overwrites recorded samples. */
int sm_cnn_gradient(sm_cnn *c, const float *x_host, const float *t_host, int n, float *grad_host, float *loss);
/* Replace the recorded samples by n explicit (input, target) pairs (HOST
 * [n][1000][2] floats rounded to BF16, [n][512]; 1 <= n <= max_samples) for
 * sm_cnn_train and sm_cnn_kernel_bench.  Errors: SM_EINVAL, SM_ECUDA. */
int sm_cnn_load_samples(sm_cnn *c, const float *x_host, const float *t_host, int n);
/* One Adam step (beta 0.9/0.999, eps 1e-8, bias-corrected) with an explicit
 * gradient (HOST [SM_CNN_PARAMS]). */
int sm_cnn_adam_step(sm_cnn *c, const float *grad_host, float lr);
/* `epochs` passes over the recorded samples in minibatches of `batch`, an
 * Adam step after each; sample order shuffled per epoch from `seed`.  Out:
 * mean loss of the last epoch.  Synchronises. */
int sm_cnn_train(sm_cnn *c, int epochs, int batch, float lr, unsigned long long seed, float *loss);
/* Timing of the network kernels (build form, no paper passage): the mean
 * duration of `reps` launches (CUDA events on the network's stream, after
 * one warm-up) over the first n recorded samples; kind 0: the forward
 * kernel (n <= max_boxes), kind 1: one training gradient pass.  *flops: the
 * model's FLOPs of one launch (16416 per voxel forward, 3x that for a
 * gradient pass); *tensor_flops: those the tensor cores execute per launch,
 * discarded tile rows included (per box: forward 135 MMAs of 128x16x16; a
 * gradient pass adds 405 of 128x16x16 for the data gradient and 288 of
 * 128x48x16 for the weight gradient of layer 2).
 * Overwrites the prediction outputs.  Errors: SM_EINVAL (kind, n, reps),
 * SM_ESTATE (fewer recorded samples than n), SM_ETIMEOUT, SM_ECUDA. */
int sm_cnn_kernel_bench(sm_cnn *c, int kind, int n, int reps, double *us_per_launch, double *flops,
                        double *tensor_flops);
/* Couple the network to a solver's sm_advance_fluid: mode 1 records
 * (input, solved change) pairs of up to per_solve leaf boxes of the two
 * finest levels (every stride-th) per solve; mode 2 predicts a warm start
 * for those boxes before each solve (taper != 0: the prediction is
 * weighted 1/4, 3/4 on the two outer cell layers of each axis) and keeps
 * it only if the relative residual of the predicted start is below accept
 * times that of the plain warm start (else the plain warm start); the
 * solve then iterates to its tolerance either way.  mode 0 detaches. */
int sm_cnn_attach(sm_ctx *ctx, sm_cnn *c, int mode, int per_solve, int stride, int taper, double accept);
/* recorded samples, predictions made and kept, last residuals
 * (last_rel[0] plain start, last_rel[1] predicted start) */
int sm_cnn_stats(const sm_cnn *c, int *n_samples, long long *predictions, long long *kept, double *last_rel);
const char *sm_cnn_last_error(const sm_cnn *c);

/* ---- allocation-free entry point ---------------------------------------- */

/* No counterpart in the paper: a service for callers that cannot allocate
 * device memory -- code running while another component owns all device
 * memory (a caching allocator or pool it must not bypass), code in regions
 * where an allocation is forbidden or would synchronise the device, and
 * embedders that only hand over their own input and output buffers.
 *
 * Solves n_problems independent Poisson problems L phi = f, each on one box
 * of 8^3 cells and side `length`, with the 7-point operator and boundary
 * rules of the multigrid solve (Dirichlet ghost 2g - phi, Neumann ghost
 * phi); this is the same eigenbasis solve as level 0 of sm_mg_fmg.
 *   bc_type: DEVICE int32 [n_problems][6] (faces -x,+x,-y,+y,-z,+z;
 *            0 Neumann zero, 1 Dirichlet); a problem without a Dirichlet
 *            face gets its constant mode set to zero
 *   bc_val:  DEVICE double [n_problems][6] Dirichlet values
 *   f:       DEVICE double [n_problems][512] right-hand side (cell i+8j+64k)
 *   phi:     DEVICE double [n_problems][512] solution (written)
 *   stream:  cudaStream_t as void*; the call only enqueues work.
 * The library allocates nothing: its only scratch (one eigenbasis per
 * problem) is a fixed device array of SM_NOALLOC_MAX_PROBLEMS x 1728 bytes
 * (1.77 MB) that every GPU loading the library holds until exit.  The first
 * call on a device looks up that array's device address (set-up, with the
 * device current); make that first call before any stream capture.  Every
 * later call made outside a capture looks the address up again, so after a
 * device reset (cudaDeviceReset) make one uncaptured call before capturing
 * again.  Each device has its own copy of the array.  All calls on one
 * device share it and each call overwrites the slots of its problems before
 * reading them, so nothing needs clearing, but calls that overlap on the
 * same device (different streams) race on it and must be ordered; calls on
 * different devices are independent.  Device ordinals 0..63 are supported.
 * Errors: SM_ENOMEM if n_problems > SM_NOALLOC_MAX_PROBLEMS (the fixed
 * scratch is too small), SM_EINVAL (n_problems < 0, length <= 0, null
 * pointer, device ordinal above 63), SM_ECUDA (no device, first call of a
 * device inside a stream capture, address lookup or launch failed). */
#define SM_NOALLOC_MAX_PROBLEMS 1024
int sm_box_solve_noalloc(double length, int n_problems, const int32_t *bc_type, const double *bc_val,
                         const double *f, double *phi, void *stream);

/* Throughput of the GPU's FP64 pipe, measured: one launch of 8 resident
 * blocks of 256 threads per SM, each thread running 8 independent chains
 * of `iters` fused multiply-adds x = x*a + b (after a shorter warm-up
 * launch), timed with CUDA events on `stream`.  *fma_per_s receives the
 * fused multiply-adds per second (one FP64-pipe instruction each; 2 flops),
 * *ms_out (optional) the timed launch's duration.  d_scratch: one device
 * word the kernel may write (a sink that keeps the arithmetic from being
 * optimised away); the caller owns it.  No counterpart in the paper: it
 * measures the roof of the FP64-bound fluid kernels (Sec. 2.3 fluxes,
 * Sec. 2.4 time step).  Synchronises the stream.  Errors: SM_EINVAL
 * (iters < 1, null pointers), SM_ECUDA (no device, launch failed). */
int sm_fp64_probe(long long iters, unsigned long long *d_scratch, double *fma_per_s, double *ms_out, void *stream);

/* Check of the library's own FP64 <-> FP32 conversions (not in the paper).
 * The FP64 kernels convert on the 32-bit integer pipe instead of with the
 * hardware conversion instructions, which share the narrow FP64 pipe; this
 * entry point compares both ways against the hardware on n seeded bit
 * patterns (SplitMix64 of seed + i; three quarters of them with exponents
 * at the edges of the FP32 range and fractions at the rounding boundary).
 * It also checks the FP64 -> 64-bit fixed-point map of the batched
 * residual (nearest multiple of 2^(E-1080), ties away from zero) against
 * exact FP64 scaling, for E from the value's exponent to +70.
 *   d_scratch:  DEVICE uint64 [3], overwritten.
 *   mismatches: HOST uint64 [3] out: FP64->FP32, FP32->FP64 and FP64->fixed
 *               patterns whose result differs from the reference (NaN =
 *               NaN).
 * Synchronises the stream.  Errors: SM_EINVAL (n < 0, null pointer),
 * SM_ECUDA. */
int sm_check_conversions(long long n, unsigned long long seed, unsigned long long *d_scratch,
                         unsigned long long *mismatches, void *stream);

/* Human-readable reason of the last error on this context. */
const char *sm_last_error(const sm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SM_STREAMER_H */
