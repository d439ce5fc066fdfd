/* oracle.c -- plain, slow, obviously correct CPU oracle for the per-time-step
 * path of arXiv:1708.08434 (Afivo-streamer): the geometric multigrid Poisson
 * solve on an octree of 8^3-cell boxes (Sec. 2.1.1-2.1.2, Eq. 1 and 5) and
 * the explicit drift-diffusion-reaction step (Sec. 2.2-2.4, Eq. 2-3, 6-7),
 * and the refinement criterion with regridding (Sec. 2.5, Eq. 8).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, the smoke check and the
 * CPU-baseline leg of bench.py.  The CUDA library never calls it and shares
 * nothing with it.
 *
 * Data structure (deliberately unlike the GPU one): every box stores its
 * variables with two ghost layers (12^3 doubles); ghost layers are filled
 * explicitly before each stencil sweep, and coarse values needed at
 * refinement boundaries are found by global cell coordinates.
 *
 * Where the paper leaves a detail open, the reading implemented here is the
 * one listed in the design notes (operator, ghost rules, restriction,
 * prolongation, cycle order, stopping rule, limiter form, flux sign, table
 * lookup, refinement-boundary fluxes, time-step limits).
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* OpenMP over the boxes of one pass (Sec. 2.1.3: with one ghost layer per
 * box, the boxes of a pass are independent).  Each box writes only its own
 * cells and ghosts, and the only reductions are maxima, so every result is
 * bit-identical for any thread count. */
#define BOXES_PAR _Pragma("omp parallel for schedule(static)")

#define NC 8                 /* cells per box side (Sec. 2.1.1, N = 8) */
#define GH 2                 /* ghost layers stored */
#define SS (NC + 2 * GH)     /* 12 */
#define BS (SS * SS * SS)    /* doubles per stored box */
#define MAXL 30
#define IX(i, j, k) ((((k) + GH) * SS + ((j) + GH)) * SS + ((i) + GH))

enum { V_PHI, V_RHS, V_RES, V_OLD, V_NE, V_NI, V_EMAG, V_RHO, V_NE0, V_NI0,
       V_NE1, V_NI1, V_TMP, NVAR };

struct orc {
  double len, org[3];
  int nb, lbase, lmax;
  int bct[6];
  double bcv[6];
  int nlev, nbox, cap;
  int *lev, *ijk, *par, *chl, *nbr;
  uint64_t *mort;
  int off[MAXL + 2];
  double *v[NVAR];
  double *lu;
  int *piv;
  double *flux; /* [box][3][9][8][8] */
  int tab_n;
  double tab_emax, *tab[3];
};

static const int pub2var[7] = {V_PHI, V_RHS, V_RES, V_NE, V_NI, V_EMAG, V_RHO};

static void die(const char *msg) {
  fprintf(stderr, "oracle: %s\n", msg);
  abort();
}

/* ---------------------------------------------------------------------- */
/* octree tables (Sec. 2.1.1)                                              */
/* ---------------------------------------------------------------------- */

static uint64_t morton(int i, int j, int k) {
  uint64_t key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= (uint64_t)((i >> b) & 1) << (3 * b);
    key |= (uint64_t)((j >> b) & 1) << (3 * b + 1);
    key |= (uint64_t)((k >> b) & 1) << (3 * b + 2);
  }
  return key;
}

static void unmorton(uint64_t key, int *i, int *j, int *k) {
  *i = *j = *k = 0;
  for (int b = 0; b < 21; ++b) {
    *i |= (int)((key >> (3 * b)) & 1) << b;
    *j |= (int)((key >> (3 * b + 1)) & 1) << b;
    *k |= (int)((key >> (3 * b + 2)) & 1) << b;
  }
}

/* index of neighbour direction (dx,dy,dz) in the 26-entry list */
static int dir26(int dx, int dy, int dz) {
  int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
  return d < 13 ? d : d - 1;
}

/* face f = 0..5 is -x,+x,-y,+y,-z,+z */
static int face_axis(int f) { return f / 2; }
static int face_side(int f) { return f & 1; }
static int face26(int f) {
  int d[3] = {0, 0, 0};
  d[face_axis(f)] = face_side(f) ? 1 : -1;
  return dir26(d[0], d[1], d[2]);
}

/* box at level l with box coordinates (i,j,k): index, -1 outside the
 * domain, -2 inside the domain but no box of that level there */
static int find_box(const orc *o, int l, int i, int j, int k) {
  int n = 1 << l;
  if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return -1;
  if (l >= o->nlev) return -2;
  uint64_t key = morton(i, j, k);
  int lo = o->off[l], hi = o->off[l + 1] - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (o->mort[mid] == key) return mid;
    if (o->mort[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return -2;
}

static void grow(orc *o, int need) {
  if (need <= o->cap) return;
  int cap = o->cap ? o->cap : 64;
  while (cap < need) cap *= 2;
  o->lev = realloc(o->lev, sizeof(int) * cap);
  o->ijk = realloc(o->ijk, sizeof(int) * 3 * cap);
  o->par = realloc(o->par, sizeof(int) * cap);
  o->chl = realloc(o->chl, sizeof(int) * 8 * cap);
  o->nbr = realloc(o->nbr, sizeof(int) * 26 * cap);
  o->mort = realloc(o->mort, sizeof(uint64_t) * cap);
  for (int v = 0; v < NVAR; ++v) {
    o->v[v] = realloc(o->v[v], sizeof(double) * BS * (size_t)cap);
    memset(o->v[v] + (size_t)BS * o->cap, 0, sizeof(double) * BS * (size_t)(cap - o->cap));
  }
  o->flux = realloc(o->flux, sizeof(double) * 3 * 9 * 64 * (size_t)cap);
  o->cap = cap;
}

static int add_box(orc *o, int l, int i, int j, int k, int parent) {
  grow(o, o->nbox + 1);
  int b = o->nbox++;
  o->lev[b] = l;
  o->ijk[3 * b] = i; o->ijk[3 * b + 1] = j; o->ijk[3 * b + 2] = k;
  o->mort[b] = morton(i, j, k);
  o->par[b] = parent;
  for (int c = 0; c < 8; ++c) o->chl[8 * b + c] = -1;
  return b;
}

static void set_neighbours(orc *o, int l) {
  for (int b = o->off[l]; b < o->off[l + 1]; ++b)
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          o->nbr[26 * b + dir26(dx, dy, dz)] =
              find_box(o, l, o->ijk[3 * b] + dx, o->ijk[3 * b + 1] + dy, o->ijk[3 * b + 2] + dz);
        }
}

orc *orc_create(double length, const double *origin, int nb, int max_level,
                const int *bc_type, const double *bc_val) {
  int lb = 0;
  while ((1 << lb) < nb) ++lb;
  if ((1 << lb) != nb || lb + max_level > MAXL - 1) return NULL;
  orc *o = calloc(1, sizeof(orc));
  o->len = length;
  for (int d = 0; d < 3; ++d) o->org[d] = origin ? origin[d] : 0.0;
  o->nb = nb; o->lbase = lb; o->lmax = lb + max_level;
  for (int f = 0; f < 6; ++f) { o->bct[f] = bc_type[f]; o->bcv[f] = bc_val[f]; }
  /* uniform levels 0..lbase, each box list in Morton order */
  for (int l = 0; l <= lb; ++l) {
    o->off[l] = o->nbox;
    uint64_t n = (uint64_t)1 << (3 * l);
    for (uint64_t key = 0; key < n; ++key) {
      int i, j, k;
      unmorton(key, &i, &j, &k);
      add_box(o, l, i, j, k, l ? o->off[l - 1] + (int)(key >> 3) : -1);
    }
    o->off[l + 1] = o->nbox;
  }
  for (int l = 0; l < lb; ++l)
    for (int b = o->off[l]; b < o->off[l + 1]; ++b)
      for (int c = 0; c < 8; ++c)
        o->chl[8 * b + c] = o->off[l + 1] + (int)((o->mort[b] << 3) | (uint64_t)c);
  o->nlev = lb + 1;
  for (int l = 0; l <= lb; ++l) set_neighbours(o, l);
  return o;
}

void orc_destroy(orc *o) {
  if (!o) return;
  free(o->lev); free(o->ijk); free(o->par); free(o->chl); free(o->nbr); free(o->mort);
  for (int v = 0; v < NVAR; ++v) free(o->v[v]);
  free(o->flux); free(o->lu); free(o->piv);
  for (int t = 0; t < 3; ++t) free(o->tab[t]);
  free(o);
}

/* threads used by the box loops (1 when built without OpenMP); returns the
 * count now in effect */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int orc_n_boxes(const orc *o) { return o->nbox; }
int orc_n_levels(const orc *o) { return o->nlev; }
int orc_level_offset(const orc *o, int l) { return (l >= 0 && l <= o->nlev) ? o->off[l] : -1; }

/* Refine the flagged boxes of the finest existing level.  Proper nesting
 * (Sec. 2.1.1): a box is refined only if all 26 neighbour positions of its
 * level hold a box or lie outside the domain; other requests are dropped. */
int orc_refine_level(orc *o, int l, const int8_t *flags, int *n_dropped) {
  if (l != o->nlev - 1 || l >= o->lmax) return -1;
  int dropped = 0, start = o->nbox;
  o->off[l + 2] = o->nbox;
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    if (flags[b - o->off[l]] <= 0) continue;
    int ok = 1;
    for (int d = 0; d < 26; ++d) if (o->nbr[26 * b + d] == -2) ok = 0;
    if (!ok) { ++dropped; continue; }
    for (int c = 0; c < 8; ++c) {
      int nb = add_box(o, l + 1, 2 * o->ijk[3 * b] + (c & 1), 2 * o->ijk[3 * b + 1] + ((c >> 1) & 1),
                       2 * o->ijk[3 * b + 2] + (c >> 2), b);
      o->chl[8 * b + c] = nb;
    }
  }
  if (n_dropped) *n_dropped = dropped;
  if (o->nbox == start) return 0;
  o->off[l + 2] = o->nbox;
  o->nlev = l + 2;
  set_neighbours(o, l + 1);
  return o->nbox - start;
}

void orc_get_tables(const orc *o, int32_t *level, int32_t *ijk, uint64_t *mort,
                    int32_t *parent, int32_t *child, int32_t *nbr) {
  for (int b = 0; b < o->nbox; ++b) {
    if (level) level[b] = o->lev[b];
    if (mort) mort[b] = o->mort[b];
    if (parent) parent[b] = o->par[b];
    for (int d = 0; d < 3; ++d) if (ijk) ijk[3 * b + d] = o->ijk[3 * b + d];
    for (int c = 0; c < 8; ++c) if (child) child[8 * b + c] = o->chl[8 * b + c];
    for (int d = 0; d < 26; ++d) if (nbr) nbr[26 * b + d] = o->nbr[26 * b + d];
  }
}

static int is_leaf(const orc *o, int b) { return o->chl[8 * b] < 0; }
static double spacing(const orc *o, int l) { return o->len / (NC * (double)(1 << l)); }
static double *box(const orc *o, int var, int b) { return o->v[var] + (size_t)BS * b; }

void orc_set(orc *o, int var, const double *src) {
  int v = pub2var[var];
  for (int b = 0; b < o->nbox; ++b)
    for (int k = 0; k < NC; ++k)
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i)
          box(o, v, b)[IX(i, j, k)] = src[(size_t)512 * b + i + 8 * j + 64 * k];
}

void orc_get(const orc *o, int var, double *dst) {
  int v = pub2var[var];
  for (int b = 0; b < o->nbox; ++b)
    for (int k = 0; k < NC; ++k)
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i)
          dst[(size_t)512 * b + i + 8 * j + 64 * k] = box(o, v, b)[IX(i, j, k)];
}

/* ---------------------------------------------------------------------- */
/* ghost cells (Sec. 2.1.3: one ghost layer per box; Sec. 2.1.1: coarse to */
/* fine interpolation)                                                     */
/* ---------------------------------------------------------------------- */

/* interior value of var at level l, global cell g; the box must exist */
static double cell_val(const orc *o, int var, int l, const int g[3]) {
  int b = find_box(o, l, g[0] >> 3, g[1] >> 3, g[2] >> 3);
  if (b < 0) die("coarse value requested where no box exists (nesting)");
  return box(o, var, b)[IX(g[0] & 7, g[1] & 7, g[2] & 7)];
}

/* physical-boundary ghost of an interior cell value across face f:
 * Dirichlet value g at the face -> 2g - inner (homogeneous: -inner);
 * Neumann zero -> inner. */
static double bc_ghost(const orc *o, int f, double inner, int homog) {
  if (o->bct[f] == 1) return (homog ? 0.0 : 2.0 * o->bcv[f]) - inner;
  return inner;
}

/* value at global cell q of level l, which is either inside the domain (a
 * box must exist) or one step outside it from the interior cell `from`. */
static double cell_val_bc(const orc *o, int var, int l, const int q[3], const int from[3], int homog) {
  int n = NC << l;
  for (int d = 0; d < 3; ++d) {
    if (q[d] < 0) return bc_ghost(o, 2 * d, cell_val(o, var, l, from), homog);
    if (q[d] >= n) return bc_ghost(o, 2 * d + 1, cell_val(o, var, l, from), homog);
  }
  return cell_val(o, var, l, q);
}

/* same with Neumann-zero (mirror) ghosts on every face: densities */
static double cell_val_mirror(const orc *o, int var, int l, const int q[3], const int from[3]) {
  int n = NC << l;
  for (int d = 0; d < 3; ++d)
    if (q[d] < 0 || q[d] >= n) return cell_val(o, var, l, from);
  return cell_val(o, var, l, q);
}

/* local cell coordinates of face cell (u,w) of face f at depth t:
 * t = 0 is the interior layer next to the face, t = -1,-2 the ghosts,
 * t = 1 the next interior layer. */
static void face_cell(int f, int t, int u, int w, int c[3]) {
  int a = face_axis(f), t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  c[a] = face_side(f) ? (NC - 1 - t) : t;
  c[t1] = u;
  c[t2] = w;
}

/* Potential ghosts, depth 1, for all boxes of level l.
 * Same-level neighbour: copy.  Physical: bc_ghost.  Refinement boundary:
 * phi_g = phi_f/3 + 2 phihat/3 with phihat = c/2 + c_t1/4 + c_t2/4 the
 * linear interpolation of the coarse cell c containing the ghost and its
 * two tangential coarse neighbours on the ghost's side. */
static void fill_ghosts_phi(orc *o, int var, int l, int homog) {
  BOXES_PAR
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    double *p = box(o, var, b);
    for (int f = 0; f < 6; ++f) {
      int a = face_axis(f), t1 = (a + 1) % 3, t2 = (a + 2) % 3;
      int nb = o->nbr[26 * b + face26(f)];
      for (int w = 0; w < NC; ++w)
        for (int u = 0; u < NC; ++u) {
          int ci[3], cg[3];
          face_cell(f, 0, u, w, ci);
          face_cell(f, -1, u, w, cg);
          double inner = p[IX(ci[0], ci[1], ci[2])];
          double val;
          if (nb >= 0) {
            int cs[3];
            face_cell(f ^ 1, 0, u, w, cs);
            val = box(o, var, nb)[IX(cs[0], cs[1], cs[2])];
          } else if (nb == -1) {
            val = bc_ghost(o, f, inner, homog);
          } else {
            int G[3], cc[3];
            for (int d = 0; d < 3; ++d) { G[d] = o->ijk[3 * b + d] * NC + cg[d]; cc[d] = G[d] >> 1; }
            double phat = 0.5 * cell_val(o, var, l - 1, cc);
            int ts[2] = {t1, t2};
            for (int e = 0; e < 2; ++e) {
              int q[3] = {cc[0], cc[1], cc[2]};
              q[ts[e]] += (G[ts[e]] & 1) ? 1 : -1;
              phat += 0.25 * cell_val_bc(o, var, l - 1, q, cc, homog);
            }
            val = inner / 3.0 + 2.0 * phat / 3.0;
          }
          p[IX(cg[0], cg[1], cg[2])] = val;
        }
    }
  }
}

/* Density ghosts, depth 2 (Sec. 2.3: two fine ghost values at refinement
 * boundaries for the Koren stencil, limited to twice the coarse value). */
static void fill_ghosts_density(orc *o, int var, int l) {
  BOXES_PAR
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    double *p = box(o, var, b);
    for (int f = 0; f < 6; ++f) {
      int nb = o->nbr[26 * b + face26(f)];
      for (int t = 1; t <= 2; ++t)
        for (int w = 0; w < NC; ++w)
          for (int u = 0; u < NC; ++u) {
            int cg[3];
            face_cell(f, -t, u, w, cg);
            double val;
            if (nb >= 0) {
              int cs[3];
              face_cell(f ^ 1, t - 1, u, w, cs);
              val = box(o, var, nb)[IX(cs[0], cs[1], cs[2])];
            } else if (nb == -1) {
              int cm[3];
              face_cell(f, t - 1, u, w, cm);
              val = p[IX(cm[0], cm[1], cm[2])];
            } else {
              /* linear prolongation of the coarse cell containing the
               * ghost: (c + c_sx + c_sy + c_sz)/4, s toward the ghost's
               * position inside c; then limited to 2c */
              int G[3], cc[3];
              for (int d = 0; d < 3; ++d) { G[d] = o->ijk[3 * b + d] * NC + cg[d]; cc[d] = G[d] >> 1; }
              double c = cell_val(o, var, l - 1, cc);
              double sum = c;
              for (int d = 0; d < 3; ++d) {
                int q[3] = {cc[0], cc[1], cc[2]};
                q[d] += (G[d] & 1) ? 1 : -1;
                sum += cell_val_mirror(o, var, l - 1, q, cc);
              }
              val = 0.25 * sum;
              if (val > 2.0 * c) val = 2.0 * c;
            }
            p[IX(cg[0], cg[1], cg[2])] = val;
          }
    }
  }
}

/* |E| ghosts, depth 1: same-level copy, Neumann at walls, and the value of
 * the coarse cell containing the ghost at refinement boundaries. */
static void fill_ghosts_emag(orc *o, int l) {
  BOXES_PAR
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    double *p = box(o, V_EMAG, b);
    for (int f = 0; f < 6; ++f) {
      int nb = o->nbr[26 * b + face26(f)];
      for (int w = 0; w < NC; ++w)
        for (int u = 0; u < NC; ++u) {
          int ci[3], cg[3];
          face_cell(f, 0, u, w, ci);
          face_cell(f, -1, u, w, cg);
          double val;
          if (nb >= 0) {
            int cs[3];
            face_cell(f ^ 1, 0, u, w, cs);
            val = box(o, V_EMAG, nb)[IX(cs[0], cs[1], cs[2])];
          } else if (nb == -1) {
            val = p[IX(ci[0], ci[1], ci[2])];
          } else {
            int cc[3];
            for (int d = 0; d < 3; ++d) cc[d] = (o->ijk[3 * b + d] * NC + cg[d]) >> 1;
            val = cell_val(o, V_EMAG, l - 1, cc);
          }
          p[IX(cg[0], cg[1], cg[2])] = val;
        }
    }
  }
}

/* ---------------------------------------------------------------------- */
/* multigrid (Sec. 2.1.2)                                                  */
/* ---------------------------------------------------------------------- */

static double nbsum(const double *p, int i, int j, int k) {
  return p[IX(i - 1, j, k)] + p[IX(i + 1, j, k)] + p[IX(i, j - 1, k)] +
         p[IX(i, j + 1, k)] + p[IX(i, j, k - 1)] + p[IX(i, j, k + 1)];
}

/* Gauss-Seidel red-black: red = (i+j+k) even in level-global indices (box
 * origins are multiples of 8, so local parity equals global parity).
 * Update phi = (sum of 6 neighbours - h^2 f)/6 of the 7-point Laplacian. */
static void smooth(orc *o, int l, int nu) {
  double h2 = spacing(o, l) * spacing(o, l);
  for (int s = 0; s < nu; ++s)
    for (int color = 0; color < 2; ++color) {
      fill_ghosts_phi(o, V_PHI, l, 0);
      BOXES_PAR
      for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
        double *p = box(o, V_PHI, b), *f = box(o, V_RHS, b);
        for (int k = 0; k < NC; ++k)
          for (int j = 0; j < NC; ++j)
            for (int i = 0; i < NC; ++i) {
              if (((i + j + k) & 1) != color) continue;
              p[IX(i, j, k)] = (nbsum(p, i, j, k) - h2 * f[IX(i, j, k)]) / 6.0;
            }
      }
    }
}

/* r = f - L phi with L phi = (sum6 - 6 phi)/h^2, for the given boxes */
static void residual_box(orc *o, int var_phi, int b, double *r) {
  int l = o->lev[b];
  double h2 = spacing(o, l) * spacing(o, l);
  double *p = box(o, var_phi, b), *f = box(o, V_RHS, b);
  for (int k = 0; k < NC; ++k)
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i)
        r[IX(i, j, k)] = f[IX(i, j, k)] - (nbsum(p, i, j, k) - 6.0 * p[IX(i, j, k)]) / h2;
}

/* average of the 8 children (cell-centred full weighting), for every box of
 * level l-1 that has children */
static void restrict_level(orc *o, int l, int src, int dst) {
  BOXES_PAR
  for (int pb = o->off[l - 1]; pb < o->off[l]; ++pb) {
    if (is_leaf(o, pb)) continue;
    double *d = box(o, dst, pb);
    for (int K = 0; K < NC; ++K)
      for (int J = 0; J < NC; ++J)
        for (int I = 0; I < NC; ++I) {
          int c = (I >> 2) + 2 * (J >> 2) + 4 * (K >> 2);
          const double *s = box(o, src, o->chl[8 * pb + c]);
          int i0 = 2 * (I & 3), j0 = 2 * (J & 3), k0 = 2 * (K & 3);
          double sum = 0.0;
          for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
              for (int di = 0; di < 2; ++di) sum += s[IX(i0 + di, j0 + dj, k0 + dk)];
          d[IX(I, J, K)] = sum / 8.0;
        }
  }
}

/* Linear prolongation of level l-1 values to each cell of each level-l box:
 * (c + c_sx + c_sy + c_sz)/4, c the parent cell and c_sd its neighbour in
 * the direction of the fine cell's offset.  add=1 adds it (correction),
 * add=0 overwrites (full solution in FMG). */
static void prolong_level(orc *o, int l, int src, int dst, int homog, int add) {
  BOXES_PAR
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    double *d = box(o, dst, b);
    for (int k = 0; k < NC; ++k)
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i) {
          int G[3] = {o->ijk[3 * b] * NC + i, o->ijk[3 * b + 1] * NC + j, o->ijk[3 * b + 2] * NC + k};
          int cc[3] = {G[0] >> 1, G[1] >> 1, G[2] >> 1};
          double sum = cell_val(o, src, l - 1, cc);
          for (int e = 0; e < 3; ++e) {
            int q[3] = {cc[0], cc[1], cc[2]};
            q[e] += (G[e] & 1) ? 1 : -1;
            sum += cell_val_bc(o, src, l - 1, q, cc, homog);
          }
          if (add) d[IX(i, j, k)] += 0.25 * sum;
          else d[IX(i, j, k)] = 0.25 * sum;
        }
  }
}

/* Exact solve on level 0 (one box): dense LU with partial pivoting of the
 * 512x512 7-point operator with the boundary rules folded in. */
static void coarse_factor(orc *o) {
  const int n = 512;
  double h2 = spacing(o, 0) * spacing(o, 0);
  o->lu = calloc((size_t)n * n, sizeof(double));
  o->piv = calloc(n, sizeof(int));
  double *A = o->lu;
  for (int k = 0; k < NC; ++k)
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) {
        int r = i + 8 * j + 64 * k, c[3] = {i, j, k};
        A[(size_t)r * n + r] -= 6.0 / h2;
        for (int f = 0; f < 6; ++f) {
          int q[3] = {c[0], c[1], c[2]};
          q[face_axis(f)] += face_side(f) ? 1 : -1;
          if (q[face_axis(f)] < 0 || q[face_axis(f)] >= NC) {
            /* ghost = (2g) - phi (Dirichlet) or phi (Neumann) */
            A[(size_t)r * n + r] += (o->bct[f] == 1 ? -1.0 : 1.0) / h2;
          } else {
            A[(size_t)r * n + (q[0] + 8 * q[1] + 64 * q[2])] += 1.0 / h2;
          }
        }
      }
  for (int col = 0; col < n; ++col) {
    int p = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(A[(size_t)r * n + col]) > fabs(A[(size_t)p * n + col])) p = r;
    o->piv[col] = p;
    if (p != col)
      for (int c = 0; c < n; ++c) {
        double t = A[(size_t)col * n + c];
        A[(size_t)col * n + c] = A[(size_t)p * n + c];
        A[(size_t)p * n + c] = t;
      }
    for (int r = col + 1; r < n; ++r) {
      double m = A[(size_t)r * n + col] / A[(size_t)col * n + col];
      A[(size_t)r * n + col] = m;
      for (int c = col + 1; c < n; ++c) A[(size_t)r * n + c] -= m * A[(size_t)col * n + c];
    }
  }
}

void orc_coarse_solve(orc *o) {
  const int n = 512;
  if (!o->lu) coarse_factor(o);
  double h2 = spacing(o, 0) * spacing(o, 0);
  double x[512];
  double *f = box(o, V_RHS, 0), *p = box(o, V_PHI, 0);
  for (int k = 0; k < NC; ++k)
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) {
        int c[3] = {i, j, k};
        double rhs = f[IX(i, j, k)];
        for (int fc = 0; fc < 6; ++fc) {
          int q = c[face_axis(fc)] + (face_side(fc) ? 1 : -1);
          if ((q < 0 || q >= NC) && o->bct[fc] == 1) rhs -= 2.0 * o->bcv[fc] / h2;
        }
        x[i + 8 * j + 64 * k] = rhs;
      }
  for (int r = 0; r < n; ++r) {
    double t = x[r]; x[r] = x[o->piv[r]]; x[o->piv[r]] = t;
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < r; ++c) x[r] -= o->lu[(size_t)r * n + c] * x[c];
  for (int r = n - 1; r >= 0; --r) {
    for (int c = r + 1; c < n; ++c) x[r] -= o->lu[(size_t)r * n + c] * x[c];
    x[r] /= o->lu[(size_t)r * n + r];
  }
  for (int k = 0; k < NC; ++k)
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) p[IX(i, j, k)] = x[i + 8 * j + 64 * k];
}

/* Full approximation scheme V-cycle with top level `top` (Sec. 2.1.2).
 * Down: smooth nu1, residual, restrict phi and residual, keep a copy of the
 * restricted coarse level, FAS right-hand side on refined coarse boxes.
 * Bottom: exact solve.  Up: add the prolonged coarse correction, smooth
 * nu2. */
static void vcycle(orc *o, int top, int nu1, int nu2) {
  for (int l = top; l >= 1; --l) {
    smooth(o, l, nu1);
    fill_ghosts_phi(o, V_PHI, l, 0);
    BOXES_PAR
    for (int b = o->off[l]; b < o->off[l + 1]; ++b) residual_box(o, V_PHI, b, box(o, V_RES, b));
    restrict_level(o, l, V_PHI, V_PHI);
    BOXES_PAR
    for (int b = o->off[l - 1]; b < o->off[l]; ++b)
      memcpy(box(o, V_OLD, b), box(o, V_PHI, b), sizeof(double) * BS);
    restrict_level(o, l, V_RES, V_RHS);
    fill_ghosts_phi(o, V_PHI, l - 1, 0);
    double h2 = spacing(o, l - 1) * spacing(o, l - 1);
    BOXES_PAR
    for (int b = o->off[l - 1]; b < o->off[l]; ++b) {
      if (is_leaf(o, b)) continue;
      double *p = box(o, V_PHI, b), *f = box(o, V_RHS, b);
      for (int k = 0; k < NC; ++k)
        for (int j = 0; j < NC; ++j)
          for (int i = 0; i < NC; ++i)
            f[IX(i, j, k)] += (nbsum(p, i, j, k) - 6.0 * p[IX(i, j, k)]) / h2;
    }
  }
  orc_coarse_solve(o);
  for (int l = 1; l <= top; ++l) {
    BOXES_PAR
    for (int b = o->off[l - 1]; b < o->off[l]; ++b) {
      double *t = box(o, V_TMP, b), *p = box(o, V_PHI, b), *q = box(o, V_OLD, b);
      for (int c = 0; c < BS; ++c) t[c] = p[c] - q[c];
    }
    prolong_level(o, l, V_TMP, V_PHI, 1, 1);
    smooth(o, l, nu2);
  }
}

/* max over leaf cells (boxes without children, or on level top) of |r| */
static double leaf_resmax(orc *o, int var_phi, int top) {
  double m = 0.0;
  for (int l = 0; l <= top; ++l) {
    fill_ghosts_phi(o, var_phi, l, 0);
#pragma omp parallel for schedule(static) reduction(max : m)
    for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
      if (!is_leaf(o, b) && l != top) continue;
      double r[BS];
      residual_box(o, var_phi, b, r);
      for (int k = 0; k < NC; ++k)
        for (int j = 0; j < NC; ++j)
          for (int i = 0; i < NC; ++i) {
            double a = fabs(r[IX(i, j, k)]);
            if (a > m) m = a;
          }
    }
  }
  return m;
}

/* relative residual: max_leaf |f - L phi| / max_leaf |f - L 0| */
double orc_rel_residual(orc *o) {
  int top = o->nlev - 1;
  double num = leaf_resmax(o, V_PHI, top);
  memset(o->v[V_TMP], 0, sizeof(double) * BS * (size_t)o->nbox);
  double den = leaf_resmax(o, V_TMP, top);
  return den > 0.0 ? num / den : num;
}

int orc_vcycles(orc *o, int n, int nu1, int nu2, double *rel) {
  for (int c = 0; c < n; ++c) vcycle(o, o->nlev - 1, nu1, nu2);
  if (rel) *rel = orc_rel_residual(o);
  return 0;
}

int orc_solve(orc *o, double tol, int max_cycles, int nu1, int nu2, double *rel, int *cycles) {
  double r = 0.0;
  int c = 0;
  do {
    vcycle(o, o->nlev - 1, nu1, nu2);
    ++c;
    r = orc_rel_residual(o);
  } while (r > tol && c < max_cycles);
  if (rel) *rel = r;
  if (cycles) *cycles = c;
  return r <= tol ? 0 : -4;
}

/* Full multigrid: restrict f to every refined box, solve on level 0, then
 * for each finer level prolong the solution and run one V-cycle with that
 * level on top; then V-cycles on the full hierarchy to the tolerance. */
int orc_fmg(orc *o, double tol, int max_cycles, int nu1, int nu2, double *rel, int *cycles) {
  int top = o->nlev - 1;
  for (int l = top; l >= 1; --l) restrict_level(o, l, V_RHS, V_RHS);
  orc_coarse_solve(o);
  for (int l = 1; l <= top; ++l) {
    prolong_level(o, l, V_PHI, V_PHI, 0, 0);
    vcycle(o, l, nu1, nu2);
  }
  int c = 1;
  double r = orc_rel_residual(o);
  while (r > tol && c < max_cycles) {
    vcycle(o, top, nu1, nu2);
    ++c;
    r = orc_rel_residual(o);
  }
  if (rel) *rel = r;
  if (cycles) *cycles = c;
  return r <= tol ? 0 : -4;
}

/* leaf residual with every refined box holding the average of its children
 * (the composite-grid operator applied to the leaf values) */
void orc_composite_residual(orc *o) {
  int top = o->nlev - 1;
  for (int l = top; l >= 1; --l) restrict_level(o, l, V_PHI, V_PHI);
  for (int l = 0; l <= top; ++l) {
    fill_ghosts_phi(o, V_PHI, l, 0);
    BOXES_PAR
    for (int b = o->off[l]; b < o->off[l + 1]; ++b)
      if (is_leaf(o, b)) residual_box(o, V_PHI, b, box(o, V_RES, b));
  }
}

/* Eq. 5 right-hand side on leaf cells: f = -q (n_i - n_e)/eps, or -rho/eps */
void orc_charge_rhs(orc *o, double q, double eps, int use_rho) {
  BOXES_PAR
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    double *f = box(o, V_RHS, b), *ne = box(o, V_NE, b), *ni = box(o, V_NI, b), *rho = box(o, V_RHO, b);
    for (int k = 0; k < NC; ++k)
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i) {
          int c = IX(i, j, k);
          f[c] = use_rho ? -rho[c] / eps : -q * (ni[c] - ne[c]) / eps;
        }
  }
}

/* ---------------------------------------------------------------------- */
/* field (Sec. 2.3)                                                        */
/* ---------------------------------------------------------------------- */

/* face field E_{i+1/2} = (phi_i - phi_{i+1})/dx; cell component = mean of
 * its two faces; |E| = sqrt of the sum of squares.  Leaf cells only. */
static void cell_field(const double *p, int i, int j, int k, double h, double e[3]) {
  int c[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    int m[3] = {c[0], c[1], c[2]}, pl[3] = {c[0], c[1], c[2]};
    m[a] -= 1; pl[a] += 1;
    double e_lo = (p[IX(m[0], m[1], m[2])] - p[IX(i, j, k)]) / h;
    double e_hi = (p[IX(i, j, k)] - p[IX(pl[0], pl[1], pl[2])]) / h;
    e[a] = (e_lo + e_hi) / 2.0;
  }
}

void orc_compute_field(orc *o) {
  for (int l = 0; l < o->nlev; ++l) {
    fill_ghosts_phi(o, V_PHI, l, 0);
    double h = spacing(o, l);
    BOXES_PAR
    for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
      double *p = box(o, V_PHI, b), *em = box(o, V_EMAG, b);
      for (int k = 0; k < NC; ++k)
        for (int j = 0; j < NC; ++j)
          for (int i = 0; i < NC; ++i) {
            if (!is_leaf(o, b)) { em[IX(i, j, k)] = 0.0; continue; }
            double e[3];
            cell_field(p, i, j, k, h, e);
            em[IX(i, j, k)] = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
          }
    }
  }
}

/* ---------------------------------------------------------------------- */
/* fluid step (Sec. 2.2-2.4)                                               */
/* ---------------------------------------------------------------------- */

void orc_set_table(orc *o, int n, double e_max, const double *mu, const double *diff,
                   const double *alpha) {
  o->tab_n = n;
  o->tab_emax = e_max;
  const double *src[3] = {mu, diff, alpha};
  for (int t = 0; t < 3; ++t) {
    free(o->tab[t]);
    o->tab[t] = malloc(sizeof(double) * n);
    memcpy(o->tab[t], src[t], sizeof(double) * n);
  }
}

/* table at E_k = k e_max/(n-1), linear interpolation, clamped at the ends */
double orc_lookup(const orc *o, int which, double e) {
  const double *t = o->tab[which];
  int n = o->tab_n;
  double x = e / (o->tab_emax / (n - 1));
  if (x <= 0.0) return t[0];
  if (x >= n - 1) return t[n - 1];
  int i = (int)x;
  double w = x - i;
  return t[i] + w * (t[i + 1] - t[i]);
}

/* psi(a/b) * b for the Koren limiter psi(x) = max(0, min(1, (2+x)/6, x)),
 * written without the division (zero when a*b <= 0) */
double orc_koren(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  double ab = fabs(b), aa = fabs(a);
  double m = ab;
  if ((2.0 * ab + aa) / 6.0 < m) m = (2.0 * ab + aa) / 6.0;
  if (aa < m) m = aa;
  return b > 0.0 ? m : -m;
}

static double *fluxp(orc *o, int b, int a) { return o->flux + ((size_t)b * 3 + a) * 9 * 64; }

/* Face fluxes of every leaf box: advective part by Eq. 6 (v < 0) or Eq. 7
 * (v >= 0) with v = -mu(E*) E_face, E* the mean of the two cell |E|;
 * diffusive part -D(E*) (n_R - n_L)/dx.  Flux index [a][m][w][u]: m = 0..8
 * is the face between cells m-1 and m along axis a, u,w the tangential
 * coordinates along axes (a+1)%3, (a+2)%3. */
static void leaf_fluxes(orc *o, int var_n) {
  BOXES_PAR
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    double h = spacing(o, o->lev[b]);
    const double *n = box(o, var_n, b), *p = box(o, V_PHI, b), *em = box(o, V_EMAG, b);
    for (int a = 0; a < 3; ++a) {
      int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
      double *F = fluxp(o, b, a);
      for (int m = 0; m <= NC; ++m)
        for (int w = 0; w < NC; ++w)
          for (int u = 0; u < NC; ++u) {
            int c[4][3];
            for (int s = 0; s < 4; ++s) {
              c[s][a] = m - 2 + s;
              c[s][t1] = u;
              c[s][t2] = w;
            }
            double nL2 = n[IX(c[0][0], c[0][1], c[0][2])], nL = n[IX(c[1][0], c[1][1], c[1][2])];
            double nR = n[IX(c[2][0], c[2][1], c[2][2])], nR2 = n[IX(c[3][0], c[3][1], c[3][2])];
            double pL = p[IX(c[1][0], c[1][1], c[1][2])], pR = p[IX(c[2][0], c[2][1], c[2][2])];
            double eL = em[IX(c[1][0], c[1][1], c[1][2])], eR = em[IX(c[2][0], c[2][1], c[2][2])];
            double e_face = (pL - pR) / h;
            double e_star = (eL + eR) / 2.0;
            double mu = orc_lookup(o, 0, e_star), dc = orc_lookup(o, 1, e_star);
            double v = -mu * e_face;
            double nf;
            if (v < 0.0) nf = nR - orc_koren(nR2 - nR, nR - nL);
            else nf = nL + orc_koren(nL - nL2, nR - nL);
            F[(m * NC + w) * NC + u] = v * nf - dc * (nR - nL) / h;
          }
    }
  }
  /* refinement boundaries: a coarse leaf face next to a refined box takes
   * the mean of the four fine face fluxes (conservation, Sec. 2.3) */
  BOXES_PAR
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    for (int f = 0; f < 6; ++f) {
      int nb = o->nbr[26 * b + face26(f)];
      if (nb < 0 || is_leaf(o, nb)) continue;
      int a = face_axis(f), side = face_side(f);
      double *F = fluxp(o, b, a);
      for (int w = 0; w < NC; ++w)
        for (int u = 0; u < NC; ++u) {
          int cidx[3];
          cidx[a] = side ? 0 : 1;
          cidx[(a + 1) % 3] = u >> 2;
          cidx[(a + 2) % 3] = w >> 2;
          int ch = o->chl[8 * nb + cidx[0] + 2 * cidx[1] + 4 * cidx[2]];
          const double *Fc = fluxp(o, ch, a);
          int mc = side ? 0 : NC;
          double s = 0.0;
          for (int dw = 0; dw < 2; ++dw)
            for (int du = 0; du < 2; ++du)
              s += Fc[(mc * NC + 2 * (w & 3) + dw) * NC + 2 * (u & 3) + du];
          F[((side ? NC : 0) * NC + w) * NC + u] = s / 4.0;
        }
    }
  }
}

/* refined boxes of both densities := average of their children, finest
 * level first */
static void restrict_densities(orc *o, int ne, int ni) {
  for (int l = o->nlev - 1; l >= 1; --l) {
    restrict_level(o, l, ne, ne);
    restrict_level(o, l, ni, ni);
  }
}

/* One forward Euler step dst = src + dt F(src) (Eq. 2-3) on leaf cells,
 * using the stored potential and |E|; then refined boxes get the average of
 * their children. */
static void euler_stage(orc *o, int sne, int sni, int dne, int dni, double dt) {
  for (int l = 0; l < o->nlev; ++l) {
    fill_ghosts_density(o, sne, l);
    fill_ghosts_phi(o, V_PHI, l, 0);
    fill_ghosts_emag(o, l);
  }
  leaf_fluxes(o, sne);
  BOXES_PAR
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    double h = spacing(o, o->lev[b]);
    const double *ne = box(o, sne, b), *ni = box(o, sni, b), *em = box(o, V_EMAG, b);
    double *one = box(o, dne, b), *oni = box(o, dni, b);
    const double *F[3] = {fluxp(o, b, 0), fluxp(o, b, 1), fluxp(o, b, 2)};
    for (int k = 0; k < NC; ++k)
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i) {
          int c[3] = {i, j, k};
          double div = 0.0;
          for (int a = 0; a < 3; ++a) {
            int u = c[(a + 1) % 3], w = c[(a + 2) % 3], m = c[a];
            div += (F[a][((m + 1) * NC + w) * NC + u] - F[a][(m * NC + w) * NC + u]) / h;
          }
          double e = em[IX(i, j, k)];
          double src = orc_lookup(o, 2, e) * orc_lookup(o, 0, e) * e * ne[IX(i, j, k)];
          one[IX(i, j, k)] = ne[IX(i, j, k)] - dt * div + dt * src;
          oni[IX(i, j, k)] = ni[IX(i, j, k)] + dt * src;
        }
  }
  restrict_densities(o, dne, dni);
}

/* one Euler stage on the current densities (refined boxes first get the
 * average of their children, so only leaf values matter) */
void orc_fluid_stage(orc *o, double dt) {
  restrict_densities(o, V_NE, V_NI);
  euler_stage(o, V_NE, V_NI, V_NE1, V_NI1, dt);
  memcpy(o->v[V_NE], o->v[V_NE1], sizeof(double) * BS * (size_t)o->nbox);
  memcpy(o->v[V_NI], o->v[V_NI1], sizeof(double) * BS * (size_t)o->nbox);
}

/* Time-step limits of Sec. 2.4 from the current field and electron density:
 * CFL 0.5 on sum |v_d|/dx, advection+diffusion (sum |v_d|/dx + 2*3*D/dx^2)
 * below 1, dielectric relaxation eps0/(e mu n_e); times the safety 0.9. */
double orc_dt_limit(orc *o, double q, double eps) {
  double m_adv = 0.0, m_ad = 0.0, m_drt = 0.0;
  for (int l = 0; l < o->nlev; ++l) fill_ghosts_phi(o, V_PHI, l, 0);
#pragma omp parallel for schedule(static) reduction(max : m_adv, m_ad, m_drt)
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    double h = spacing(o, o->lev[b]);
    const double *p = box(o, V_PHI, b), *em = box(o, V_EMAG, b), *ne = box(o, V_NE, b);
    for (int k = 0; k < NC; ++k)
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i) {
          double e[3];
          cell_field(p, i, j, k, h, e);
          double mu = orc_lookup(o, 0, em[IX(i, j, k)]), dc = orc_lookup(o, 1, em[IX(i, j, k)]);
          double adv = (fabs(mu * e[0]) + fabs(mu * e[1]) + fabs(mu * e[2])) / h;
          double ad = adv + 2.0 * 3.0 * dc / (h * h);
          double drt = mu * ne[IX(i, j, k)];
          if (adv > m_adv) m_adv = adv;
          if (ad > m_ad) m_ad = ad;
          if (drt > m_drt) m_drt = drt;
        }
  }
  double dt = 1e300;
  if (m_adv > 0.0 && 0.5 / m_adv < dt) dt = 0.5 / m_adv;
  if (m_ad > 0.0 && 1.0 / m_ad < dt) dt = 1.0 / m_ad;
  if (m_drt > 0.0 && eps / (q * m_drt) < dt) dt = eps / (q * m_drt);
  return 0.9 * dt;
}

/* Explicit trapezoidal (Heun) step of Sec. 2.4: keep n0; Euler to n1; new
 * field; Euler from n1 to n2; n = (n0 + n2)/2; new field.  The next time
 * step is evaluated at the second stage. */
int orc_advance(orc *o, double dt, double q, double eps, double tol, int max_cycles,
                int nu1, int nu2, double *dt_next, int *cycles1, int *cycles2) {
  size_t bytes = sizeof(double) * BS * (size_t)o->nbox;
  restrict_densities(o, V_NE, V_NI);
  memcpy(o->v[V_NE0], o->v[V_NE], bytes);
  memcpy(o->v[V_NI0], o->v[V_NI], bytes);
  euler_stage(o, V_NE0, V_NI0, V_NE, V_NI, dt);
  orc_charge_rhs(o, q, eps, 0);
  int st = orc_solve(o, tol, max_cycles, nu1, nu2, NULL, cycles1);
  orc_compute_field(o);
  if (dt_next) *dt_next = orc_dt_limit(o, q, eps);
  euler_stage(o, V_NE, V_NI, V_NE1, V_NI1, dt);
  for (size_t c = 0; c < (size_t)BS * o->nbox; ++c) {
    o->v[V_NE][c] = (o->v[V_NE0][c] + o->v[V_NE1][c]) / 2.0;
    o->v[V_NI][c] = (o->v[V_NI0][c] + o->v[V_NI1][c]) / 2.0;
  }
  orc_charge_rhs(o, q, eps, 0);
  int st2 = orc_solve(o, tol, max_cycles, nu1, nu2, NULL, cycles2);
  orc_compute_field(o);
  return st ? st : st2;
}

/* ---------------------------------------------------------------------- */
/* refinement criterion and regridding (Sec. 2.5, Eq. 8)                   */
/* ---------------------------------------------------------------------- */

/* Eq. 8 asks dx < c0 c1 / alpha(c1 |E|) of every cell.  With the ionization
 * coefficient from the table (Sec. 2.3) a cell needs refinement where the
 * criterion fails, alpha(c1 |E|) dx >= c0 c1 (no division).  A leaf box is
 * flagged +1 when one of its cells needs refinement, or when a cell of a
 * same-level leaf neighbour within `buffer` cells of it (Chebyshev distance
 * in cells of that level) does, and its level is below the maximum.  A
 * leaf above the base grid that is not flagged is derefinable (-1) when
 * every cell satisfies the criterion with c0_deref and dx < dx_deref.
 * Other boxes get 0.  Uses the stored |E| of the leaf cells. */
void orc_refine_flags(orc *o, double c0, double c1, double c0_deref, double dx_deref, int buffer,
                      int8_t *flags) {
  unsigned char *need = calloc((size_t)512 * o->nbox, 1);
  unsigned char *any = calloc((size_t)o->nbox, 1), *fine = calloc((size_t)o->nbox, 1);
  for (int b = 0; b < o->nbox; ++b) {
    flags[b] = 0;
    if (!is_leaf(o, b)) continue;
    double dx = spacing(o, o->lev[b]);
    const double *em = box(o, V_EMAG, b);
    int ok = dx < dx_deref;
    for (int k = 0; k < NC; ++k)
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i) {
          double a = orc_lookup(o, 2, c1 * em[IX(i, j, k)]);
          if (a * dx >= c0 * c1) { need[(size_t)512 * b + i + 8 * j + 64 * k] = 1; any[b] = 1; }
          if (!(a * dx < c0_deref * c1)) ok = 0;
        }
    fine[b] = (unsigned char)ok;
  }
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    int marked = any[b];
    for (int d = 0; d < 26 && !marked; ++d) {
      int n = o->nbr[26 * b + d];
      if (n < 0 || !is_leaf(o, n) || !any[n]) continue;
      for (int c = 0; c < 512 && !marked; ++c) {
        if (!need[(size_t)512 * n + c]) continue;
        int g[3] = {o->ijk[3 * n] * NC + (c & 7), o->ijk[3 * n + 1] * NC + ((c >> 3) & 7),
                    o->ijk[3 * n + 2] * NC + (c >> 6)};
        int dist = 0;
        for (int e = 0; e < 3; ++e) {
          int lo = o->ijk[3 * b + e] * NC, hi = lo + NC - 1;
          int de = g[e] < lo ? lo - g[e] : (g[e] > hi ? g[e] - hi : 0);
          if (de > dist) dist = de;
        }
        if (dist <= buffer) marked = 1;
      }
    }
    if (marked) {
      if (o->lev[b] < o->lmax) flags[b] = 1;
    } else if (fine[b] && o->lev[b] > o->lbase) {
      flags[b] = -1;
    }
  }
  free(need); free(any); free(fine);
}

typedef struct { int lev, i, j, k, src; uint64_t key; } orc_ent;

static int ent_cmp(const void *pa, const void *pb) {
  const orc_ent *a = pa, *b = pb;
  if (a->lev != b->lev) return a->lev < b->lev ? -1 : 1;
  return a->key < b->key ? -1 : (a->key > b->key ? 1 : 0);
}

/* Apply per-box flags (+1 refine, -1 derefine, leaves only; the layout of
 * orc_refine_flags).  Refinement: a flagged leaf below the maximum level
 * gets 8 children when all 26 neighbour positions of its level hold a box
 * or lie outside the domain (proper nesting, Sec. 2.1.1); other requests
 * are dropped.  Derefinement: a box whose 8 children are all leaves
 * flagged -1 loses them, unless a neighbour of one of the children (not a
 * sibling) has children or is refined in this call, which would break the
 * nesting.  The mesh is rebuilt in (level, Morton) order; kept boxes keep
 * all their data; new children get the potential by the linear
 * prolongation (c + c_sx + c_sy + c_sz)/4 of their parent's cells and the
 * densities by the same prolongation limited to 2c (mirror ghosts at the
 * walls), every other variable zero.  Densities are restricted first, so a
 * box that becomes a leaf holds the mean of its former children. */
int orc_regrid(orc *o, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped) {
  restrict_densities(o, V_NE, V_NI);
  int nb0 = o->nbox;
  unsigned char *ref = calloc((size_t)nb0, 1), *der = calloc((size_t)nb0, 1);
  int nref = 0, nder = 0, ndrop = 0;
  for (int b = 0; b < nb0; ++b) {
    if (!is_leaf(o, b) || flags[b] <= 0 || o->lev[b] >= o->lmax) continue;
    int ok = 1;
    for (int d = 0; d < 26; ++d) if (o->nbr[26 * b + d] == -2) ok = 0;
    if (ok) { ref[b] = 1; ++nref; } else ++ndrop;
  }
  for (int p = 0; p < nb0; ++p) {
    if (is_leaf(o, p)) continue;
    int ok = 1;
    for (int c = 0; c < 8 && ok; ++c) {
      int ch = o->chl[8 * p + c];
      if (!is_leaf(o, ch) || flags[ch] >= 0) ok = 0;
    }
    for (int c = 0; c < 8 && ok; ++c) {
      int ch = o->chl[8 * p + c];
      for (int d = 0; d < 26 && ok; ++d) {
        int n = o->nbr[26 * ch + d];
        if (n >= 0 && o->par[n] != p && (!is_leaf(o, n) || ref[n])) ok = 0;
      }
    }
    if (ok) { der[p] = 1; ++nder; }
  }
  /* new box list: old boxes except children of derefined boxes, plus the
   * children of refined leaves; their prolonged data computed on the old mesh */
  int nnew = 0;
  orc_ent *e = malloc(sizeof(orc_ent) * (size_t)(nb0 + 8 * nref));
  double *pro = malloc(sizeof(double) * 3 * 512 * (size_t)(8 * nref + 1));
  int npro = 0;
  for (int b = 0; b < nb0; ++b) {
    if (o->par[b] >= 0 && der[o->par[b]]) continue;
    orc_ent x = {o->lev[b], o->ijk[3 * b], o->ijk[3 * b + 1], o->ijk[3 * b + 2], b, o->mort[b]};
    e[nnew++] = x;
    if (!ref[b]) continue;
    int l = o->lev[b];
    for (int c = 0; c < 8; ++c) {
      int ci = 2 * o->ijk[3 * b] + (c & 1), cj = 2 * o->ijk[3 * b + 1] + ((c >> 1) & 1),
          ck = 2 * o->ijk[3 * b + 2] + (c >> 2);
      orc_ent y = {l + 1, ci, cj, ck, -1 - npro, morton(ci, cj, ck)};
      e[nnew++] = y;
      double *dst = pro + (size_t)3 * 512 * npro;
      const int vars[3] = {V_PHI, V_NE, V_NI};
      for (int v = 0; v < 3; ++v)
        for (int kk = 0; kk < NC; ++kk)
          for (int jj = 0; jj < NC; ++jj)
            for (int ii = 0; ii < NC; ++ii) {
              int G[3] = {ci * NC + ii, cj * NC + jj, ck * NC + kk};
              int cc[3] = {G[0] >> 1, G[1] >> 1, G[2] >> 1};
              double cval = cell_val(o, vars[v], l, cc), sum = cval;
              for (int a = 0; a < 3; ++a) {
                int q[3] = {cc[0], cc[1], cc[2]};
                q[a] += (G[a] & 1) ? 1 : -1;
                sum += v == 0 ? cell_val_bc(o, vars[v], l, q, cc, 0) : cell_val_mirror(o, vars[v], l, q, cc);
              }
              double val = 0.25 * sum;
              if (v > 0 && val > 2.0 * cval) val = 2.0 * cval;
              dst[(size_t)512 * v + ii + 8 * jj + 64 * kk] = val;
            }
      ++npro;
    }
  }
  qsort(e, (size_t)nnew, sizeof(orc_ent), ent_cmp);
  /* rebuild tables and fields */
  int cap = o->cap > nnew ? o->cap : nnew;
  int *lev = malloc(sizeof(int) * cap), *ijk = malloc(sizeof(int) * 3 * cap);
  int *par = malloc(sizeof(int) * cap), *chl = malloc(sizeof(int) * 8 * cap);
  int *nbr = malloc(sizeof(int) * 26 * cap);
  uint64_t *mort = malloc(sizeof(uint64_t) * cap);
  double *nv[NVAR];
  for (int v = 0; v < NVAR; ++v) nv[v] = calloc((size_t)BS * cap, sizeof(double));
  for (int b = 0; b < nnew; ++b) {
    lev[b] = e[b].lev;
    ijk[3 * b] = e[b].i; ijk[3 * b + 1] = e[b].j; ijk[3 * b + 2] = e[b].k;
    mort[b] = e[b].key;
    if (e[b].src >= 0) {
      for (int v = 0; v < NVAR; ++v)
        memcpy(nv[v] + (size_t)BS * b, o->v[v] + (size_t)BS * e[b].src, sizeof(double) * BS);
    } else {
      const double *src = pro + (size_t)3 * 512 * (-1 - e[b].src);
      const int vars[3] = {V_PHI, V_NE, V_NI};
      for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 512; ++c)
          nv[vars[v]][(size_t)BS * b + IX(c & 7, (c >> 3) & 7, c >> 6)] = src[(size_t)512 * v + c];
    }
  }
  free(o->lev); free(o->ijk); free(o->par); free(o->chl); free(o->nbr); free(o->mort);
  for (int v = 0; v < NVAR; ++v) { free(o->v[v]); o->v[v] = nv[v]; }
  o->lev = lev; o->ijk = ijk; o->par = par; o->chl = chl; o->nbr = nbr; o->mort = mort;
  if (cap > o->cap) o->flux = realloc(o->flux, sizeof(double) * 3 * 9 * 64 * (size_t)cap);
  o->cap = cap;
  o->nbox = nnew;
  int nlev = 0;
  for (int b = 0; b < nnew; ++b) if (lev[b] + 1 > nlev) nlev = lev[b] + 1;
  o->nlev = nlev;
  for (int l = 0, b = 0; l <= nlev; ++l) {
    while (b < nnew && lev[b] < l) ++b;
    o->off[l] = b;
  }
  for (int l = nlev + 1; l <= MAXL + 1; ++l) o->off[l] = nnew;
  for (int b = 0; b < nnew; ++b) {
    par[b] = lev[b] ? find_box(o, lev[b] - 1, ijk[3 * b] >> 1, ijk[3 * b + 1] >> 1, ijk[3 * b + 2] >> 1) : -1;
    for (int c = 0; c < 8; ++c)
      chl[8 * b + c] = lev[b] + 1 < nlev ? find_box(o, lev[b] + 1, 2 * ijk[3 * b] + (c & 1),
                                                    2 * ijk[3 * b + 1] + ((c >> 1) & 1), 2 * ijk[3 * b + 2] + (c >> 2))
                                         : -2;
    if (chl[8 * b] < 0)
      for (int c = 0; c < 8; ++c) chl[8 * b + c] = -1;
  }
  for (int l = 0; l < nlev; ++l) set_neighbours(o, l);
  free(e); free(pro); free(ref); free(der);
  if (n_refined) *n_refined = nref;
  if (n_derefined) *n_derefined = nder;
  if (n_dropped) *n_dropped = ndrop;
  return nref + nder;
}
