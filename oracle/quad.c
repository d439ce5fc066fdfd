/* quad.c -- plain, slow, obviously correct CPU oracle of the 2-D and
 * axisymmetric variants of the path of arXiv:1708.08434 (Sec. 1 and 2.1.1:
 * quadtree grids; 2-D, axisymmetric and 3-D runs are supported): the
 * geometric multigrid Poisson solve on a quadtree of 8^2-cell boxes
 * (Sec. 2.1.2, Eq. 1 and 5) and the explicit drift-diffusion-reaction step
 * (Sec. 2.2-2.4, Eq. 2-3, 6-7), in Cartesian (x, y) or cylindrical (r, z)
 * coordinates.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, the smoke check and the
 * CPU-baseline leg of bench.py.  The CUDA library never calls it and shares
 * nothing with it.
 *
 * Data structure: every box stores its variables with two ghost layers
 * (12^2 doubles); ghost layers are filled explicitly before each stencil
 * sweep, and coarse values needed at refinement boundaries are found by
 * global cell coordinates and binary search over Morton keys.
 *
 * The paper states no 2-D or cylindrical formulas.  The readings (all
 * listed in the design notes): the 2-D forms of the 3-D rules (coarse-fine
 * ghost phi_f/3 + 2 phihat/3 with phihat = 3/4 c + 1/4 c_t; prolongation
 * (2c + c_x + c_y)/4; restriction the mean of the four children), and in
 * cylindrical coordinates the finite-volume operators of the divergence
 * form, (1/r) d/dr (r d/dr) + d2/dz2: radial face fluxes weighted by the
 * face radius over the cell-centre radius, restriction and refinement-face
 * flux means weighted by cell and face radius (volume and area), and no
 * flux through the axis r = 0.
 */
#include "quad.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* OpenMP over the boxes of one pass: each box writes only its own cells
 * and ghosts, the only cross-box reductions are maxima, so results do not
 * depend on the thread count. */
#define BOXES_PAR _Pragma("omp parallel for schedule(static)")

#define NC 8               /* cells per box side */
#define GH 2               /* ghost layers stored */
#define SS (NC + 2 * GH)   /* 12 */
#define BS (SS * SS)       /* doubles per stored box */
#define MAXL 30
#define IX(i, j) ((((j) + GH) * SS) + ((i) + GH))
#define FPB (2 * (NC + 1) * NC) /* face fluxes per box: [axis][face m][u] */

enum { V_PHI, V_RHS, V_RES, V_OLD, V_NE, V_NI, V_EMAG, V_RHO, V_NE0, V_NI0, V_NE1, V_NI1, V_TMP, NVAR };

struct q2 {
  double len, org[2];
  int nb, lbase, lmax, geom;
  int bct[4];
  double bcv[4];
  int nlev, nbox, cap;
  int *lev, *ij, *par, *chl, *nbr; /* chl: 4 per box; nbr: 8 directions */
  uint64_t *mort;
  int off[MAXL + 2];
  double *v[NVAR];
  double *lu;
  int *piv;
  double *flux;
  int tab_n;
  double tab_emax, *tab[3];
};

static const int pub2var[7] = {V_PHI, V_RHS, V_RES, V_NE, V_NI, V_EMAG, V_RHO};

static void die(const char *msg) {
  fprintf(stderr, "quad oracle: %s\n", msg);
  abort();
}

/* ---------------------------------------------------------------------- */
/* quadtree tables (Sec. 2.1.1)                                            */
/* ---------------------------------------------------------------------- */

static uint64_t morton2(int i, int j) {
  uint64_t key = 0;
  for (int b = 0; b < 31; ++b) {
    key |= (uint64_t)((i >> b) & 1) << (2 * b);
    key |= (uint64_t)((j >> b) & 1) << (2 * b + 1);
  }
  return key;
}

static void unmorton2(uint64_t key, int *i, int *j) {
  *i = *j = 0;
  for (int b = 0; b < 31; ++b) {
    *i |= (int)((key >> (2 * b)) & 1) << b;
    *j |= (int)((key >> (2 * b + 1)) & 1) << b;
  }
}

/* neighbour direction (dx,dy) -> 0..7, x fastest, centre skipped */
static int dir8(int dx, int dy) {
  int d = (dx + 1) + 3 * (dy + 1);
  return d < 4 ? d : d - 1;
}

/* face f = 0..3 is -x,+x,-y,+y */
static int face_axis(int f) { return f / 2; }
static int face_side(int f) { return f & 1; }
static int face8(int f) { return face_axis(f) == 0 ? dir8(face_side(f) ? 1 : -1, 0) : dir8(0, face_side(f) ? 1 : -1); }

/* box of level l at box coordinates (i,j): index, -1 outside the domain,
 * -2 inside but no box of that level there */
static int find_box(const q2 *o, int l, int i, int j) {
  int n = 1 << l;
  if (i < 0 || j < 0 || i >= n || j >= n) return -1;
  if (l >= o->nlev) return -2;
  uint64_t key = morton2(i, j);
  int lo = o->off[l], hi = o->off[l + 1] - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (o->mort[mid] == key) return mid;
    if (o->mort[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return -2;
}

static void grow(q2 *o, int need) {
  if (need <= o->cap) return;
  int cap = o->cap ? o->cap : 64;
  while (cap < need) cap *= 2;
  o->lev = realloc(o->lev, sizeof(int) * cap);
  o->ij = realloc(o->ij, sizeof(int) * 2 * cap);
  o->par = realloc(o->par, sizeof(int) * cap);
  o->chl = realloc(o->chl, sizeof(int) * 4 * cap);
  o->nbr = realloc(o->nbr, sizeof(int) * 8 * cap);
  o->mort = realloc(o->mort, sizeof(uint64_t) * cap);
  for (int v = 0; v < NVAR; ++v) {
    o->v[v] = realloc(o->v[v], sizeof(double) * BS * (size_t)cap);
    memset(o->v[v] + (size_t)BS * o->cap, 0, sizeof(double) * BS * (size_t)(cap - o->cap));
  }
  o->flux = realloc(o->flux, sizeof(double) * FPB * (size_t)cap);
  o->cap = cap;
}

static int add_box(q2 *o, int l, int i, int j, int parent) {
  grow(o, o->nbox + 1);
  int b = o->nbox++;
  o->lev[b] = l;
  o->ij[2 * b] = i;
  o->ij[2 * b + 1] = j;
  o->mort[b] = morton2(i, j);
  o->par[b] = parent;
  for (int c = 0; c < 4; ++c) o->chl[4 * b + c] = -1;
  return b;
}

static void set_neighbours(q2 *o, int l) {
  for (int b = o->off[l]; b < o->off[l + 1]; ++b)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy) continue;
        o->nbr[8 * b + dir8(dx, dy)] = find_box(o, l, o->ij[2 * b] + dx, o->ij[2 * b + 1] + dy);
      }
}

q2 *q2_create(double length, const double *origin, int nb, int max_level, int geom,
              const int *bc_type, const double *bc_val) {
  int lb = 0;
  while ((1 << lb) < nb) ++lb;
  if ((1 << lb) != nb || lb + max_level > MAXL - 1 || (geom != 0 && geom != 1)) return NULL;
  if (geom == 1 && origin && origin[0] != 0.0) return NULL; /* the axis is x = 0 */
  q2 *o = calloc(1, sizeof(q2));
  o->len = length;
  for (int d = 0; d < 2; ++d) o->org[d] = origin ? origin[d] : 0.0;
  o->nb = nb;
  o->lbase = lb;
  o->lmax = lb + max_level;
  o->geom = geom;
  for (int f = 0; f < 4; ++f) {
    o->bct[f] = bc_type[f];
    o->bcv[f] = bc_val[f];
  }
  if (geom == 1) { /* the axis: no flux, mirror ghosts */
    o->bct[0] = 0;
    o->bcv[0] = 0.0;
  }
  for (int l = 0; l <= lb; ++l) {
    o->off[l] = o->nbox;
    uint64_t n = (uint64_t)1 << (2 * l);
    for (uint64_t key = 0; key < n; ++key) {
      int i, j;
      unmorton2(key, &i, &j);
      add_box(o, l, i, j, l ? o->off[l - 1] + (int)(key >> 2) : -1);
    }
    o->off[l + 1] = o->nbox;
  }
  for (int l = 0; l < lb; ++l)
    for (int b = o->off[l]; b < o->off[l + 1]; ++b)
      for (int c = 0; c < 4; ++c) o->chl[4 * b + c] = o->off[l + 1] + (int)((o->mort[b] << 2) | (uint64_t)c);
  o->nlev = lb + 1;
  for (int l = 0; l <= lb; ++l) set_neighbours(o, l);
  return o;
}

void q2_destroy(q2 *o) {
  if (!o) return;
  free(o->lev); free(o->ij); free(o->par); free(o->chl); free(o->nbr); free(o->mort);
  for (int v = 0; v < NVAR; ++v) free(o->v[v]);
  free(o->flux); free(o->lu); free(o->piv);
  for (int t = 0; t < 3; ++t) free(o->tab[t]);
  free(o);
}

int q2_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int q2_n_boxes(const q2 *o) { return o->nbox; }
int q2_n_levels(const q2 *o) { return o->nlev; }
int q2_level_offset(const q2 *o, int l) { return (l >= 0 && l <= o->nlev) ? o->off[l] : -1; }

/* Refine the flagged boxes of the finest existing level.  Proper nesting:
 * a box is refined only if all 8 neighbour positions of its level hold a
 * box or lie outside the domain; other requests are dropped. */
int q2_refine_level(q2 *o, int l, const int8_t *flags, int *n_dropped) {
  if (l != o->nlev - 1 || l >= o->lmax) return -1;
  int dropped = 0, start = o->nbox;
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    if (flags[b - o->off[l]] <= 0) continue;
    int ok = 1;
    for (int d = 0; d < 8; ++d)
      if (o->nbr[8 * b + d] == -2) ok = 0;
    if (!ok) {
      ++dropped;
      continue;
    }
    for (int c = 0; c < 4; ++c) {
      /* add_box may move the tables: store through them only afterwards */
      int nb = add_box(o, l + 1, 2 * o->ij[2 * b] + (c & 1), 2 * o->ij[2 * b + 1] + (c >> 1), b);
      o->chl[4 * b + c] = nb;
    }
  }
  if (n_dropped) *n_dropped = dropped;
  if (o->nbox == start) return 0;
  o->off[l + 2] = o->nbox;
  o->nlev = l + 2;
  set_neighbours(o, l + 1);
  return o->nbox - start;
}

void q2_get_tables(const q2 *o, int32_t *level, int32_t *ij, uint64_t *mort, int32_t *parent,
                   int32_t *child, int32_t *nbr) {
  for (int b = 0; b < o->nbox; ++b) {
    if (level) level[b] = o->lev[b];
    if (ij) { ij[2 * b] = o->ij[2 * b]; ij[2 * b + 1] = o->ij[2 * b + 1]; }
    if (mort) mort[b] = o->mort[b];
    if (parent) parent[b] = o->par[b];
    if (child) for (int c = 0; c < 4; ++c) child[4 * b + c] = o->chl[4 * b + c];
    if (nbr) for (int d = 0; d < 8; ++d) nbr[8 * b + d] = o->nbr[8 * b + d];
  }
}

static int is_leaf(const q2 *o, int b) { return o->chl[4 * b] < 0; }
static double spacing(const q2 *o, int l) { return o->len / (NC * (double)(1 << l)); }
static double *box(const q2 *o, int var, int b) { return o->v[var] + (size_t)BS * b; }

void q2_set(q2 *o, int var, const double *src) {
  double *d = o->v[pub2var[var]];
  for (int b = 0; b < o->nbox; ++b)
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) d[(size_t)BS * b + IX(i, j)] = src[(size_t)64 * b + i + NC * j];
}

void q2_get(const q2 *o, int var, double *dst) {
  const double *s = o->v[pub2var[var]];
  for (int b = 0; b < o->nbox; ++b)
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) dst[(size_t)64 * b + i + NC * j] = s[(size_t)BS * b + IX(i, j)];
}

/* ---------------------------------------------------------------------- */
/* geometry                                                                */
/* ---------------------------------------------------------------------- */

/* Radial face weights of the cell with global x index gx: the face radius
 * over the cell-centre radius, r_{i-1/2}/r_i and r_{i+1/2}/r_i with r at
 * (index + 1/2) h from the axis; 1 in Cartesian coordinates. */
static double w_lo(const q2 *o, int gx) { return o->geom ? (double)gx / (gx + 0.5) : 1.0; }
static double w_hi(const q2 *o, int gx) { return o->geom ? (gx + 1.0) / (gx + 0.5) : 1.0; }
/* cell volume weight (proportional to the centre radius) and face area
 * weight of the face at global x position gx (in cells) */
static double w_vol(const q2 *o, int gx) { return o->geom ? gx + 0.5 : 1.0; }

/* ---------------------------------------------------------------------- */
/* ghost cells                                                              */
/* ---------------------------------------------------------------------- */

/* value at global cell g of level l; the box must exist */
static double cell_val(const q2 *o, int var, int l, const int g[2]) {
  int b = find_box(o, l, g[0] >> 3, g[1] >> 3);
  if (b < 0) die("coarse value requested where no box exists (nesting)");
  return box(o, var, b)[IX(g[0] & 7, g[1] & 7)];
}

/* physical-boundary ghost across face f of an interior value: Dirichlet g
 * at the face -> 2g - inner (homogeneous: -inner); Neumann zero and the
 * axis -> inner */
static double bc_ghost(const q2 *o, int f, double inner, int homog) {
  if (o->bct[f] == 1) return (homog ? 0.0 : 2.0 * o->bcv[f]) - inner;
  return inner;
}

static double cell_val_bc(const q2 *o, int var, int l, const int q[2], const int from[2], int homog) {
  int n = NC << l;
  for (int d = 0; d < 2; ++d) {
    if (q[d] < 0) return bc_ghost(o, 2 * d, cell_val(o, var, l, from), homog);
    if (q[d] >= n) return bc_ghost(o, 2 * d + 1, cell_val(o, var, l, from), homog);
  }
  return cell_val(o, var, l, q);
}

static double cell_val_mirror(const q2 *o, int var, int l, const int q[2], const int from[2]) {
  int n = NC << l;
  for (int d = 0; d < 2; ++d)
    if (q[d] < 0 || q[d] >= n) return cell_val(o, var, l, from);
  return cell_val(o, var, l, q);
}

/* cell at depth t from face f (t = 0 the inner layer, t < 0 ghost layers),
 * u along the face */
static void face_cell(int f, int t, int u, int c[2]) {
  int a = face_axis(f);
  c[a] = face_side(f) ? NC - 1 - t : t;
  c[1 - a] = u;
}

/* Potential ghosts, depth 1.  Same-level neighbour: copy.  Wall: as above.
 * Refinement boundary: phi_f/3 + 2 phihat/3, phihat = 3/4 c + 1/4 c_t, c the
 * coarse cell containing the ghost and c_t its tangential neighbour on the
 * ghost's side. */
static void fill_ghosts_phi(q2 *o, int var, int l, int homog) {
  BOXES_PAR
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    double *p = box(o, var, b);
    for (int f = 0; f < 4; ++f) {
      int a = face_axis(f), t = 1 - a;
      int nb = o->nbr[8 * b + face8(f)];
      for (int u = 0; u < NC; ++u) {
        int ci[2], cg[2];
        face_cell(f, 0, u, ci);
        face_cell(f, -1, u, cg);
        double inner = p[IX(ci[0], ci[1])], val;
        if (nb >= 0) {
          int cs[2];
          face_cell(f ^ 1, 0, u, cs);
          val = box(o, var, nb)[IX(cs[0], cs[1])];
        } else if (nb == -1) {
          val = bc_ghost(o, f, inner, homog);
        } else {
          int G[2], cc[2];
          for (int d = 0; d < 2; ++d) { G[d] = o->ij[2 * b + d] * NC + cg[d]; cc[d] = G[d] >> 1; }
          int qt[2] = {cc[0], cc[1]};
          qt[t] += (G[t] & 1) ? 1 : -1;
          double phat = 0.75 * cell_val(o, var, l - 1, cc) + 0.25 * cell_val_bc(o, var, l - 1, qt, cc, homog);
          val = inner / 3.0 + 2.0 * phat / 3.0;
        }
        p[IX(cg[0], cg[1])] = val;
      }
    }
  }
}

/* Density ghosts, depth 2: same-level copy, mirror at walls and the axis,
 * and at refinement boundaries the prolongation (2c + c_x + c_y)/4 of the
 * coarse cell containing the ghost, limited to 2c. */
static void fill_ghosts_density(q2 *o, int var, int l) {
  BOXES_PAR
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    double *p = box(o, var, b);
    for (int f = 0; f < 4; ++f) {
      int nb = o->nbr[8 * b + face8(f)];
      for (int t = 1; t <= 2; ++t)
        for (int u = 0; u < NC; ++u) {
          int cg[2];
          face_cell(f, -t, u, cg);
          double val;
          if (nb >= 0) {
            int cs[2];
            face_cell(f ^ 1, t - 1, u, cs);
            val = box(o, var, nb)[IX(cs[0], cs[1])];
          } else if (nb == -1) {
            int cm[2];
            face_cell(f, t - 1, u, cm);
            val = p[IX(cm[0], cm[1])];
          } else {
            int G[2], cc[2];
            for (int d = 0; d < 2; ++d) { G[d] = o->ij[2 * b + d] * NC + cg[d]; cc[d] = G[d] >> 1; }
            double c = cell_val(o, var, l - 1, cc), sum = 2.0 * c;
            for (int d = 0; d < 2; ++d) {
              int q[2] = {cc[0], cc[1]};
              q[d] += (G[d] & 1) ? 1 : -1;
              sum += cell_val_mirror(o, var, l - 1, q, cc);
            }
            val = 0.25 * sum;
            if (val > 2.0 * c) val = 2.0 * c;
          }
          p[IX(cg[0], cg[1])] = val;
        }
    }
  }
}

/* |E| ghosts, depth 1: same-level copy, the inner value at walls, the
 * coarse cell containing the ghost at refinement boundaries */
static void fill_ghosts_emag(q2 *o, int l) {
  BOXES_PAR
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    double *p = box(o, V_EMAG, b);
    for (int f = 0; f < 4; ++f) {
      int nb = o->nbr[8 * b + face8(f)];
      for (int u = 0; u < NC; ++u) {
        int ci[2], cg[2];
        face_cell(f, 0, u, ci);
        face_cell(f, -1, u, cg);
        double val;
        if (nb >= 0) {
          int cs[2];
          face_cell(f ^ 1, 0, u, cs);
          val = box(o, V_EMAG, nb)[IX(cs[0], cs[1])];
        } else if (nb == -1) {
          val = p[IX(ci[0], ci[1])];
        } else {
          int cc[2];
          for (int d = 0; d < 2; ++d) cc[d] = (o->ij[2 * b + d] * NC + cg[d]) >> 1;
          val = cell_val(o, V_EMAG, l - 1, cc);
        }
        p[IX(cg[0], cg[1])] = val;
      }
    }
  }
}

/* ---------------------------------------------------------------------- */
/* multigrid (Sec. 2.1.2)                                                  */
/* ---------------------------------------------------------------------- */

/* L phi at cell (i,j) of box b (ghosts filled): the five-point operator,
 * radial terms weighted by the face radii over the centre radius in
 * cylindrical coordinates */
static double lap(const q2 *o, const double *p, int b, int i, int j, double h2) {
  int gx = o->ij[2 * b] * NC + i;
  double c = p[IX(i, j)];
  return (w_lo(o, gx) * (p[IX(i - 1, j)] - c) + w_hi(o, gx) * (p[IX(i + 1, j)] - c) +
          (p[IX(i, j - 1)] - c) + (p[IX(i, j + 1)] - c)) / h2;
}

/* Gauss-Seidel red-black: red = (i+j) even in level-global indices.
 * phi = (w_lo phi_W + w_hi phi_E + phi_S + phi_N - h^2 f) / (w_lo + w_hi + 2) */
static void smooth(q2 *o, int l, int nu) {
  double h2 = spacing(o, l) * spacing(o, l);
  for (int s = 0; s < nu; ++s)
    for (int color = 0; color < 2; ++color) {
      fill_ghosts_phi(o, V_PHI, l, 0);
      BOXES_PAR
      for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
        double *p = box(o, V_PHI, b), *f = box(o, V_RHS, b);
        for (int j = 0; j < NC; ++j)
          for (int i = 0; i < NC; ++i) {
            if (((i + j) & 1) != color) continue;
            int gx = o->ij[2 * b] * NC + i;
            double wl = w_lo(o, gx), wh = w_hi(o, gx);
            p[IX(i, j)] = (wl * p[IX(i - 1, j)] + wh * p[IX(i + 1, j)] + p[IX(i, j - 1)] + p[IX(i, j + 1)] -
                           h2 * f[IX(i, j)]) / (wl + wh + 2.0);
          }
      }
    }
}

static void residual_box(q2 *o, int var_phi, int b, double *r) {
  double h2 = spacing(o, o->lev[b]) * spacing(o, o->lev[b]);
  double *p = box(o, var_phi, b), *f = box(o, V_RHS, b);
  for (int j = 0; j < NC; ++j)
    for (int i = 0; i < NC; ++i) r[IX(i, j)] = f[IX(i, j)] - lap(o, p, b, i, j, h2);
}

/* mean of the four children (cell-centred full weighting); in cylindrical
 * coordinates weighted by the cell volumes (the centre radii) */
static void restrict_level(q2 *o, int l, int src, int dst) {
  BOXES_PAR
  for (int pb = o->off[l - 1]; pb < o->off[l]; ++pb) {
    if (is_leaf(o, pb)) continue;
    double *d = box(o, dst, pb);
    for (int J = 0; J < NC; ++J)
      for (int I = 0; I < NC; ++I) {
        int c = (I >> 2) + 2 * (J >> 2), cb = o->chl[4 * pb + c];
        const double *s = box(o, src, cb);
        int i0 = 2 * (I & 3), j0 = 2 * (J & 3);
        double sum = 0.0, wsum = 0.0;
        for (int dj = 0; dj < 2; ++dj)
          for (int di = 0; di < 2; ++di) {
            double w = w_vol(o, o->ij[2 * cb] * NC + i0 + di);
            sum += w * s[IX(i0 + di, j0 + dj)];
            wsum += w;
          }
        d[IX(I, J)] = sum / wsum;
      }
  }
}

/* linear prolongation of level l-1 to each cell of each level-l box:
 * (2c + c_sx + c_sy)/4, c the parent cell, c_sd its neighbour in the
 * direction of the fine cell's offset; add = 1 adds (correction) */
static void prolong_level(q2 *o, int l, int src, int dst, int homog, int add) {
  BOXES_PAR
  for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
    double *d = box(o, dst, b);
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) {
        int G[2] = {o->ij[2 * b] * NC + i, o->ij[2 * b + 1] * NC + j};
        int cc[2] = {G[0] >> 1, G[1] >> 1};
        double sum = 2.0 * cell_val(o, src, l - 1, cc);
        for (int e = 0; e < 2; ++e) {
          int q[2] = {cc[0], cc[1]};
          q[e] += (G[e] & 1) ? 1 : -1;
          sum += cell_val_bc(o, src, l - 1, q, cc, homog);
        }
        if (add) d[IX(i, j)] += 0.25 * sum;
        else d[IX(i, j)] = 0.25 * sum;
      }
  }
}

/* Exact solve on level 0 (one box): the operator's matrix, column k being
 * L applied to the k-th unit vector with homogeneous ghosts, by dense LU
 * with partial pivoting; the boundary values enter as f - L(0). */
static void coarse_factor(q2 *o) {
  const int n = 64;
  double h2 = spacing(o, 0) * spacing(o, 0);
  o->lu = calloc((size_t)n * n, sizeof(double));
  o->piv = calloc(n, sizeof(int));
  double *A = o->lu, *t = box(o, V_TMP, 0);
  for (int k = 0; k < n; ++k) {
    memset(t, 0, sizeof(double) * BS);
    t[IX(k % NC, k / NC)] = 1.0;
    fill_ghosts_phi(o, V_TMP, 0, 1);
    for (int r = 0; r < n; ++r) A[(size_t)r * n + k] = lap(o, t, 0, r % NC, r / NC, h2);
  }
  for (int col = 0; col < n; ++col) {
    int p = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(A[(size_t)r * n + col]) > fabs(A[(size_t)p * n + col])) p = r;
    o->piv[col] = p;
    if (p != col)
      for (int c = 0; c < n; ++c) {
        double s = A[(size_t)col * n + c];
        A[(size_t)col * n + c] = A[(size_t)p * n + c];
        A[(size_t)p * n + c] = s;
      }
    for (int r = col + 1; r < n; ++r) {
      double m = A[(size_t)r * n + col] / A[(size_t)col * n + col];
      A[(size_t)r * n + col] = m;
      for (int c = col + 1; c < n; ++c) A[(size_t)r * n + c] -= m * A[(size_t)col * n + c];
    }
  }
}

void q2_coarse_solve(q2 *o) {
  const int n = 64;
  if (!o->lu) coarse_factor(o);
  double h2 = spacing(o, 0) * spacing(o, 0);
  double x[64];
  double *t = box(o, V_TMP, 0), *f = box(o, V_RHS, 0), *p = box(o, V_PHI, 0);
  memset(t, 0, sizeof(double) * BS);
  fill_ghosts_phi(o, V_TMP, 0, 0);
  for (int r = 0; r < n; ++r) x[r] = f[IX(r % NC, r / NC)] - lap(o, t, 0, r % NC, r / NC, h2);
  for (int r = 0; r < n; ++r) {
    double s = x[r]; x[r] = x[o->piv[r]]; x[o->piv[r]] = s;
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < r; ++c) x[r] -= o->lu[(size_t)r * n + c] * x[c];
  for (int r = n - 1; r >= 0; --r) {
    for (int c = r + 1; c < n; ++c) x[r] -= o->lu[(size_t)r * n + c] * x[c];
    x[r] /= o->lu[(size_t)r * n + r];
  }
  for (int r = 0; r < n; ++r) p[IX(r % NC, r / NC)] = x[r];
}

/* FAS V-cycle with top level `top`, the steps of the 3-D cycle */
static void vcycle(q2 *o, int top, int nu1, int nu2) {
  for (int l = top; l >= 1; --l) {
    smooth(o, l, nu1);
    fill_ghosts_phi(o, V_PHI, l, 0);
    BOXES_PAR
    for (int b = o->off[l]; b < o->off[l + 1]; ++b) residual_box(o, V_PHI, b, box(o, V_RES, b));
    restrict_level(o, l, V_PHI, V_PHI);
    BOXES_PAR
    for (int b = o->off[l - 1]; b < o->off[l]; ++b) memcpy(box(o, V_OLD, b), box(o, V_PHI, b), sizeof(double) * BS);
    restrict_level(o, l, V_RES, V_RHS);
    fill_ghosts_phi(o, V_PHI, l - 1, 0);
    double h2 = spacing(o, l - 1) * spacing(o, l - 1);
    BOXES_PAR
    for (int b = o->off[l - 1]; b < o->off[l]; ++b) {
      if (is_leaf(o, b)) continue;
      double *p = box(o, V_PHI, b), *f = box(o, V_RHS, b);
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i) f[IX(i, j)] += lap(o, p, b, i, j, h2);
    }
  }
  q2_coarse_solve(o);
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
static double leaf_resmax(q2 *o, int var_phi, int top) {
  double m = 0.0;
  for (int l = 0; l <= top; ++l) {
    fill_ghosts_phi(o, var_phi, l, 0);
#pragma omp parallel for schedule(static) reduction(max : m)
    for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
      if (!is_leaf(o, b) && l != top) continue;
      double r[BS];
      residual_box(o, var_phi, b, r);
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i) {
          double a = fabs(r[IX(i, j)]);
          if (a > m) m = a;
        }
    }
  }
  return m;
}

double q2_rel_residual(q2 *o) {
  int top = o->nlev - 1;
  double num = leaf_resmax(o, V_PHI, top);
  memset(o->v[V_TMP], 0, sizeof(double) * BS * (size_t)o->nbox);
  double den = leaf_resmax(o, V_TMP, top);
  return den > 0.0 ? num / den : num;
}

int q2_vcycles(q2 *o, int n, int nu1, int nu2, double *rel) {
  for (int c = 0; c < n; ++c) vcycle(o, o->nlev - 1, nu1, nu2);
  if (rel) *rel = q2_rel_residual(o);
  return 0;
}

int q2_solve(q2 *o, double tol, int max_cycles, int nu1, int nu2, double *rel, int *cycles) {
  double r = 0.0;
  int c = 0;
  do {
    vcycle(o, o->nlev - 1, nu1, nu2);
    ++c;
    r = q2_rel_residual(o);
  } while (r > tol && c < max_cycles);
  if (rel) *rel = r;
  if (cycles) *cycles = c;
  return r <= tol ? 0 : -4;
}

/* Full multigrid: restrict f to every refined box, solve on level 0, then
 * per finer level prolong the solution and one V-cycle with that level on
 * top; then V-cycles on the full hierarchy to the tolerance */
int q2_fmg(q2 *o, double tol, int max_cycles, int nu1, int nu2, double *rel, int *cycles) {
  int top = o->nlev - 1;
  for (int l = top; l >= 1; --l) restrict_level(o, l, V_RHS, V_RHS);
  q2_coarse_solve(o);
  for (int l = 1; l <= top; ++l) {
    prolong_level(o, l, V_PHI, V_PHI, 0, 0);
    vcycle(o, l, nu1, nu2);
  }
  int c = 1;
  double r = q2_rel_residual(o);
  while (r > tol && c < max_cycles) {
    vcycle(o, top, nu1, nu2);
    ++c;
    r = q2_rel_residual(o);
  }
  if (rel) *rel = r;
  if (cycles) *cycles = c;
  return r <= tol ? 0 : -4;
}

/* every refined box := restriction of its children, finest level first */
void q2_restrict_all(q2 *o, int var) {
  for (int l = o->nlev - 1; l >= 1; --l) restrict_level(o, l, pub2var[var], pub2var[var]);
}

/* leaf residual with every refined box holding the restriction of its
 * children (the composite-grid operator applied to the leaf values) */
void q2_composite_residual(q2 *o) {
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
void q2_charge_rhs(q2 *o, double q, double eps, int use_rho) {
  BOXES_PAR
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    double *f = box(o, V_RHS, b), *ne = box(o, V_NE, b), *ni = box(o, V_NI, b), *rho = box(o, V_RHO, b);
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) {
        int c = IX(i, j);
        f[c] = use_rho ? -rho[c] / eps : -q * (ni[c] - ne[c]) / eps;
      }
  }
}

/* ---------------------------------------------------------------------- */
/* field (Sec. 2.3)                                                        */
/* ---------------------------------------------------------------------- */

/* face field (phi_i - phi_{i+1})/dx; cell component the mean of its two
 * faces; |E| the root of the sum of squares.  Leaf cells only. */
static void cell_field(const double *p, int i, int j, double h, double e[2]) {
  e[0] = ((p[IX(i - 1, j)] - p[IX(i, j)]) / h + (p[IX(i, j)] - p[IX(i + 1, j)]) / h) / 2.0;
  e[1] = ((p[IX(i, j - 1)] - p[IX(i, j)]) / h + (p[IX(i, j)] - p[IX(i, j + 1)]) / h) / 2.0;
}

void q2_compute_field(q2 *o) {
  for (int l = 0; l < o->nlev; ++l) {
    fill_ghosts_phi(o, V_PHI, l, 0);
    double h = spacing(o, l);
    BOXES_PAR
    for (int b = o->off[l]; b < o->off[l + 1]; ++b) {
      double *p = box(o, V_PHI, b), *em = box(o, V_EMAG, b);
      for (int j = 0; j < NC; ++j)
        for (int i = 0; i < NC; ++i) {
          if (!is_leaf(o, b)) {
            em[IX(i, j)] = 0.0;
            continue;
          }
          double e[2];
          cell_field(p, i, j, h, e);
          em[IX(i, j)] = sqrt(e[0] * e[0] + e[1] * e[1]);
        }
    }
  }
}

/* ---------------------------------------------------------------------- */
/* fluid step (Sec. 2.2-2.4)                                               */
/* ---------------------------------------------------------------------- */

void q2_set_table(q2 *o, int n, double e_max, const double *mu, const double *diff,
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
static double lookup(const q2 *o, int which, double e) {
  const double *t = o->tab[which];
  int n = o->tab_n;
  double x = e / (o->tab_emax / (n - 1));
  if (x <= 0.0) return t[0];
  if (x >= n - 1) return t[n - 1];
  int i = (int)x;
  double w = x - i;
  return t[i] + w * (t[i + 1] - t[i]);
}

double q2_lookup(const q2 *o, int which, double e) { return lookup(o, which, e); }

/* psi(a/b) b of the Koren limiter, psi(x) = max(0, min(1, (2+x)/6, x))
 * (Eq. 7), in the division-free form */
static double koren(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  double s = b > 0.0 ? 1.0 : -1.0;
  double aa = fabs(a), bb = fabs(b);
  double m = bb;
  if ((2.0 * bb + aa) / 6.0 < m) m = (2.0 * bb + aa) / 6.0;
  if (aa < m) m = aa;
  return s * m;
}

double q2_koren(double a, double b) { return koren(a, b); }

static double *fluxp(q2 *o, int b, int a) { return o->flux + (size_t)b * FPB + (size_t)a * (NC + 1) * NC; }

/* Face fluxes of every leaf box, index [a][m][u]: m = 0..8 the face between
 * cells m-1 and m along axis a, u the coordinate along the other axis.
 * Advective part by Eq. 6 (v < 0) or Eq. 7 (v >= 0) with v = -mu(E*)
 * E_face, E* the mean of the two cell |E|; diffusive part
 * -D(E*) (n_R - n_L)/dx. */
static void leaf_fluxes(q2 *o, int var_n) {
  BOXES_PAR
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    double h = spacing(o, o->lev[b]);
    const double *n = box(o, var_n, b), *p = box(o, V_PHI, b), *em = box(o, V_EMAG, b);
    for (int a = 0; a < 2; ++a) {
      double *F = fluxp(o, b, a);
      for (int m = 0; m <= NC; ++m)
        for (int u = 0; u < NC; ++u) {
          int c[4][2];
          for (int s = 0; s < 4; ++s) {
            c[s][a] = m - 2 + s;
            c[s][1 - a] = u;
          }
          double nL2 = n[IX(c[0][0], c[0][1])], nL = n[IX(c[1][0], c[1][1])];
          double nR = n[IX(c[2][0], c[2][1])], nR2 = n[IX(c[3][0], c[3][1])];
          double pL = p[IX(c[1][0], c[1][1])], pR = p[IX(c[2][0], c[2][1])];
          double eL = em[IX(c[1][0], c[1][1])], eR = em[IX(c[2][0], c[2][1])];
          double e_face = (pL - pR) / h, e_star = (eL + eR) / 2.0;
          double mu = lookup(o, 0, e_star), dc = lookup(o, 1, e_star);
          double v = -mu * e_face, nf;
          if (v < 0.0) nf = nR - koren(nR2 - nR, nR - nL);
          else nf = nL + koren(nL - nL2, nR - nL);
          F[m * NC + u] = v * nf - dc * (nR - nL) / h;
        }
    }
  }
  /* refinement boundaries: a coarse leaf face next to a refined box takes
   * the area-weighted mean of the two fine face fluxes (conservation; the
   * face area is proportional to the radius of the face centre in
   * cylindrical coordinates) */
  BOXES_PAR
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    for (int f = 0; f < 4; ++f) {
      int nb = o->nbr[8 * b + face8(f)];
      if (nb < 0 || is_leaf(o, nb)) continue;
      int a = face_axis(f), side = face_side(f);
      double *F = fluxp(o, b, a);
      for (int u = 0; u < NC; ++u) {
        int cidx[2];
        cidx[a] = side ? 0 : 1;
        cidx[1 - a] = u >> 2;
        int ch = o->chl[4 * nb + cidx[0] + 2 * cidx[1]];
        const double *Fc = fluxp(o, ch, a);
        int mc = side ? 0 : NC;
        double s = 0.0, ws = 0.0;
        for (int du = 0; du < 2; ++du) {
          int uf = 2 * (u & 3) + du;
          /* faces normal to x share one radius; faces normal to y are
           * weighted by the radius of their centres */
          double w = a == 0 ? 1.0 : w_vol(o, o->ij[2 * ch] * NC + uf);
          s += w * Fc[mc * NC + uf];
          ws += w;
        }
        F[(side ? NC : 0) * NC + u] = s / ws;
      }
    }
  }
}

static void restrict_densities(q2 *o, int ne, int ni) {
  for (int l = o->nlev - 1; l >= 1; --l) {
    restrict_level(o, l, ne, ne);
    restrict_level(o, l, ni, ni);
  }
}

/* One forward Euler step dst = src + dt F(src) (Eq. 2-3) on leaf cells: the
 * divergence of the face fluxes (radial faces weighted by their radius over
 * the cell-centre radius in cylindrical coordinates) and the source
 * alpha mu |E| n_e; then refined boxes get the restriction of their
 * children. */
static void euler_stage(q2 *o, int sne, int sni, int dne, int dni, double dt) {
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
    const double *Fx = fluxp(o, b, 0), *Fy = fluxp(o, b, 1);
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) {
        int gx = o->ij[2 * b] * NC + i;
        double div = (w_hi(o, gx) * Fx[(i + 1) * NC + j] - w_lo(o, gx) * Fx[i * NC + j]) / h +
                     (Fy[(j + 1) * NC + i] - Fy[j * NC + i]) / h;
        double e = em[IX(i, j)];
        double src = lookup(o, 2, e) * lookup(o, 0, e) * e * ne[IX(i, j)];
        one[IX(i, j)] = ne[IX(i, j)] - dt * div + dt * src;
        oni[IX(i, j)] = ni[IX(i, j)] + dt * src;
      }
  }
  restrict_densities(o, dne, dni);
}

void q2_fluid_stage(q2 *o, double dt) {
  restrict_densities(o, V_NE, V_NI);
  euler_stage(o, V_NE, V_NI, V_NE1, V_NI1, dt);
  memcpy(o->v[V_NE], o->v[V_NE1], sizeof(double) * BS * (size_t)o->nbox);
  memcpy(o->v[V_NI], o->v[V_NI1], sizeof(double) * BS * (size_t)o->nbox);
}

/* Time-step limits of Sec. 2.4 in two dimensions: CFL 0.5 on sum |v_d|/dx,
 * advection + diffusion (sum |v_d|/dx + 2*2*D/dx^2) below 1, dielectric
 * relaxation eps/(e mu n_e); times the safety 0.9. */
double q2_dt_limit(q2 *o, double q, double eps) {
  double m_adv = 0.0, m_ad = 0.0, m_drt = 0.0;
  for (int l = 0; l < o->nlev; ++l) fill_ghosts_phi(o, V_PHI, l, 0);
#pragma omp parallel for schedule(static) reduction(max : m_adv, m_ad, m_drt)
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    double h = spacing(o, o->lev[b]);
    const double *p = box(o, V_PHI, b), *em = box(o, V_EMAG, b), *ne = box(o, V_NE, b);
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) {
        double e[2];
        cell_field(p, i, j, h, e);
        double mu = lookup(o, 0, em[IX(i, j)]), dc = lookup(o, 1, em[IX(i, j)]);
        double adv = (fabs(mu * e[0]) + fabs(mu * e[1])) / h;
        double ad = adv + 2.0 * 2.0 * dc / (h * h);
        double drt = mu * ne[IX(i, j)];
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

/* Explicit trapezoidal (Heun) step of Sec. 2.4, as in 3-D: keep n0; Euler
 * to n1; new field; Euler from n1 to n2; n = (n0 + n2)/2; new field.  The
 * next time step is evaluated at the second stage. */
int q2_advance(q2 *o, double dt, double q, double eps, double tol, int max_cycles, int nu1,
               int nu2, double *dt_next, int *cycles1, int *cycles2) {
  size_t bytes = sizeof(double) * BS * (size_t)o->nbox;
  restrict_densities(o, V_NE, V_NI);
  memcpy(o->v[V_NE0], o->v[V_NE], bytes);
  memcpy(o->v[V_NI0], o->v[V_NI], bytes);
  euler_stage(o, V_NE0, V_NI0, V_NE, V_NI, dt);
  q2_charge_rhs(o, q, eps, 0);
  int st = q2_solve(o, tol, max_cycles, nu1, nu2, NULL, cycles1);
  q2_compute_field(o);
  if (dt_next) *dt_next = q2_dt_limit(o, q, eps);
  euler_stage(o, V_NE, V_NI, V_NE1, V_NI1, dt);
  for (size_t c = 0; c < (size_t)BS * o->nbox; ++c) {
    o->v[V_NE][c] = (o->v[V_NE0][c] + o->v[V_NE1][c]) / 2.0;
    o->v[V_NI][c] = (o->v[V_NI0][c] + o->v[V_NI1][c]) / 2.0;
  }
  q2_charge_rhs(o, q, eps, 0);
  int st2 = q2_solve(o, tol, max_cycles, nu1, nu2, NULL, cycles2);
  q2_compute_field(o);
  return st ? st : st2;
}

/* ---------------------------------------------------------------------- */
/* refinement criterion and regridding (Sec. 2.5, Eq. 8) in two dimensions */
/* ---------------------------------------------------------------------- */

/* As in 3-D: a cell needs refinement where alpha(c1 |E|) dx >= c0 c1 (Eq. 8
 * fails).  A leaf box is flagged +1 when one of its cells needs it, or a
 * needing cell of a same-level leaf neighbour (one of the 8) lies within
 * `buffer` cells of it (Chebyshev distance in cells of that level), and its
 * level is below the maximum.  A leaf above the base grid that is not
 * flagged is derefinable (-1) when every cell has alpha(c1 |E|) dx <
 * c0_deref c1 and dx < dx_deref.  Uses the stored |E| of the leaf cells. */
void q2_refine_flags(q2 *o, double c0, double c1, double c0_deref, double dx_deref, int buffer,
                     int8_t *flags) {
  unsigned char *need = calloc((size_t)64 * o->nbox, 1);
  unsigned char *any = calloc((size_t)o->nbox, 1), *fine = calloc((size_t)o->nbox, 1);
  for (int b = 0; b < o->nbox; ++b) {
    flags[b] = 0;
    if (!is_leaf(o, b)) continue;
    double dx = spacing(o, o->lev[b]);
    const double *em = box(o, V_EMAG, b);
    int ok = dx < dx_deref;
    for (int j = 0; j < NC; ++j)
      for (int i = 0; i < NC; ++i) {
        double a = lookup(o, 2, c1 * em[IX(i, j)]);
        if (a * dx >= c0 * c1) {
          need[(size_t)64 * b + i + 8 * j] = 1;
          any[b] = 1;
        }
        if (!(a * dx < c0_deref * c1)) ok = 0;
      }
    fine[b] = (unsigned char)ok;
  }
  for (int b = 0; b < o->nbox; ++b) {
    if (!is_leaf(o, b)) continue;
    int marked = any[b];
    for (int d = 0; d < 8 && !marked; ++d) {
      int n = o->nbr[8 * b + d];
      if (n < 0 || !is_leaf(o, n) || !any[n]) continue;
      for (int c = 0; c < 64 && !marked; ++c) {
        if (!need[(size_t)64 * n + c]) continue;
        int g[2] = {o->ij[2 * n] * NC + (c & 7), o->ij[2 * n + 1] * NC + (c >> 3)};
        int dist = 0;
        for (int e = 0; e < 2; ++e) {
          int lo = o->ij[2 * b + e] * NC, hi = lo + NC - 1;
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
  free(need);
  free(any);
  free(fine);
}

typedef struct {
  int lev, i, j, src;
  uint64_t key;
} q2_ent;

static int ent_cmp(const void *pa, const void *pb) {
  const q2_ent *a = pa, *b = pb;
  if (a->lev != b->lev) return a->lev < b->lev ? -1 : 1;
  return a->key < b->key ? -1 : (a->key > b->key ? 1 : 0);
}

/* Apply per-box flags (+1 refine, -1 derefine, leaves only), as in 3-D:
 * refinement of a flagged leaf below the maximum level when all 8 neighbour
 * positions of its level hold a box or lie outside the domain, otherwise
 * dropped; a box whose 4 children are all leaves flagged -1 loses them,
 * unless a neighbour of one of the children (not a sibling) has children or
 * is refined in this call.  Rebuilt in (level, Morton) order; kept boxes
 * keep all their data; new children get the potential by the prolongation
 * (2c + c_sx + c_sy)/4 of their parent's cells and the densities by the
 * same prolongation limited to 2c (mirror ghosts at walls and the axis),
 * every other variable zero.  Densities are restricted first. */
int q2_regrid(q2 *o, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped) {
  restrict_densities(o, V_NE, V_NI);
  int nb0 = o->nbox;
  unsigned char *ref = calloc((size_t)nb0, 1), *der = calloc((size_t)nb0, 1);
  int nref = 0, nder = 0, ndrop = 0;
  for (int b = 0; b < nb0; ++b) {
    if (!is_leaf(o, b) || flags[b] <= 0 || o->lev[b] >= o->lmax) continue;
    int ok = 1;
    for (int d = 0; d < 8; ++d)
      if (o->nbr[8 * b + d] == -2) ok = 0;
    if (ok) {
      ref[b] = 1;
      ++nref;
    } else {
      ++ndrop;
    }
  }
  for (int p = 0; p < nb0; ++p) {
    if (is_leaf(o, p)) continue;
    int ok = 1;
    for (int c = 0; c < 4 && ok; ++c) {
      int ch = o->chl[4 * p + c];
      if (!is_leaf(o, ch) || flags[ch] >= 0) ok = 0;
    }
    for (int c = 0; c < 4 && ok; ++c) {
      int ch = o->chl[4 * p + c];
      for (int d = 0; d < 8 && ok; ++d) {
        int n = o->nbr[8 * ch + d];
        if (n >= 0 && o->par[n] != p && (!is_leaf(o, n) || ref[n])) ok = 0;
      }
    }
    if (ok) {
      der[p] = 1;
      ++nder;
    }
  }
  int nnew = 0;
  q2_ent *e = malloc(sizeof(q2_ent) * (size_t)(nb0 + 4 * nref));
  double *pro = malloc(sizeof(double) * 3 * 64 * (size_t)(4 * nref + 1));
  int npro = 0;
  for (int b = 0; b < nb0; ++b) {
    if (o->par[b] >= 0 && der[o->par[b]]) continue;
    q2_ent x = {o->lev[b], o->ij[2 * b], o->ij[2 * b + 1], b, o->mort[b]};
    e[nnew++] = x;
    if (!ref[b]) continue;
    int l = o->lev[b];
    for (int c = 0; c < 4; ++c) {
      int ci = 2 * o->ij[2 * b] + (c & 1), cj = 2 * o->ij[2 * b + 1] + (c >> 1);
      q2_ent y = {l + 1, ci, cj, -1 - npro, morton2(ci, cj)};
      e[nnew++] = y;
      double *dst = pro + (size_t)3 * 64 * npro;
      const int vars[3] = {V_PHI, V_NE, V_NI};
      for (int v = 0; v < 3; ++v)
        for (int jj = 0; jj < NC; ++jj)
          for (int ii = 0; ii < NC; ++ii) {
            int G[2] = {ci * NC + ii, cj * NC + jj};
            int cc[2] = {G[0] >> 1, G[1] >> 1};
            double cval = cell_val(o, vars[v], l, cc), sum = 2.0 * cval;
            for (int a = 0; a < 2; ++a) {
              int q[2] = {cc[0], cc[1]};
              q[a] += (G[a] & 1) ? 1 : -1;
              sum += v == 0 ? cell_val_bc(o, vars[v], l, q, cc, 0) : cell_val_mirror(o, vars[v], l, q, cc);
            }
            double val = 0.25 * sum;
            if (v > 0 && val > 2.0 * cval) val = 2.0 * cval;
            dst[(size_t)64 * v + ii + 8 * jj] = val;
          }
      ++npro;
    }
  }
  qsort(e, (size_t)nnew, sizeof(q2_ent), ent_cmp);
  int cap = o->cap > nnew ? o->cap : nnew;
  int *lev = malloc(sizeof(int) * cap), *ij = malloc(sizeof(int) * 2 * cap);
  int *par = malloc(sizeof(int) * cap), *chl = malloc(sizeof(int) * 4 * cap);
  int *nbr = malloc(sizeof(int) * 8 * cap);
  uint64_t *mort = malloc(sizeof(uint64_t) * cap);
  double *nv[NVAR];
  for (int v = 0; v < NVAR; ++v) nv[v] = calloc((size_t)BS * cap, sizeof(double));
  for (int b = 0; b < nnew; ++b) {
    lev[b] = e[b].lev;
    ij[2 * b] = e[b].i;
    ij[2 * b + 1] = e[b].j;
    mort[b] = e[b].key;
    if (e[b].src >= 0) {
      for (int v = 0; v < NVAR; ++v)
        memcpy(nv[v] + (size_t)BS * b, o->v[v] + (size_t)BS * e[b].src, sizeof(double) * BS);
    } else {
      const double *src = pro + (size_t)3 * 64 * (-1 - e[b].src);
      const int vars[3] = {V_PHI, V_NE, V_NI};
      for (int v = 0; v < 3; ++v)
        for (int c = 0; c < 64; ++c) nv[vars[v]][(size_t)BS * b + IX(c & 7, c >> 3)] = src[(size_t)64 * v + c];
    }
  }
  free(o->lev); free(o->ij); free(o->par); free(o->chl); free(o->nbr); free(o->mort);
  for (int v = 0; v < NVAR; ++v) {
    free(o->v[v]);
    o->v[v] = nv[v];
  }
  o->lev = lev; o->ij = ij; o->par = par; o->chl = chl; o->nbr = nbr; o->mort = mort;
  if (cap > o->cap) o->flux = realloc(o->flux, sizeof(double) * FPB * (size_t)cap);
  o->cap = cap;
  o->nbox = nnew;
  int nlev = 0;
  for (int b = 0; b < nnew; ++b)
    if (lev[b] + 1 > nlev) nlev = lev[b] + 1;
  o->nlev = nlev;
  for (int l = 0, b = 0; l <= nlev; ++l) {
    while (b < nnew && lev[b] < l) ++b;
    o->off[l] = b;
  }
  for (int l = nlev + 1; l <= MAXL + 1; ++l) o->off[l] = nnew;
  for (int b = 0; b < nnew; ++b) {
    par[b] = lev[b] ? find_box(o, lev[b] - 1, ij[2 * b] >> 1, ij[2 * b + 1] >> 1) : -1;
    for (int c = 0; c < 4; ++c)
      chl[4 * b + c] = lev[b] + 1 < nlev ? find_box(o, lev[b] + 1, 2 * ij[2 * b] + (c & 1), 2 * ij[2 * b + 1] + (c >> 1))
                                         : -2;
    if (chl[4 * b] < 0)
      for (int c = 0; c < 4; ++c) chl[4 * b + c] = -1;
  }
  for (int l = 0; l < nlev; ++l) set_neighbours(o, l);
  free(e); free(pro); free(ref); free(der);
  if (n_refined) *n_refined = nref;
  if (n_derefined) *n_derefined = nder;
  if (n_dropped) *n_dropped = ndrop;
  return nref + nder;
}
