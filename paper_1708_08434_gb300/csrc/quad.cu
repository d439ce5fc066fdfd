// quad.cu -- 2-D and axisymmetric variants (arXiv:1708.08434, Sec. 1 and
// 2.1.1: quadtree grids; Sec. 2.1.2 multigrid; Sec. 2.2-2.4 fluid step) on a
// quadtree of 8^2-cell boxes, in Cartesian (x, y) or cylindrical (r, z)
// coordinates.
//
// The initial mesh's tables are built by host C++ (proper nesting, Morton
// order per level) and copied into the arena; a regrid forms the new box set
// and its tables on the device (k_qrg_*) and the host keeps a copy of them
// for its own queries.  Every field operation runs in the kernels below,
// one warp per box: the box and the ghost layer a kernel needs are staged in
// shared memory, with coarse values at refinement boundaries read through
// the parent's 8-neighbour table (proper nesting guarantees every coarse
// cell a ghost or a prolongation needs lies in the parent or one of its
// neighbours).
//
// Discretisation (the paper gives no 2-D or cylindrical formulas; these are
// the finite-volume forms of the 3-D rules):
//   L phi = [w_lo (phi_W - phi) + w_hi (phi_E - phi) + (phi_S - phi) + (phi_N - phi)] / h^2
// with w_lo = r_{i-1/2}/r_i, w_hi = r_{i+1/2}/r_i in cylindrical coordinates
// (r at (index + 1/2) h from the axis, so w_lo = 0 on the axis) and 1 in
// Cartesian; red-black Gauss-Seidel solves the cell's row of that operator;
// restriction is the volume-weighted mean of the four children (weights
// proportional to the centre radius); prolongation (2c + c_x + c_y)/4;
// coarse-fine potential ghost phi_f/3 + 2 phihat/3, phihat = 3/4 c + 1/4 c_t;
// fluxes as in 3-D with the radial divergence weighted like L and the
// coarse flux at a refinement boundary the area-weighted mean of the two
// fine fluxes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "sm_quad.h"
#include "sm_nvtx.h"

namespace {

constexpr int QN = 8;            // cells per box side
constexpr int QC = QN * QN;      // cells per box
constexpr int WPB = 4;           // boxes (warps) per block
constexpr int QT = 32 * WPB;     // threads per block
constexpr int QMAXL = SM_MAX_LEVELS;
constexpr int S1 = QN + 2;       // staged side with one ghost layer
constexpr int S2 = QN + 4;       // staged side with two ghost layers

// fields in the arena: the public sm_var numbering first
enum { V_PHI = 0, V_RHS, V_RES, V_NE, V_NI, V_EMAG, V_RHO, V_OLD, V_TMP, V_NE0, V_NI0, V_NE1, V_NI1, NV };

struct QBc {
  int type[4];      // 0 Neumann zero (and the axis), 1 Dirichlet
  double g2[4];     // 2 g
};

struct QTabs {
  const int *lev, *par, *chl, *nbr8;
  const int *pn;     // [box][9]: the parent's 3x3 neighbourhood, (dx+1) + 3 (dy+1) (-1 outside, -2 none)
  const int *ref;    // [box]: bit f = face neighbour f has children, bit 4 = the box has children
  const int2 *ij;
  const double *w;   // [box][8][3]: w_lo, w_hi, 1/(w_lo + w_hi + 2) of column i
  const double *wv;  // [box][8]: volume (and y-face area) weight of column i
};

struct QLut {
  const double *mu, *diff, *alpha;
  int n;
  double inv_de;     // (n - 1) / e_max
};

__device__ __forceinline__ int dir8(int dx, int dy) {
  const int d = (dx + 1) + 3 * (dy + 1);
  return d < 4 ? d : d - 1;
}
__device__ __forceinline__ int face_dir8(int f) {
  return f < 2 ? dir8(f ? 1 : -1, 0) : dir8(0, f == 3 ? 1 : -1);
}
// cell at depth t from face f (t = 0 inner layer, t < 0 ghost layers), u along the face
__device__ __forceinline__ void face_cell(int f, int t, int u, int &ci, int &cj) {
  const int v = (f & 1) ? QN - 1 - t : t;
  if (f < 2) {
    ci = v;
    cj = u;
  } else {
    ci = u;
    cj = v;
  }
}

// What a warp needs to know about its box, loaded in one round of
// independent loads at kernel start (the tables are built on the host):
// face neighbours, the parent's 3x3 neighbourhood, coordinates, level and
// the refinement bits.  Every coarse or neighbour value a kernel reads is
// then one dependent load away.
struct BoxCtx {
  int nb[4], pn[9];
  int ix, iy, lev, ref;
};

__device__ __forceinline__ void load_ctx(const QTabs &T, int b, BoxCtx &c, int lane) {
  if (lane < 4) c.nb[lane] = T.nbr8[8 * b + face_dir8(lane)];
  else if (lane < 13) c.pn[lane - 4] = T.pn[9 * b + lane - 4];
  else if (lane == 13) {
    const int2 v = T.ij[b];
    c.ix = v.x;
    c.iy = v.y;
  } else if (lane == 14) c.lev = T.lev[b];
  else if (lane == 15) c.ref = T.ref[b];
  __syncwarp();
}

// Box of level l-1 holding coarse cell (cx, cy) (cells per side ncl): -1
// outside the domain; -2 (and the error flag) when it does not exist.
__device__ __forceinline__ int coarse_box(const BoxCtx &C, int cx, int cy, int ncl, unsigned *err) {
  if (cx < 0 || cy < 0 || cx >= ncl || cy >= ncl) return -1;
  const int dx = (cx >> 3) - (C.ix >> 1), dy = (cy >> 3) - (C.iy >> 1);
  int b = -2;
  if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) b = C.pn[(dx + 1) + 3 * (dy + 1)];
  if (b < 0) {
    atomicOr(err, 1u);
    b = -2;
  }
  return b;
}

// value of var at coarse cell q, or across the wall from coarse cell `from`
// (inside): Dirichlet (homog ? 0 : 2g) - v, Neumann / axis v; mirror: always v
__device__ __forceinline__ double coarse_val(const double *var, const BoxCtx &C, int qx, int qy, int fx, int fy,
                                             int ncl, const QBc &bc, int homog, bool mirror, unsigned *err) {
  const bool out = qx < 0 || qy < 0 || qx >= ncl || qy >= ncl;
  const int b = coarse_box(C, out ? fx : qx, out ? fy : qy, ncl, err);
  const double v = b >= 0 ? var[(size_t)b * QC + ((out ? fx : qx) & 7) + QN * ((out ? fy : qy) & 7)] : 0.0;
  if (!out || mirror) return v;
  const int f = qx < 0 ? 0 : (qx >= ncl ? 1 : (qy < 0 ? 2 : 3));
  return bc.type[f] ? (homog ? 0.0 : bc.g2[f]) - v : v;
}

// Programmatic dependent launch: a kernel launched with it may start while
// its predecessor drains; it loads only tables (which no kernel writes)
// before this wait, and every field value after it.
__device__ __forceinline__ void q_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The start of a box kernel: the box's context, the wait for the
// predecessor, then the box's own values (cells lane and lane + 32).
__device__ __forceinline__ void begin_box(const double *var, const QTabs &T, int b, BoxCtx &C, int lane, double &v0,
                                          double &v1) {
  load_ctx(T, b, C, lane);
  q_wait();
  v0 = var[(size_t)b * QC + lane];
  v1 = var[(size_t)b * QC + lane + 32];
}

// Stage box b into s (S1 x S1, interior at (i+1, j+1)) with the potential
// ghost rules: same-level copy, wall ghost, refinement boundary
// phi_f/3 + 2 phihat/3.  v0, v1: the box's own values (cells lane and
// lane + 32).  With `alt`, neighbours with children are read from alt
// instead of var (the FAS step's restricted values); with alt_all every
// same-level neighbour is.
__device__ void stage_phi(const double *var, const double *alt, const BoxCtx &C, int b, const QBc &bc, int homog,
                          double *s, int lane, unsigned *err, double v0, double v1, bool alt_all = false) {
  s[(lane / QN + 1) * S1 + lane % QN + 1] = v0;
  s[((lane + 32) / QN + 1) * S1 + lane % QN + 1] = v1;
  __syncwarp();
  const int f = lane >> 3, u = lane & 7;
  int ci, cj, gi, gj;
  face_cell(f, 0, u, ci, cj);
  face_cell(f, -1, u, gi, gj);
  const double inner = s[(cj + 1) * S1 + ci + 1];
  const int nb = C.nb[f];
  double v;
  if (nb >= 0) {
    int si, sj;
    face_cell(f ^ 1, 0, u, si, sj);
    v = ((alt && (alt_all || ((C.ref >> f) & 1))) ? alt : var)[(size_t)nb * QC + si + QN * sj];
  } else if (nb == -1) {
    v = bc.type[f] ? (homog ? 0.0 : bc.g2[f]) - inner : inner;
  } else {
    const int ncl = QN << (C.lev - 1);
    const int Gx = C.ix * QN + gi, Gy = C.iy * QN + gj, cx = Gx >> 1, cy = Gy >> 1;
    int qx = cx, qy = cy;
    if (f < 2) qy += (Gy & 1) ? 1 : -1;
    else qx += (Gx & 1) ? 1 : -1;
    // the cells across a refinement face belong to a leaf: var holds them
    const double c = coarse_val(var, C, cx, cy, cx, cy, ncl, bc, homog, false, err);
    const double ct = coarse_val(var, C, qx, qy, cx, cy, ncl, bc, homog, false, err);
    const double phat = 0.75 * c + 0.25 * ct;
    v = inner * (1.0 / 3.0) + phat * (2.0 / 3.0);
  }
  s[(gj + 1) * S1 + gi + 1] = v;
  __syncwarp();
}

// L phi at staged cell (i, j) of box b
__device__ __forceinline__ double lap_s(const double *s, const QTabs &T, int b, int i, int j, double inv_h2) {
  const double c = s[(j + 1) * S1 + i + 1];
  const double wl = T.w[(size_t)b * 24 + 3 * i], wh = T.w[(size_t)b * 24 + 3 * i + 1];
  return (wl * (s[(j + 1) * S1 + i] - c) + wh * (s[(j + 1) * S1 + i + 2] - c) + (s[j * S1 + i + 1] - c) +
          (s[(j + 2) * S1 + i + 1] - c)) * inv_h2;
}

#define QWARP()                                  \
  __shared__ BoxCtx ctx_[WPB];                   \
  const int wv_ = threadIdx.x >> 5, lane = threadIdx.x & 31; \
  const int k_ = blockIdx.x * WPB + wv_;         \
  BoxCtx &C = ctx_[wv_];

// one colour pass of red-black Gauss-Seidel on the n boxes of level l
__global__ void __launch_bounds__(QT) k_q_rbgs(int off, int n, int l, int colour, double *__restrict__ phi,
                                               const double *__restrict__ rhs, QTabs T, const __grid_constant__ QBc bc, double h2,
                                               unsigned *err) {
  __shared__ double sm[WPB][S1 * S1];
  QWARP();
  if (k_ >= n) return;  // the whole warp
  const int b = off + k_;
  double *s = sm[wv_];
  const int j = lane >> 2, i = 2 * (lane & 3) + ((j + colour) & 1);
  const double *wc = T.w + (size_t)b * 24 + 3 * i;
  const double w0 = wc[0], w1 = wc[1], w2 = wc[2];
  double v0, v1;
  begin_box(phi, T, b, C, lane, v0, v1);
  const double fr = rhs[(size_t)b * QC + i + QN * j];
  stage_phi(phi, nullptr, C, b, bc, 0, s, lane, err, v0, v1);
  phi[(size_t)b * QC + i + QN * j] =
      (w0 * s[(j + 1) * S1 + i] + w1 * s[(j + 1) * S1 + i + 2] + s[j * S1 + i + 1] + s[(j + 2) * S1 + i + 1] -
       h2 * fr) *
      w2;
}

// Residual of every box of level l restricted to its parent's quadrant:
// the restricted potential into old[parent] (committed by k_q_fas, so that
// coarse values read for ghosts here stay unchanged), the restricted
// residual into rhs[parent].  Volume-weighted mean of the four children.
// Warps [0, n) take the boxes of level l; warps [n, n + nc) the boxes
// coff.. of level l-1, copying those without children into old (so that
// k_q_fas_rbgs0 finds the whole level in old).
__global__ void __launch_bounds__(QT) k_q_resid_restrict(int off, int n, int l, const double *__restrict__ phi,
                                                         double *__restrict__ rhs, double *__restrict__ old,
                                                         QTabs T, const __grid_constant__ QBc bc, double inv_h2, unsigned *err,
                                                         int coff = 0, int nc = 0) {
  __shared__ double sm[WPB][S1 * S1];
  __shared__ double sr[WPB][QC];
  QWARP();
  if (k_ >= n) {
    if (k_ >= n + nc) return;
    const int bc2 = coff + k_ - n;
    const bool leaf = __ldg(T.chl + 4 * bc2) < 0;
    q_wait();
    if (leaf)
      for (int c = lane; c < QC; c += 32) old[(size_t)bc2 * QC + c] = phi[(size_t)bc2 * QC + c];
    return;
  }
  const int b = off + k_;
  double *s = sm[wv_];
  double v0, v1;
  begin_box(phi, T, b, C, lane, v0, v1);
  stage_phi(phi, nullptr, C, b, bc, 0, s, lane, err, v0, v1);
  for (int c = lane; c < QC; c += 32) {
    const int i = c % QN, j = c / QN;
    sr[wv_][c] = rhs[(size_t)b * QC + c] - lap_s(s, T, b, i, j, inv_h2);
  }
  __syncwarp();
  const int p = C.pn[4];
  const int2 B = make_int2(C.ix, C.iy);
  const int m = lane & 15, ii = m & 3, jj = m >> 2;
  double sum = 0.0, wsum = 0.0;
  for (int dj = 0; dj < 2; ++dj)
    for (int di = 0; di < 2; ++di) {
      const int i = 2 * ii + di, j = 2 * jj + dj;
      const double w = T.wv[(size_t)b * QN + i];
      sum += w * (lane < 16 ? s[(j + 1) * S1 + i + 1] : sr[wv_][i + QN * j]);
      wsum += w;
    }
  const int I = 4 * (B.x & 1) + ii, J = 4 * (B.y & 1) + jj;
  (lane < 16 ? old : rhs)[(size_t)p * QC + I + QN * J] = sum / wsum;
}

// Level l (all boxes): refined boxes take their restricted potential from
// old and get the FAS right-hand side f += L phi; every box ends with
// old = phi (the values the coarse correction is measured against).
__global__ void __launch_bounds__(QT) k_q_fas(int off, int n, int l, double *__restrict__ phi,
                                              double *__restrict__ rhs, double *__restrict__ old, QTabs T, const __grid_constant__ QBc bc,
                                              double inv_h2, unsigned *err) {
  __shared__ double sm[WPB][S1 * S1];
  QWARP();
  if (k_ >= n) return;
  const int b = off + k_;
  const size_t g0 = (size_t)b * QC + lane, g1 = g0 + 32;
  double v0, v1;
  begin_box(phi, T, b, C, lane, v0, v1);
  const double o0 = old[g0], o1 = old[g1], f0 = rhs[g0], f1 = rhs[g1];
  const bool refined = C.ref & 16;
  double *s = sm[wv_];
  if (refined) {
    // the box's restricted values; neighbours with children read old too
    stage_phi(phi, old, C, b, bc, 0, s, lane, err, o0, o1);
    rhs[g0] = f0 + lap_s(s, T, b, lane % QN, lane / QN, inv_h2);
    rhs[g1] = f1 + lap_s(s, T, b, lane % QN, lane / QN + 4, inv_h2);
    phi[g0] = o0;
    phi[g1] = o1;
  } else {
    old[g0] = v0;
    old[g1] = v1;
  }
}

// k_q_fas fused with the first colour pass (colour 0) of the smoothing that
// follows it on level l.  The FAS term of a box reads its neighbours' face
// cells, whose colour-0 values the neighbours' own warps of this launch
// overwrite; so the box and every same-level neighbour value are read from
// old, which the restriction launch before filled with the whole level as
// it is now (k_q_resid_restrict with nc) and which nothing in this launch
// writes.  The staged box serves the FAS step and the colour-0 update (which
// reads colour-1 cells and ghosts only); the warp's rhs and phi writes are
// ordered before the update by __syncwarp.  The same operations as k_q_fas
// followed by k_q_rbgs with colour 0.
__global__ void __launch_bounds__(QT) k_q_fas_rbgs0(int off, int n, int l, double *__restrict__ phi,
                                                    double *__restrict__ rhs, const double *__restrict__ old,
                                                    QTabs T, const __grid_constant__ QBc bc, double inv_h2, double h2,
                                                    unsigned *err) {
  __shared__ double sm[WPB][S1 * S1];
  QWARP();
  if (k_ >= n) return;
  const int b = off + k_;
  const size_t g0 = (size_t)b * QC + lane, g1 = g0 + 32;
  double o0, o1;
  begin_box(old, T, b, C, lane, o0, o1);
  const double f0 = rhs[g0], f1 = rhs[g1];
  const bool refined = C.ref & 16;
  double *s = sm[wv_];
  const int j = lane >> 2, i = 2 * (lane & 3) + (j & 1);  // this lane's colour-0 cell
  const double *wc = T.w + (size_t)b * 24 + 3 * i;
  const double w0 = wc[0], w1 = wc[1], w2 = wc[2];
  stage_phi(phi, old, C, b, bc, 0, s, lane, err, o0, o1, true);
  if (refined) {
    rhs[g0] = f0 + lap_s(s, T, b, lane % QN, lane / QN, inv_h2);
    rhs[g1] = f1 + lap_s(s, T, b, lane % QN, lane / QN + 4, inv_h2);
    phi[g0] = o0;
    phi[g1] = o1;
  }
  __syncwarp();
  const double fr = rhs[(size_t)b * QC + i + QN * j];
  phi[(size_t)b * QC + i + QN * j] =
      (w0 * s[(j + 1) * S1 + i] + w1 * s[(j + 1) * S1 + i + 2] + s[j * S1 + i + 1] + s[(j + 2) * S1 + i + 1] -
       h2 * fr) *
      w2;
}

// Prolongation to every box of level l: (2c + c_x + c_y)/4 of the parent
// level.  corr: the correction phi - old (homogeneous wall ghosts) added to
// phi; otherwise phi itself (FMG, wall values) replaces phi.
__global__ void __launch_bounds__(QT) k_q_prolong(int off, int n, int l, double *__restrict__ phi,
                                                  const double *__restrict__ old, int corr, QTabs T, const __grid_constant__ QBc bc,
                                                  unsigned *err) {
  QWARP();
  if (k_ >= n) return;
  const int b = off + k_, ncl = QN << (l - 1);
  load_ctx(T, b, C, lane);
  q_wait();
  const int2 B = make_int2(C.ix, C.iy);
  auto cv = [&](int qx, int qy, int fx, int fy) {
    const double a = coarse_val(phi, C, qx, qy, fx, fy, ncl, bc, corr, false, err);
    return corr ? a - coarse_val(old, C, qx, qy, fx, fy, ncl, bc, corr, false, err) : a;
  };
  for (int c = lane; c < QC; c += 32) {
    const int Gx = B.x * QN + c % QN, Gy = B.y * QN + c / QN, cx = Gx >> 1, cy = Gy >> 1;
    const double sum = 2.0 * cv(cx, cy, cx, cy) + cv(cx + ((Gx & 1) ? 1 : -1), cy, cx, cy) +
                       cv(cx, cy + ((Gy & 1) ? 1 : -1), cx, cy);
    const size_t g = (size_t)b * QC + c;
    if (corr) phi[g] += 0.25 * sum;
    else phi[g] = 0.25 * sum;
  }
}

// Exact level-0 solve (one box): phi = A^-1 (f - L0), A the operator's
// matrix with homogeneous wall ghosts (inverted on the host), L0 the
// operator of phi = 0 with the wall values.
__global__ void k_q_coarse(double *__restrict__ phi, const double *__restrict__ rhs, const double *__restrict__ ainv,
                           QTabs T, const __grid_constant__ QBc bc, double inv_h2) {
  __shared__ double r[QC];
  const int c = threadIdx.x, i = c % QN, j = c / QN;
  const double wl = T.w[3 * i], wh = T.w[3 * i + 1];
  q_wait();
  double l0 = 0.0;
  if (i == 0 && bc.type[0]) l0 += wl * bc.g2[0];
  if (i == QN - 1 && bc.type[1]) l0 += wh * bc.g2[1];
  if (j == 0 && bc.type[2]) l0 += bc.g2[2];
  if (j == QN - 1 && bc.type[3]) l0 += bc.g2[3];
  r[c] = rhs[c] - l0 * inv_h2;
  __syncthreads();
  double acc = 0.0;
  for (int k = 0; k < QC; ++k) acc += ainv[c * QC + k] * r[k];
  phi[c] = acc;
}

__device__ __forceinline__ void max_bits(unsigned long long *slot, double v) {
  unsigned long long x = (unsigned long long)__double_as_longlong(fabs(v));
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(slot, x);
}

// max |f - L var| over the leaf cells of all boxes (var = a zero array for
// the denominator)
__global__ void __launch_bounds__(QT) k_q_resmax(int n, const double *__restrict__ var,
                                                 const double *__restrict__ rhs, QTabs T, const __grid_constant__ QBc bc,
                                                 const double *__restrict__ inv_h2, unsigned long long *slot,
                                                 unsigned *err) {
  __shared__ double sm[WPB][S1 * S1];
  QWARP();
  if (k_ >= n) return;
  const int b = k_;
  double v0, v1;
  begin_box(var, T, b, C, lane, v0, v1);
  if (C.ref & 16) return;
  double *s = sm[wv_];
  const int l = C.lev;
  stage_phi(var, nullptr, C, b, bc, 0, s, lane, err, v0, v1);
  double m = 0.0;
  for (int c = lane; c < QC; c += 32)
    m = fmax(m, fabs(rhs[(size_t)b * QC + c] - lap_s(s, T, b, c % QN, c / QN, inv_h2[l])));
  max_bits(slot, m);
}

// Eq. 5 on leaf cells
__global__ void k_q_charge(int n, double *__restrict__ rhs, const double *__restrict__ ne,
                           const double *__restrict__ ni, const double *__restrict__ rho, const int *__restrict__ chl,
                           double q, double eps, int use_rho) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= (long long)n * QC) return;
  if (chl[4 * (g / QC)] >= 0) return;
  rhs[g] = use_rho ? -rho[g] / eps : -q * (ni[g] - ne[g]) / eps;
}

// |E| on leaf cells: face fields (phi_i - phi_{i+1})/h, cell components the
// mean of the two faces; zero on refined boxes
__global__ void __launch_bounds__(QT) k_q_field(int n, const double *__restrict__ phi, double *__restrict__ emag,
                                                QTabs T, const __grid_constant__ QBc bc, const double *__restrict__ inv_h,
                                                unsigned *err) {
  __shared__ double sm[WPB][S1 * S1];
  QWARP();
  if (k_ >= n) return;
  const int b = k_;
  double v0, v1;
  begin_box(phi, T, b, C, lane, v0, v1);
  if (C.ref & 16) {
    for (int c = lane; c < QC; c += 32) emag[(size_t)b * QC + c] = 0.0;
    return;
  }
  double *s = sm[wv_];
  const int l = C.lev;
  stage_phi(phi, nullptr, C, b, bc, 0, s, lane, err, v0, v1);
  const double ih = inv_h[l];
  for (int c = lane; c < QC; c += 32) {
    const int i = c % QN, j = c / QN;
    const double pc = s[(j + 1) * S1 + i + 1];
    const double ex = ((s[(j + 1) * S1 + i] - pc) * ih + (pc - s[(j + 1) * S1 + i + 2]) * ih) / 2.0;
    const double ey = ((s[j * S1 + i + 1] - pc) * ih + (pc - s[(j + 2) * S1 + i + 1]) * ih) / 2.0;
    emag[(size_t)b * QC + c] = sqrt(ex * ex + ey * ey);
  }
}

__device__ __forceinline__ double lut(const double *t, const QLut &L, double e) {
  const double x = e * L.inv_de;
  if (x <= 0.0) return t[0];
  if (x >= L.n - 1) return t[L.n - 1];
  const int i = (int)x;
  const double w = x - i;
  return t[i] + w * (t[i + 1] - t[i]);
}

// psi(a/b) b of the Koren limiter, division-free (Eq. 7)
__device__ __forceinline__ double koren(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  const double s = b > 0.0 ? 1.0 : -1.0, aa = fabs(a), bb = fabs(b);
  double m = bb;
  m = fmin(m, (2.0 * bb + aa) * (1.0 / 6.0));
  m = fmin(m, aa);
  return s * m;
}

// Stage the density n with two ghost layers (S2 x S2, interior at (i+2,
// j+2)), the potential (S1) and |E| with one layer: density ghosts are
// same-level copies, mirrors at walls and the axis, and at refinement
// boundaries the prolongation (2c + c_x + c_y)/4 of the coarse cell
// containing the ghost, limited to 2c; |E| ghosts the inner value at walls
// and the coarse cell's value at refinement boundaries.
__device__ void stage_fluid(const double *nv, const double *phi, const double *emag, const BoxCtx &C, int b,
                            const QBc &bc, double *sn, double *sp, double *se, int lane, unsigned *err) {
  const int l = C.lev;
  stage_phi(phi, nullptr, C, b, bc, 0, sp, lane, err, phi[(size_t)b * QC + lane], phi[(size_t)b * QC + lane + 32]);
  for (int c = lane; c < QC; c += 32) {
    sn[(c / QN + 2) * S2 + c % QN + 2] = nv[(size_t)b * QC + c];
    se[(c / QN + 1) * S1 + c % QN + 1] = emag[(size_t)b * QC + c];
  }
  __syncwarp();
  const int2 B = make_int2(C.ix, C.iy);
  const int ncl = l > 0 ? (QN << (l - 1)) : 0;
  for (int g = lane; g < 64; g += 32) {  // density: 4 faces x 2 layers x 8
    const int f = g >> 4, t = 1 + ((g >> 3) & 1), u = g & 7;
    int gi, gj;
    face_cell(f, -t, u, gi, gj);
    const int nb = C.nb[f];
    double v;
    if (nb >= 0) {
      int si, sj;
      face_cell(f ^ 1, t - 1, u, si, sj);
      v = nv[(size_t)nb * QC + si + QN * sj];
    } else if (nb == -1) {
      int mi, mj;
      face_cell(f, t - 1, u, mi, mj);
      v = sn[(mj + 2) * S2 + mi + 2];
    } else {
      const int Gx = B.x * QN + gi, Gy = B.y * QN + gj, cx = Gx >> 1, cy = Gy >> 1;
      const double c = coarse_val(nv, C, cx, cy, cx, cy, ncl, bc, 0, true, err);
      const double sum = 2.0 * c + coarse_val(nv, C, cx + ((Gx & 1) ? 1 : -1), cy, cx, cy, ncl, bc, 0, true, err) +
                         coarse_val(nv, C, cx, cy + ((Gy & 1) ? 1 : -1), cx, cy, ncl, bc, 0, true, err);
      v = fmin(0.25 * sum, 2.0 * c);
    }
    sn[(gj + 2) * S2 + gi + 2] = v;
  }
  {  // |E|: 4 faces x 8
    const int f = lane >> 3, u = lane & 7;
    int ci, cj, gi, gj;
    face_cell(f, 0, u, ci, cj);
    face_cell(f, -1, u, gi, gj);
    const int nb = C.nb[f];
    double v;
    if (nb >= 0) {
      int si, sj;
      face_cell(f ^ 1, 0, u, si, sj);
      v = emag[(size_t)nb * QC + si + QN * sj];
    } else if (nb == -1) {
      v = se[(cj + 1) * S1 + ci + 1];
    } else {
      const int cx = (B.x * QN + gi) >> 1, cy = (B.y * QN + gj) >> 1;
      v = coarse_val(emag, C, cx, cy, cx, cy, ncl, bc, 0, true, err);
    }
    se[(gj + 1) * S1 + gi + 1] = v;
  }
  __syncwarp();
}

// flux through face m (between cells m-1 and m) along axis a at u
__device__ __forceinline__ double face_flux(const double *sn, const double *sp, const double *se, int a, int m, int u,
                                            double h, double ih, const QLut &L) {
  auto N_ = [&](int t) { return a == 0 ? sn[(u + 2) * S2 + t + 2] : sn[(t + 2) * S2 + u + 2]; };
  auto P_ = [&](int t) { return a == 0 ? sp[(u + 1) * S1 + t + 1] : sp[(t + 1) * S1 + u + 1]; };
  auto E_ = [&](int t) { return a == 0 ? se[(u + 1) * S1 + t + 1] : se[(t + 1) * S1 + u + 1]; };
  const double nL2 = N_(m - 2), nL = N_(m - 1), nR = N_(m), nR2 = N_(m + 1);
  const double e_face = (P_(m - 1) - P_(m)) * ih, e_star = (E_(m - 1) + E_(m)) / 2.0;
  const double mu = lut(L.mu, L, e_star), dc = lut(L.diff, L, e_star);
  const double v = -mu * e_face;
  const double nf = v < 0.0 ? nR - koren(nR2 - nR, nR - nL) : nL + koren(nL - nL2, nR - nL);
  return v * nf - dc * (nR - nL) * ih;
  (void)h;
}

// Fine-side fluxes of every leaf box face that borders a coarser leaf:
// cflux[box][face][u]
__global__ void __launch_bounds__(QT) k_q_cf_flux(int n, const double *__restrict__ nv, const double *__restrict__ phi,
                                                  const double *__restrict__ emag, double *__restrict__ cflux,
                                                  QTabs T, const __grid_constant__ QBc bc, QLut L, const double *__restrict__ hs,
                                                  unsigned *err) {
  __shared__ double snm[WPB][S2 * S2], spm[WPB][S1 * S1], sem[WPB][S1 * S1];
  QWARP();
  if (k_ >= n) return;
  const int b = k_;
  load_ctx(T, b, C, lane);
  q_wait();
  if (C.ref & 16) return;
  bool any = false;
  for (int f = 0; f < 4; ++f) any |= C.nb[f] == -2;
  if (!any) return;
  const int l = C.lev;
  stage_fluid(nv, phi, emag, C, b, bc, snm[wv_], spm[wv_], sem[wv_], lane, err);
  const int f = lane >> 3, u = lane & 7;
  if (C.nb[f] == -2)
    cflux[(size_t)b * 32 + f * 8 + u] =
        face_flux(snm[wv_], spm[wv_], sem[wv_], f >> 1, (f & 1) ? QN : 0, u, hs[l], 1.0 / hs[l], L);
}

// One forward Euler stage on every leaf box: dst = src - dt div F + dt
// alpha mu |E| n_e (Eq. 2-3); a face next to a refined box takes the
// area-weighted mean of the two fine fluxes from cflux.
__global__ void __launch_bounds__(QT) k_q_update(int n, const double *__restrict__ ne, const double *__restrict__ ni,
                                                 double *__restrict__ ne_out, double *__restrict__ ni_out,
                                                 const double *__restrict__ phi, const double *__restrict__ emag,
                                                 const double *__restrict__ cflux, QTabs T, const __grid_constant__ QBc bc, QLut L,
                                                 const double *__restrict__ hs, double dt, unsigned *err) {
  __shared__ double snm[WPB][S2 * S2], spm[WPB][S1 * S1], sem[WPB][S1 * S1];
  __shared__ double sf[WPB][2][(QN + 1) * QN];
  QWARP();
  if (k_ >= n) return;
  const int b = k_;
  load_ctx(T, b, C, lane);
  q_wait();
  if (C.ref & 16) return;
  const int l = C.lev;
  const double h = hs[l], ih = 1.0 / h;
  stage_fluid(ne, phi, emag, C, b, bc, snm[wv_], spm[wv_], sem[wv_], lane, err);
  for (int g = lane; g < 2 * (QN + 1) * QN; g += 32) {
    const int a = g / ((QN + 1) * QN), r = g % ((QN + 1) * QN), m = r / QN, u = r % QN;
    double F = face_flux(snm[wv_], spm[wv_], sem[wv_], a, m, u, h, ih, L);
    if (m == 0 || m == QN) {
      const int f = 2 * a + (m == QN ? 1 : 0);
      const int nb = C.nb[f];
      if ((C.ref >> f) & 1) {  // refined neighbour: mean of its fine fluxes
        int cx, cy;
        if (a == 0) {
          cx = (f & 1) ? 0 : 1;
          cy = u >> 2;
        } else {
          cx = u >> 2;
          cy = (f & 1) ? 0 : 1;
        }
        const int ch = T.chl[4 * nb + cx + 2 * cy];
        double s = 0.0, ws = 0.0;
        for (int du = 0; du < 2; ++du) {
          const int uf = 2 * (u & 3) + du;
          const double w = a == 0 ? 1.0 : T.wv[(size_t)ch * QN + uf];
          s += w * cflux[(size_t)ch * 32 + (f ^ 1) * 8 + uf];
          ws += w;
        }
        F = s / ws;
      }
    }
    sf[wv_][a][m * QN + u] = F;
  }
  __syncwarp();
  for (int c = lane; c < QC; c += 32) {
    const int i = c % QN, j = c / QN;
    const double wl = T.w[(size_t)b * 24 + 3 * i], wh = T.w[(size_t)b * 24 + 3 * i + 1];
    const double div = (wh * sf[wv_][0][(i + 1) * QN + j] - wl * sf[wv_][0][i * QN + j]) * ih +
                       (sf[wv_][1][(j + 1) * QN + i] - sf[wv_][1][j * QN + i]) * ih;
    const double e = sem[wv_][(j + 1) * S1 + i + 1];
    const size_t g = (size_t)b * QC + c;
    const double src = lut(L.alpha, L, e) * lut(L.mu, L, e) * e * ne[g];
    ne_out[g] = ne[g] - dt * div + dt * src;
    ni_out[g] = ni[g] + dt * src;
  }
}

// parents' quadrants := volume-weighted restriction of the n boxes of a level
__global__ void __launch_bounds__(QT) k_q_restrict(int off, int n, double *__restrict__ v, QTabs T) {
  QWARP();
  if (k_ >= n) return;
  const int b = off + k_;
  load_ctx(T, b, C, lane);
  q_wait();
  if (lane >= 16) return;
  const int p = C.pn[4];
  const int2 B = make_int2(C.ix, C.iy);
  const int ii = lane & 3, jj = lane >> 2;
  double sum = 0.0, wsum = 0.0;
  for (int dj = 0; dj < 2; ++dj)
    for (int di = 0; di < 2; ++di) {
      const int i = 2 * ii + di, j = 2 * jj + dj;
      const double w = T.wv[(size_t)b * QN + i];
      sum += w * v[(size_t)b * QC + i + QN * j];
      wsum += w;
    }
  v[(size_t)p * QC + 4 * (B.x & 1) + ii + QN * (4 * (B.y & 1) + jj)] = sum / wsum;
}

// time-step limits: max over leaf cells of sum|v_d|/dx, that plus 4D/dx^2,
// and mu n_e (slots 0..2, bit patterns of non-negative doubles)
__global__ void __launch_bounds__(QT) k_q_dt(int n, const double *__restrict__ phi, const double *__restrict__ emag,
                                             const double *__restrict__ ne, QTabs T, const __grid_constant__ QBc bc, QLut L,
                                             const double *__restrict__ hs, unsigned long long *slots,
                                             unsigned *err) {
  __shared__ double sm[WPB][S1 * S1];
  QWARP();
  if (k_ >= n) return;
  const int b = k_;
  double v0, v1;
  begin_box(phi, T, b, C, lane, v0, v1);
  if (C.ref & 16) return;
  const int l = C.lev;
  double *s = sm[wv_];
  stage_phi(phi, nullptr, C, b, bc, 0, s, lane, err, v0, v1);
  const double h = hs[l], ih = 1.0 / h;
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  for (int c = lane; c < QC; c += 32) {
    const int i = c % QN, j = c / QN;
    const double pc = s[(j + 1) * S1 + i + 1];
    const double ex = ((s[(j + 1) * S1 + i] - pc) * ih + (pc - s[(j + 1) * S1 + i + 2]) * ih) * 0.5;
    const double ey = ((s[j * S1 + i + 1] - pc) * ih + (pc - s[(j + 2) * S1 + i + 1]) * ih) * 0.5;
    const double e = emag[(size_t)b * QC + c];
    const double mu = lut(L.mu, L, e), dc = lut(L.diff, L, e);
    const double adv = (fabs(mu * ex) + fabs(mu * ey)) * ih;
    m0 = fmax(m0, adv);
    m1 = fmax(m1, adv + 2.0 * 2.0 * dc * (ih * ih));
    m2 = fmax(m2, mu * ne[(size_t)b * QC + c]);
  }
  max_bits(slots, m0);
  max_bits(slots + 1, m1);
  max_bits(slots + 2, m2);
}

__global__ void k_q_average(long long n, double *__restrict__ a, const double *__restrict__ b0,
                            const double *__restrict__ b1) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < n) a[g] = (b0[g] + b1[g]) / 2.0;
}

// alpha(e) from the table with every operation rounded on its own (no fused
// multiply-add), the arithmetic of the refinement test on both sides
__device__ __forceinline__ double alpha_rn(const double *__restrict__ t, int n, double de, double e) {
  const double x = __ddiv_rn(e, de);
  if (x <= 0.0) return t[0];
  if (x >= (double)(n - 1)) return t[n - 1];
  const int i = (int)x;
  const double w = __dsub_rn(x, (double)i);
  return __dadd_rn(t[i], __dmul_rn(w, __dsub_rn(t[i + 1], t[i])));
}

// Eq. 8 on every leaf box (one warp per box, cells lane and lane + 32):
// need[b] bit c where alpha(c1 |E|) dx >= c0 c1; fine[b] = 1 when every cell
// has alpha(c1 |E|) dx < c0_deref c1 and dx < dx_deref
__global__ void __launch_bounds__(QT) k_q_refcrit(int n, const double *__restrict__ emag, QTabs T,
                                                  const double *__restrict__ alpha, int tab_n, double de, double c1,
                                                  double c0c1, double c0dc1, double dxd,
                                                  const double *__restrict__ hs, unsigned long long *__restrict__ need,
                                                  unsigned char *__restrict__ fine) {
  QWARP();
  if (k_ >= n) return;
  const int b = k_;
  load_ctx(T, b, C, lane);
  q_wait();
  if (C.ref & 16) {
    if (lane == 0) {
      need[b] = 0ull;
      fine[b] = 0;
    }
    return;
  }
  const double dx = hs[C.lev];
  bool nd[2], ok = true;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double ad = __dmul_rn(alpha_rn(alpha, tab_n, de, __dmul_rn(c1, emag[(size_t)b * QC + lane + 32 * h])), dx);
    nd[h] = ad >= c0c1;
    ok &= ad < c0dc1;
  }
  const unsigned lo = __ballot_sync(0xffffffffu, nd[0]), hi = __ballot_sync(0xffffffffu, nd[1]);
  const bool all = __all_sync(0xffffffffu, ok);
  if (lane == 0) {
    need[b] = (unsigned long long)lo | ((unsigned long long)hi << 32);
    fine[b] = (unsigned char)(all && dx < dxd);
  }
}

// After a regrid, box b of the new mesh takes the data of old box
// rg[10 b] (>= 0) from the snapshot snap[var][old box][64] (vars: phi,
// n_e, n_i, f, |E|, rho), or, as a new child (rg[10 b] < 0), the
// prolongation (2c + c_x + c_y)/4 of its old parent's cells, rg[10 b + 1 ..
// 9] being the old parent's 3x3 neighbourhood: wall ghosts for the
// potential, mirrors and the 2c limit for the densities; f, |E| and rho of
// new boxes are zero.
__global__ void __launch_bounds__(QT) k_q_regrid_move(int n, const int *__restrict__ rg,
                                                      const double *__restrict__ snap, size_t stride,
                                                      double *__restrict__ phi, double *__restrict__ ne,
                                                      double *__restrict__ ni, double *__restrict__ rhs,
                                                      double *__restrict__ emag, double *__restrict__ rho, QTabs T,
                                                      const __grid_constant__ QBc bc, unsigned *err) {
  QWARP();
  if (k_ >= n) return;
  const int b = k_;
  double *dst[6] = {phi, ne, ni, rhs, emag, rho};
  const int src = rg[10 * (size_t)b];
  if (src >= 0) {
    for (int v = 0; v < 6; ++v)
      for (int c = lane; c < QC; c += 32) dst[v][(size_t)b * QC + c] = snap[v * stride + (size_t)src * QC + c];
    return;
  }
  if (lane < 9) C.pn[lane] = rg[10 * (size_t)b + 1 + lane];
  if (lane == 9) {
    const int2 v = T.ij[b];
    C.ix = v.x;
    C.iy = v.y;
  }
  if (lane == 10) C.lev = T.lev[b];
  __syncwarp();
  const int ncl = QN << (C.lev - 1);
  for (int c = lane; c < QC; c += 32) {
    const int Gx = C.ix * QN + c % QN, Gy = C.iy * QN + c / QN, cx = Gx >> 1, cy = Gy >> 1;
    const int qx = cx + ((Gx & 1) ? 1 : -1), qy = cy + ((Gy & 1) ? 1 : -1);
    for (int v = 0; v < 3; ++v) {
      const double *sv = snap + v * stride;
      const bool mirror = v > 0;
      const double cv = coarse_val(sv, C, cx, cy, cx, cy, ncl, bc, 0, mirror, err);
      double val = 2.0 * cv;
      val += coarse_val(sv, C, qx, cy, cx, cy, ncl, bc, 0, mirror, err);
      val += coarse_val(sv, C, cx, qy, cx, cy, ncl, bc, 0, mirror, err);
      val = 0.25 * val;
      if (mirror && val > 2.0 * cv) val = 2.0 * cv;
      dst[v][(size_t)b * QC + c] = val;
    }
    for (int v = 3; v < 6; ++v) dst[v][(size_t)b * QC + c] = 0.0;
  }
}

// ---- regrid: the new box set on the device ---------------------------------
//
// Old boxes are stored level by level in Morton order.  The new set keeps
// every box but the children of derefined boxes and adds 4 children per
// refined box; each new level is the merge of two Morton-sorted lists (the
// kept boxes of the level and the children of the refined boxes of the level
// below, whose keys are parent key * 4 + child), so a box's new index is its
// rank in its own list plus the count of keys of the other list below its
// own (binary searches).  Parents, children and same-level neighbours follow
// by binary search in the new levels' keys.

// per-level starts of the compacted lists and of the new levels
struct QRgLevels {
  int kept[QMAXL + 2];  // level l in the kept list
  int ref[QMAXL + 2];   // level l in the refined list
  int nw[QMAXL + 2];    // level l in the new numbering
};
struct QOffsets {
  int v[QMAXL + 2];
};

// Morton key of (i, j) within its level: bit b of i to bit 2b, of j to 2b + 1
__device__ __forceinline__ uint64_t qmorton(int i, int j) {
  auto spread = [](unsigned v) {
    uint64_t x = v & 0x7fffffffu;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
  };
  return spread((unsigned)i) | (spread((unsigned)j) << 1);
}

// first index in [lo, hi) whose key is >= x
__device__ __forceinline__ int qlower_bound(const uint64_t *__restrict__ a, int lo, int hi, uint64_t x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// refinement: a flagged leaf below the maximum level whose 8 neighbour
// positions of its level hold a box or lie outside the domain (else the
// request is dropped: cnt[0])
__global__ void k_qrg_refine(int n, const int *__restrict__ lev, const int *__restrict__ chl,
                             const int *__restrict__ nbr8, const int8_t *__restrict__ flags, int lmax,
                             int *__restrict__ refv, int *cnt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  int r = 0;
  if (chl[4 * b] < 0 && flags[b] > 0 && lev[b] < lmax) {
    bool ok = true;
    for (int d = 0; d < 8; ++d) ok = ok && nbr8[8 * b + d] != -2;
    if (ok) r = 1;
    else atomicAdd(cnt, 1);
  }
  refv[b] = r;
}

// derefinement of box p: its 4 children are leaves flagged < 0 and no
// neighbour of a child outside the siblings has or gets children (cnt[1]
// counts them)
__global__ void k_qrg_derefine(int n, const int *__restrict__ chl, const int *__restrict__ par,
                               const int *__restrict__ nbr8, const int8_t *__restrict__ flags,
                               const int *__restrict__ refv, int *__restrict__ derv, int *cnt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  bool ok = chl[4 * p] >= 0;
  for (int c = 0; c < 4 && ok; ++c) {
    const int ch = chl[4 * p + c];
    ok = chl[4 * ch] < 0 && flags[ch] < 0;
  }
  for (int c = 0; c < 4 && ok; ++c) {
    const int ch = chl[4 * p + c];
    for (int d = 0; d < 8 && ok; ++d) {
      const int nb = nbr8[8 * ch + d];
      if (nb >= 0 && par[nb] != p && (chl[4 * nb] >= 0 || refv[nb])) ok = false;
    }
  }
  derv[p] = ok ? 1 : 0;
  if (ok) atomicAdd(cnt + 1, 1);
}

// keepv[b] = b is not a child of a derefined box
__global__ void k_qrg_keep(int n, const int *__restrict__ par, const int *__restrict__ derv,
                           int *__restrict__ keepv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int p = par[b];
  keepv[b] = (p >= 0 && derv[p]) ? 0 : 1;
}

// exclusive prefix sums of two int arrays of n entries (block y = 0: in0 ->
// out0, y = 1: in1 -> out1), out[n] = the total: each thread sums a
// contiguous chunk, the chunk sums are scanned in the block, then each
// thread writes its chunk's prefixes
__global__ void __launch_bounds__(1024) k_qrg_scan2(const int *__restrict__ in0, int *__restrict__ out0,
                                                    const int *__restrict__ in1, int *__restrict__ out1, int n) {
  __shared__ int wsum[32];
  const int *in = blockIdx.y ? in1 : in0;
  int *out = blockIdx.y ? out1 : out0;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int chunk = (n + 1023) / 1024, lo = min(n, t * chunk), hi = min(n, lo + chunk);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += in[i];
  int x = s;  // inclusive scan of the chunk sums: warps, then the warp totals
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int v = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    wsum[lane] = v;
  }
  __syncthreads();
  int run = x - s + (w ? wsum[w - 1] : 0);
  for (int i = lo; i < hi; ++i) {
    const int v = in[i];
    out[i] = run;
    run += v;
  }
  if (t == 1023) out[n] = wsum[31];
}

// the counts the host needs in one array: dropped and derefined requests,
// then the kept and the refined list positions at the old level offsets
__global__ void k_qrg_counts(const int *__restrict__ cnt, const int *__restrict__ keep_pos,
                             const int *__restrict__ ref_pos, QOffsets off, int nl, int *__restrict__ out) {
  const int t = threadIdx.x;
  if (t < 2) out[t] = cnt[t];
  if (t <= nl) {
    out[2 + t] = keep_pos[off.v[t]];
    out[3 + nl + t] = ref_pos[off.v[t]];
  }
}

// the Morton keys of the kept and of the refined boxes, compacted
__global__ void k_qrg_keys(int n, const int2 *__restrict__ ij, const int *__restrict__ keepv,
                           const int *__restrict__ keep_pos, const int *__restrict__ refv,
                           const int *__restrict__ ref_pos, uint64_t *__restrict__ kept_keys,
                           uint64_t *__restrict__ ref_keys) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int2 v = ij[b];
  const uint64_t key = qmorton(v.x, v.y);
  if (keepv[b]) kept_keys[keep_pos[b]] = key;
  if (refv[b]) ref_keys[ref_pos[b]] = key;
}

// new index, level, coordinates and key of every kept box and of the 4
// children of every refined box (4 threads per old box: thread 0 places the
// box itself when kept, thread c its child c when refined), with the move
// descriptor of the new box: its old index, or -1 and the old parent's 3x3
// neighbourhood (old numbering) for a new child
__global__ void k_qrg_place(int n, const int *__restrict__ lev, const int2 *__restrict__ ij,
                            const int *__restrict__ nbr8, const int *__restrict__ keepv,
                            const int *__restrict__ keep_pos, const int *__restrict__ refv,
                            const int *__restrict__ ref_pos, const uint64_t *__restrict__ kept_keys,
                            const uint64_t *__restrict__ ref_keys, QRgLevels L, int *__restrict__ nlev,
                            int2 *__restrict__ nij, uint64_t *__restrict__ nkey, int *__restrict__ rg) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = t >> 2, c = t & 3;
  if (b >= n) return;
  const int l = lev[b];
  const int2 v = ij[b];
  const uint64_t key = qmorton(v.x, v.y);
  if (c == 0 && keepv[b]) {
    // children of refined boxes of level l-1 whose parent key is below this box's
    const int below = l > 0 ? qlower_bound(ref_keys, L.ref[l - 1], L.ref[l], key >> 2) - L.ref[l - 1] : 0;
    const int x = L.nw[l] + (keep_pos[b] - L.kept[l]) + 4 * below;
    nlev[x] = l;
    nij[x] = v;
    nkey[x] = key;
    rg[10 * (size_t)x] = b;
  }
  if (refv[b]) {
    const uint64_t ck = (key << 2) | (uint64_t)c;
    const int below = qlower_bound(kept_keys, L.kept[l + 1], L.kept[l + 2], ck) - L.kept[l + 1];
    const int x = L.nw[l + 1] + 4 * (ref_pos[b] - L.ref[l]) + c + below;
    nlev[x] = l + 1;
    nij[x] = make_int2(2 * v.x + (c & 1), 2 * v.y + (c >> 1));
    nkey[x] = ck;
    int *r = rg + 10 * (size_t)x;
    r[0] = -1;
    for (int k = 0; k < 9; ++k) r[1 + k] = k == 4 ? b : nbr8[8 * b + (k < 4 ? k : k - 1)];
  }
}

// parent and children of every new box by binary search in the new keys
__global__ void k_qrg_links(int m, const int *__restrict__ nlev, const uint64_t *__restrict__ nkey, QRgLevels L,
                            int nlevels, int *__restrict__ par, int *__restrict__ chl) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m) return;
  const int l = nlev[b];
  const uint64_t key = nkey[b];
  int p = -1;
  if (l > 0) {
    const int i = qlower_bound(nkey, L.nw[l - 1], L.nw[l], key >> 2);
    if (i < L.nw[l] && nkey[i] == key >> 2) p = i;
  }
  par[b] = p;
  int c0 = -1;  // the first child; the four siblings are consecutive keys
  if (l + 1 < nlevels) {
    const int i = qlower_bound(nkey, L.nw[l + 1], L.nw[l + 2], key << 2);
    if (i + 3 < L.nw[l + 2] && nkey[i] == key << 2 && nkey[i + 3] == ((key << 2) | 3ull)) c0 = i;
  }
  for (int c = 0; c < 4; ++c) chl[4 * b + c] = c0 >= 0 ? c0 + c : -1;
}

// same-level neighbours (8 threads per new box, direction d): -1 outside
// the domain, -2 where the level holds no box
__global__ void k_qrg_nbr(int m, const int *__restrict__ nlev, const int2 *__restrict__ nij,
                          const uint64_t *__restrict__ nkey, QRgLevels L, int *__restrict__ nbr8) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = t >> 3, d = t & 7;
  if (b >= m) return;
  const int k = d < 4 ? d : d + 1, dx = k % 3 - 1, dy = k / 3 - 1;
  const int l = nlev[b], side = 1 << l;
  const int2 v = nij[b];
  const int i = v.x + dx, j = v.y + dy;
  int r = -1;
  if (i >= 0 && j >= 0 && i < side && j < side) {
    const uint64_t key = qmorton(i, j);
    const int x = qlower_bound(nkey, L.nw[l], L.nw[l + 1], key);
    r = (x < L.nw[l + 1] && nkey[x] == key) ? x : -2;
  }
  nbr8[8 * b + d] = r;
}

// the tables derived from the links: the parent's 3x3 neighbourhood, the
// refinement bits and the column weights (8 threads per new box, column c)
__global__ void k_qrg_derived(int m, int cyl, const int *__restrict__ par, const int *__restrict__ chl,
                              const int *__restrict__ nbr8, const int2 *__restrict__ ij, int *__restrict__ pn,
                              int *__restrict__ ref, double *__restrict__ w, double *__restrict__ wv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = t >> 3, c = t & 7;
  if (b >= m) return;
  const int p = par[b];
  const int k = c < 4 ? c : c + 1;  // the 3x3 slots other than the centre
  pn[9 * (size_t)b + k] = p >= 0 ? nbr8[8 * p + c] : -1;
  if (c == 0) {
    pn[9 * (size_t)b + 4] = p;
    int r = chl[4 * b] >= 0 ? 16 : 0;
    const int fd[4] = {3, 4, 1, 6};  // faces -x, +x, -y, +y among the 8 directions
    for (int f = 0; f < 4; ++f) {
      const int nb = nbr8[8 * b + fd[f]];
      if (nb >= 0 && chl[4 * nb] >= 0) r |= 1 << f;
    }
    ref[b] = r;
  }
  // column weights, each operation rounded on its own as on the host
  const int gx = ij[b].x * QN + c;
  const double g = (double)gx, gh = __dadd_rn(g, 0.5);
  const double wl = cyl ? __ddiv_rn(g, gh) : 1.0, wh = cyl ? __ddiv_rn(__dadd_rn(g, 1.0), gh) : 1.0;
  w[24 * (size_t)b + 3 * c] = wl;
  w[24 * (size_t)b + 3 * c + 1] = wh;
  w[24 * (size_t)b + 3 * c + 2] = __ddiv_rn(1.0, __dadd_rn(__dadd_rn(wl, wh), 2.0));
  wv[8 * (size_t)b + c] = cyl ? gh : 1.0;
}

int blocks_for(long long boxes) { return (int)std::max<long long>(1, (boxes + WPB - 1) / WPB); }

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct sm_quad {
  sm_quad_domain dom{};
  int max_boxes = 0, nu1 = 2, nu2 = 2, lbase = 0, lmax = 0;
  cudaStream_t stream = nullptr;
  QBc bc{};
  std::string err;
  long long launches = 0;
  // host tables
  std::vector<int> lev, ix, iy, par, chl, nbr8;
  std::vector<uint64_t> mort;
  int nlev = 0;
  int off[QMAXL + 2] = {0};
  // arena
  char *arena = nullptr;
  int *d_lev = nullptr, *d_par = nullptr, *d_chl = nullptr, *d_nbr8 = nullptr, *d_pn = nullptr, *d_ref = nullptr;
  int2 *d_ij = nullptr;
  double *d_w = nullptr, *d_wv = nullptr;
  double *var[NV] = {nullptr};
  double *cflux = nullptr, *ainv = nullptr, *lut = nullptr, *d_h = nullptr;
  unsigned long long *slots = nullptr;
  unsigned *d_err = nullptr;
  double *snap = nullptr;                 // regrid snapshot [6][max_boxes][64]
  int *d_rg = nullptr;                    // regrid move descriptors [max_boxes][10]
  unsigned long long *d_need = nullptr;   // refinement test: cells that need refinement, per box
  unsigned char *d_fine = nullptr;        // refinement test: derefinable, per box
  int lut_n = 0;
  double lut_emax = 0.0;
  double h[QMAXL], inv_h2[QMAXL];
  std::vector<double> h_ainv;
  // V-cycle graphs per top level (captured on first use, dropped when the
  // mesh changes) and the launches each holds
  cudaStream_t cap = nullptr;
  cudaGraphExec_t vgraph[QMAXL] = {nullptr};
  long long vgraph_launches[QMAXL] = {0};
  bool graphs = true, pdl = true;
  ~sm_quad() {
    for (auto &g : vgraph)
      if (g) cudaGraphExecDestroy(g);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace {

int qfail(sm_quad *q, int code, const std::string &msg) {
  if (q) q->err = msg;
  return code;
}

uint64_t morton2(int i, int j) {
  uint64_t k = 0;
  for (int b = 0; b < 31; ++b) k |= (uint64_t)((i >> b) & 1) << (2 * b) | (uint64_t)((j >> b) & 1) << (2 * b + 1);
  return k;
}

int dir8h(int dx, int dy) {
  const int d = (dx + 1) + 3 * (dy + 1);
  return d < 4 ? d : d - 1;
}

int find_box(const sm_quad *q, int l, int i, int j) {
  const int n = 1 << l;
  if (i < 0 || j < 0 || i >= n || j >= n) return -1;
  if (l >= q->nlev) return -2;
  const uint64_t key = morton2(i, j);
  int lo = q->off[l], hi = q->off[l + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) / 2;
    if (q->mort[mid] == key) return mid;
    if (q->mort[mid] < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -2;
}

// weights of the column with global x index gx (at its box's level):
// w_lo, w_hi, 1/(w_lo + w_hi + 2) and the volume weight; the same roundings
// as the device's regrid tables (col_weights_dev)
void col_weights(const sm_quad *q, int gx, double *w3, double *wv) {
  const bool cyl = q->dom.geometry == SM_AXISYMMETRIC;
  const double wl = cyl ? (double)gx / (gx + 0.5) : 1.0, wh = cyl ? (gx + 1.0) / (gx + 0.5) : 1.0;
  w3[0] = wl;
  w3[1] = wh;
  w3[2] = 1.0 / (wl + wh + 2.0);
  *wv = cyl ? gx + 0.5 : 1.0;
}

void add_box(sm_quad *q, int l, int i, int j, int parent) {
  q->lev.push_back(l);
  q->ix.push_back(i);
  q->iy.push_back(j);
  q->par.push_back(parent);
  q->mort.push_back(morton2(i, j));
  for (int c = 0; c < 4; ++c) q->chl.push_back(-1);
  for (int d = 0; d < 8; ++d) q->nbr8.push_back(-2);
}

void set_neighbours(sm_quad *q, int l) {
  for (int b = q->off[l]; b < q->off[l + 1]; ++b)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        if (dx || dy) q->nbr8[8 * b + dir8h(dx, dy)] = find_box(q, l, q->ix[b] + dx, q->iy[b] + dy);
}

int n_boxes(const sm_quad *q) { return (int)q->lev.size(); }

int upload_tables(sm_quad *q) {
  const int n = n_boxes(q);
  std::vector<int2> ij(n);
  std::vector<int> pn(9 * (size_t)n, -1), ref(n, 0);
  std::vector<double> w(24 * (size_t)n), wv(8 * (size_t)n);
  for (int b = 0; b < n; ++b) {
    ij[b] = make_int2(q->ix[b], q->iy[b]);
    for (int c = 0; c < QN; ++c) col_weights(q, q->ix[b] * QN + c, &w[24 * (size_t)b + 3 * c], &wv[8 * (size_t)b + c]);
    const int p = q->par[b];
    if (p >= 0)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
          pn[9 * (size_t)b + (dx + 1) + 3 * (dy + 1)] = (dx || dy) ? q->nbr8[8 * p + dir8h(dx, dy)] : p;
    int r = q->chl[4 * b] >= 0 ? 16 : 0;
    const int fd[4] = {dir8h(-1, 0), dir8h(1, 0), dir8h(0, -1), dir8h(0, 1)};
    for (int f = 0; f < 4; ++f) {
      const int nb = q->nbr8[8 * b + fd[f]];
      if (nb >= 0 && q->chl[4 * nb] >= 0) r |= 1 << f;
    }
    ref[b] = r;
  }
  cudaStream_t s = q->stream;
  if (cudaMemcpyAsync(q->d_lev, q->lev.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_par, q->par.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_chl, q->chl.data(), sizeof(int) * 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_nbr8, q->nbr8.data(), sizeof(int) * 8 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_ij, ij.data(), sizeof(int2) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_pn, pn.data(), sizeof(int) * 9 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_ref, ref.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_w, w.data(), sizeof(double) * 24 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_wv, wv.data(), sizeof(double) * 8 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return qfail(q, SM_ECUDA, "table upload");
  return SM_OK;
}

QTabs tabs(const sm_quad *q) {
  return {q->d_lev, q->d_par, q->d_chl, q->d_nbr8, q->d_pn, q->d_ref, q->d_ij, q->d_w, q->d_wv};
}
QLut qlut(const sm_quad *q) {
  return {q->lut, q->lut + q->lut_n, q->lut + 2 * q->lut_n, q->lut_n, (q->lut_n - 1) / q->lut_emax};
}

// the level-0 operator with homogeneous wall ghosts (columns L e_k) and its
// inverse by Gauss-Jordan elimination with partial pivoting (host)
void coarse_inverse(sm_quad *q) {
  const int n = QC;
  std::vector<double> A((size_t)n * n, 0.0), I((size_t)n * n, 0.0);
  const double ih2 = q->inv_h2[0];
  for (int r = 0; r < n; ++r) {
    const int i = r % QN, j = r / QN;
    double w3[3], wvol;
    col_weights(q, i, w3, &wvol);  // level 0: box 0, global column i
    const double wl = w3[0], wh = w3[1];
    const double wf[4] = {wl, wh, 1.0, 1.0};
    const int nbr[4] = {i > 0 ? r - 1 : -1, i < QN - 1 ? r + 1 : -1, j > 0 ? r - QN : -1, j < QN - 1 ? r + QN : -1};
    for (int f = 0; f < 4; ++f) {
      // L phi = sum_f w_f (phi_f - phi): a wall ghost is -phi (Dirichlet) or phi
      A[(size_t)r * n + r] -= wf[f] * ih2;
      if (nbr[f] >= 0) A[(size_t)r * n + nbr[f]] += wf[f] * ih2;
      else A[(size_t)r * n + r] += (q->bc.type[f] ? -1.0 : 1.0) * wf[f] * ih2;
    }
    I[(size_t)r * n + r] = 1.0;
  }
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)p * n + c])) p = r;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)c * n + k], A[(size_t)p * n + k]);
        std::swap(I[(size_t)c * n + k], I[(size_t)p * n + k]);
      }
    const double d = A[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      A[(size_t)c * n + k] /= d;
      I[(size_t)c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double m = A[(size_t)r * n + c];
      if (m == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)r * n + k] -= m * A[(size_t)c * n + k];
        I[(size_t)r * n + k] -= m * I[(size_t)c * n + k];
      }
    }
  }
  q->h_ainv = I;
}

int check(sm_quad *q, const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return qfail(q, SM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return SM_OK;
}

int level_count(const sm_quad *q, int l) { return q->off[l + 1] - q->off[l]; }

// launch with programmatic dependent launch (every kernel of this file
// waits for its predecessor before reading a field)
template <typename... KArgs, typename... Args>
void qlaunch(sm_quad *q, void (*k)(KArgs...), int grid, int block, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = q->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = q->pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
  ++q->launches;
}

// nu red-black sweeps of level l; with skip_first the first colour pass has
// already run (k_q_fas_rbgs0)
void smooth(sm_quad *q, int l, int nu, bool skip_first = false) {
  const int n = level_count(q, l);
  for (int s = 0; s < nu; ++s)
    for (int c = 0; c < 2; ++c) {
      if (skip_first && s == 0 && c == 0) continue;
      qlaunch(q, k_q_rbgs, blocks_for(n), QT, q->off[l], n, l, c, q->var[V_PHI], (const double *)q->var[V_RHS],
              tabs(q), q->bc, q->h[l] * q->h[l], q->d_err);
    }
}

void coarse_solve(sm_quad *q) {
  qlaunch(q, k_q_coarse, 1, QC, q->var[V_PHI], (const double *)q->var[V_RHS], (const double *)q->ainv, tabs(q),
          q->bc, q->inv_h2[0]);
}

void vcycle(sm_quad *q, int top) {
  bool fused = false;  // the first colour pass of level l has run (k_q_fas_rbgs0)
  for (int l = top; l >= 1; --l) {
    smooth(q, l, q->nu1, fused);
    const int n = level_count(q, l), nc = level_count(q, l - 1);
    // below the top level but above level 0 the FAS step also runs the first
    // colour pass; the restriction then copies the level's leaves into old
    fused = l - 1 >= 1;
    const int ncp = fused ? nc : 0;
    qlaunch(q, k_q_resid_restrict, blocks_for(n + ncp), QT, q->off[l], n, l, (const double *)q->var[V_PHI],
            q->var[V_RHS], q->var[V_OLD], tabs(q), q->bc, q->inv_h2[l], q->d_err, q->off[l - 1], ncp);
    if (fused)
      qlaunch(q, k_q_fas_rbgs0, blocks_for(nc), QT, q->off[l - 1], nc, l - 1, q->var[V_PHI], q->var[V_RHS],
              (const double *)q->var[V_OLD], tabs(q), q->bc, q->inv_h2[l - 1], q->h[l - 1] * q->h[l - 1], q->d_err);
    else
      qlaunch(q, k_q_fas, blocks_for(nc), QT, q->off[l - 1], nc, l - 1, q->var[V_PHI], q->var[V_RHS],
              q->var[V_OLD], tabs(q), q->bc, q->inv_h2[l - 1], q->d_err);
  }
  coarse_solve(q);
  for (int l = 1; l <= top; ++l) {
    const int n = level_count(q, l);
    qlaunch(q, k_q_prolong, blocks_for(n), QT, q->off[l], n, l, q->var[V_PHI], (const double *)q->var[V_OLD], 1,
            tabs(q), q->bc, q->d_err);
    smooth(q, l, q->nu2);
  }
}

void drop_graphs(sm_quad *q) {
  for (int l = 0; l < QMAXL; ++l)
    if (q->vgraph[l]) {
      cudaGraphExecDestroy(q->vgraph[l]);
      q->vgraph[l] = nullptr;
    }
}

// One V-cycle with level `top` on top, as a CUDA graph captured on first
// use (the same launches as vcycle; host launch gaps removed)
int vcycle_g(sm_quad *q, int top) {
  if (!q->graphs) {
    vcycle(q, top);
    return check(q, "V-cycle");
  }
  if (!q->vgraph[top]) {
    if (!q->cap && cudaStreamCreateWithFlags(&q->cap, cudaStreamNonBlocking) != cudaSuccess)
      return qfail(q, SM_ECUDA, "capture stream");
    cudaStream_t saved = q->stream;
    const long long l0 = q->launches;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(q->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return qfail(q, SM_ECUDA, "begin capture");
    q->stream = q->cap;
    vcycle(q, top);
    q->stream = saved;
    const cudaError_t e = cudaStreamEndCapture(q->cap, &g);
    if (e != cudaSuccess || !g) {
      cudaGetLastError();
      return qfail(q, SM_ECUDA, "V-cycle capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&q->vgraph[top], g, 0);
    cudaGraphDestroy(g);
    q->vgraph_launches[top] = q->launches - l0;
    q->launches = l0;
    if (ei != cudaSuccess) {
      q->vgraph[top] = nullptr;
      return qfail(q, SM_ECUDA, "V-cycle instantiate");
    }
  }
  if (cudaGraphLaunch(q->vgraph[top], q->stream) != cudaSuccess) return qfail(q, SM_ECUDA, "graph launch");
  q->launches += q->vgraph_launches[top];
  return SM_OK;
}

// max leaf residual of var (the potential, or the zero array)
int resmax(sm_quad *q, int v, double *out) {
  const int n = n_boxes(q);
  if (cudaMemsetAsync(q->slots + 4, 0, sizeof(unsigned long long), q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "memset");
  k_q_resmax<<<blocks_for(n), QT, 0, q->stream>>>(n, q->var[v], q->var[V_RHS], tabs(q), q->bc, q->d_h + QMAXL,
                                                   q->slots + 4, q->d_err);
  ++q->launches;
  unsigned long long bits = 0;
  unsigned e = 0;
  if (cudaMemcpyAsync(&bits, q->slots + 4, sizeof(bits), cudaMemcpyDeviceToHost, q->stream) != cudaSuccess ||
      cudaMemcpyAsync(&e, q->d_err, sizeof(e), cudaMemcpyDeviceToHost, q->stream) != cudaSuccess ||
      cudaStreamSynchronize(q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "residual norm");
  if (e) return qfail(q, SM_ESTATE, "a coarse box needed at a refinement boundary is missing");
  double d;
  std::memcpy(&d, &bits, sizeof(d));
  *out = d;
  return SM_OK;
}

int rel_residual(sm_quad *q, double *rel) {
  double num = 0.0, den = 0.0;
  if (cudaMemsetAsync(q->var[V_TMP], 0, sizeof(double) * QC * (size_t)n_boxes(q), q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "memset");
  if (int st = resmax(q, V_PHI, &num)) return st;
  if (int st = resmax(q, V_TMP, &den)) return st;
  *rel = den > 0.0 ? num / den : num;
  return SM_OK;
}

int solve_loop(sm_quad *q, double tol, int max_cycles, int c0, int *cycles, double *rel) {
  int c = c0;
  double r = 0.0;
  if (c0 > 0) {
    if (int st = rel_residual(q, &r)) return st;
  }
  while (c == 0 || (r > tol && c < max_cycles)) {
    if (int st = vcycle_g(q, q->nlev - 1)) return st;
    ++c;
    if (int st = rel_residual(q, &r)) return st;
  }
  if (cycles) *cycles = c;
  if (rel) *rel = r;
  return r <= tol ? SM_OK : qfail(q, SM_ENOCONV, "tolerance not reached");
}

void restrict_all(sm_quad *q, int v) {
  for (int l = q->nlev - 1; l >= 1; --l) {
    const int n = level_count(q, l);
    k_q_restrict<<<blocks_for(n), QT, 0, q->stream>>>(q->off[l], n, q->var[v], tabs(q));
    ++q->launches;
  }
}

int euler_stage(sm_quad *q, int sne, int sni, int dne, int dni, double dt) {
  const int n = n_boxes(q);
  k_q_cf_flux<<<blocks_for(n), QT, 0, q->stream>>>(n, q->var[sne], q->var[V_PHI], q->var[V_EMAG], q->cflux, tabs(q),
                                                    q->bc, qlut(q), q->d_h, q->d_err);
  k_q_update<<<blocks_for(n), QT, 0, q->stream>>>(n, q->var[sne], q->var[sni], q->var[dne], q->var[dni],
                                                   q->var[V_PHI], q->var[V_EMAG], q->cflux, tabs(q), q->bc, qlut(q),
                                                   q->d_h, dt, q->d_err);
  q->launches += 2;
  restrict_all(q, dne);
  restrict_all(q, dni);
  return check(q, "fluid stage");
}

int charge(sm_quad *q, double c, double eps, int use_rho) {
  const long long cells = (long long)n_boxes(q) * QC;
  k_q_charge<<<(int)((cells + 255) / 256), 256, 0, q->stream>>>(n_boxes(q), q->var[V_RHS], q->var[V_NE],
                                                                  q->var[V_NI], q->var[V_RHO], q->d_chl, c, eps,
                                                                  use_rho);
  ++q->launches;
  return check(q, "charge");
}

int field(sm_quad *q) {
  const int n = n_boxes(q);
  k_q_field<<<blocks_for(n), QT, 0, q->stream>>>(n, q->var[V_PHI], q->var[V_EMAG], tabs(q), q->bc,
                                                  q->d_h + 2 * QMAXL, q->d_err);
  ++q->launches;
  return check(q, "field");
}

int dt_limit(sm_quad *q, double c, double eps, double *dt) {
  const int n = n_boxes(q);
  if (cudaMemsetAsync(q->slots, 0, 3 * sizeof(unsigned long long), q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "memset");
  k_q_dt<<<blocks_for(n), QT, 0, q->stream>>>(n, q->var[V_PHI], q->var[V_EMAG], q->var[V_NE], tabs(q), q->bc,
                                               qlut(q), q->d_h, q->slots, q->d_err);
  ++q->launches;
  unsigned long long bits[3];
  if (cudaMemcpyAsync(bits, q->slots, sizeof(bits), cudaMemcpyDeviceToHost, q->stream) != cudaSuccess ||
      cudaStreamSynchronize(q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "dt limit");
  double m[3];
  std::memcpy(m, bits, sizeof(m));
  double d = 1e300;
  if (m[0] > 0.0 && 0.5 / m[0] < d) d = 0.5 / m[0];
  if (m[1] > 0.0 && 1.0 / m[1] < d) d = 1.0 / m[1];
  if (m[2] > 0.0 && eps / (c * m[2]) < d) d = eps / (c * m[2]);
  *dt = 0.9 * d;
  return SM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int sm_quad_create(sm_quad **out, const sm_quad_domain *dom, int max_boxes, int nu1, int nu2,
                              void *stream) {
  if (!out || !dom) return SM_EINVAL;
  *out = nullptr;
  int lb = 0;
  while ((1 << lb) < dom->nb) ++lb;
  if (dom->nb < 1 || (1 << lb) != dom->nb || dom->max_level < 0 || lb + dom->max_level >= QMAXL ||
      !(dom->length > 0.0) || nu1 < 1 || nu2 < 1 || nu1 > 16 || nu2 > 16 ||
      (dom->geometry != SM_CARTESIAN && dom->geometry != SM_AXISYMMETRIC))
    return SM_EINVAL;
  if (dom->geometry == SM_AXISYMMETRIC && dom->origin[0] != 0.0) return SM_EINVAL;
  int dir = 0;
  for (int f = 0; f < 4; ++f) {
    if (dom->bc_type[f] != 0 && dom->bc_type[f] != 1) return SM_EINVAL;
    if (f > 0 || dom->geometry == SM_CARTESIAN) dir |= dom->bc_type[f];
  }
  if (!dir) return SM_EINVAL;
  long long uniform = 0;
  for (int l = 0; l <= lb; ++l) uniform += 1ll << (2 * l);
  if (max_boxes < uniform) return SM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SM_ECUDA;
  }
  sm_quad *q = new sm_quad();
  q->dom = *dom;
  q->max_boxes = max_boxes;
  q->nu1 = nu1;
  q->nu2 = nu2;
  q->lbase = lb;
  q->lmax = lb + dom->max_level;
  q->stream = (cudaStream_t)stream;
  for (int f = 0; f < 4; ++f) {
    const bool axis = dom->geometry == SM_AXISYMMETRIC && f == 0;
    q->bc.type[f] = axis ? 0 : dom->bc_type[f];
    q->bc.g2[f] = axis ? 0.0 : 2.0 * dom->bc_val[f];
  }
  for (int l = 0; l < QMAXL; ++l) {
    q->h[l] = dom->length / (QN * (double)(1ll << l));
    q->inv_h2[l] = 1.0 / (q->h[l] * q->h[l]);
  }
  // uniform levels, each in Morton order
  for (int l = 0; l <= lb; ++l) {
    q->off[l] = n_boxes(q);
    const uint64_t nk = 1ull << (2 * l);
    for (uint64_t key = 0; key < nk; ++key) {
      int i = 0, j = 0;
      for (int b = 0; b < 31; ++b) {
        i |= (int)((key >> (2 * b)) & 1) << b;
        j |= (int)((key >> (2 * b + 1)) & 1) << b;
      }
      add_box(q, l, i, j, l ? q->off[l - 1] + (int)(key >> 2) : -1);
    }
    q->off[l + 1] = n_boxes(q);
  }
  for (int l = 0; l < lb; ++l)
    for (int b = q->off[l]; b < q->off[l + 1]; ++b)
      for (int c = 0; c < 4; ++c) q->chl[4 * b + c] = q->off[l + 1] + (int)((q->mort[b] << 2) | (uint64_t)c);
  q->nlev = lb + 1;
  for (int l = 0; l <= lb; ++l) set_neighbours(q, l);
  coarse_inverse(q);
  *out = q;
  return SM_OK;
}

extern "C" int sm_quad_destroy(sm_quad *q) {
  delete q;
  return SM_OK;
}

namespace {
struct QLayout {
  size_t lev, par, chl, nbr8, pn, ref, ij, w, wv, var[NV], cflux, ainv, lut, h, slots, err, snap, rg, need, fine,
      total;
};
QLayout qlayout(const sm_quad *q) {
  QLayout L{};
  size_t t = 0;
  auto take = [&](size_t bytes) {
    const size_t at = t;
    t = (t + bytes + 255) & ~(size_t)255;
    return at;
  };
  const size_t nb = (size_t)q->max_boxes;
  L.lev = take(sizeof(int) * nb);
  L.par = take(sizeof(int) * nb);
  L.chl = take(sizeof(int) * 4 * nb);
  L.nbr8 = take(sizeof(int) * 8 * nb);
  L.pn = take(sizeof(int) * 9 * nb);
  L.ref = take(sizeof(int) * nb);
  L.ij = take(sizeof(int2) * nb);
  L.w = take(sizeof(double) * 24 * nb);
  L.wv = take(sizeof(double) * 8 * nb);
  for (int v = 0; v < NV; ++v) L.var[v] = take(sizeof(double) * QC * nb);
  L.cflux = take(sizeof(double) * 32 * nb);
  L.ainv = take(sizeof(double) * QC * QC);
  L.lut = take(sizeof(double) * 3 * 4096);
  L.h = take(sizeof(double) * 3 * QMAXL);
  L.slots = take(sizeof(unsigned long long) * 8);
  L.err = take(sizeof(unsigned));
  L.snap = take(sizeof(double) * 6 * QC * nb);
  L.rg = take(sizeof(int) * 10 * nb);
  L.need = take(sizeof(unsigned long long) * nb);
  L.fine = take(nb);
  L.total = t;
  return L;
}
}  // namespace

extern "C" int sm_quad_arena_size(const sm_quad *q, size_t *bytes) {
  if (!q || !bytes) return SM_EINVAL;
  *bytes = qlayout(q).total;
  return SM_OK;
}

extern "C" int sm_quad_bind_arena(sm_quad *q, void *dev_ptr, size_t bytes) {
  if (!q || !dev_ptr) return SM_EINVAL;
  const QLayout L = qlayout(q);
  if (bytes < L.total) return qfail(q, SM_ENOMEM, "arena too small");
  if (((uintptr_t)dev_ptr & 255) != 0) return qfail(q, SM_EINVAL, "arena not 256-byte aligned");
  char *a = (char *)dev_ptr;
  drop_graphs(q);
  q->arena = a;
  q->d_lev = (int *)(a + L.lev);
  q->d_par = (int *)(a + L.par);
  q->d_chl = (int *)(a + L.chl);
  q->d_nbr8 = (int *)(a + L.nbr8);
  q->d_pn = (int *)(a + L.pn);
  q->d_ref = (int *)(a + L.ref);
  q->d_ij = (int2 *)(a + L.ij);
  q->d_w = (double *)(a + L.w);
  q->d_wv = (double *)(a + L.wv);
  for (int v = 0; v < NV; ++v) q->var[v] = (double *)(a + L.var[v]);
  q->cflux = (double *)(a + L.cflux);
  q->ainv = (double *)(a + L.ainv);
  q->lut = (double *)(a + L.lut);
  q->d_h = (double *)(a + L.h);
  q->slots = (unsigned long long *)(a + L.slots);
  q->d_err = (unsigned *)(a + L.err);
  q->snap = (double *)(a + L.snap);
  q->d_rg = (int *)(a + L.rg);
  q->d_need = (unsigned long long *)(a + L.need);
  q->d_fine = (unsigned char *)(a + L.fine);
  std::vector<double> hs(3 * QMAXL);
  for (int l = 0; l < QMAXL; ++l) {
    hs[l] = q->h[l];
    hs[QMAXL + l] = q->inv_h2[l];
    hs[2 * QMAXL + l] = 1.0 / q->h[l];
  }
  if (cudaMemsetAsync(a, 0, L.total, q->stream) != cudaSuccess ||
      cudaMemcpyAsync(q->ainv, q->h_ainv.data(), sizeof(double) * QC * QC, cudaMemcpyHostToDevice, q->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(q->d_h, hs.data(), sizeof(double) * 3 * QMAXL, cudaMemcpyHostToDevice, q->stream) !=
          cudaSuccess)
    return qfail(q, SM_ECUDA, "arena initialisation");
  return upload_tables(q);
}

extern "C" int sm_quad_refine_level(sm_quad *q, int level, const int8_t *flags, int *n_new, int *n_dropped) {
  SM_RANGE();
  if (!q || !flags) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  if (level != q->nlev - 1 || level >= q->lmax) return qfail(q, SM_ESTATE, "not the finest refinable level");
  std::vector<int> todo;
  int dropped = 0;
  for (int b = q->off[level]; b < q->off[level + 1]; ++b) {
    if (flags[b - q->off[level]] <= 0) continue;
    bool ok = true;
    for (int d = 0; d < 8; ++d) ok &= q->nbr8[8 * b + d] != -2;
    if (ok) todo.push_back(b);
    else ++dropped;
  }
  if ((long long)n_boxes(q) + 4ll * (long long)todo.size() > q->max_boxes)
    return qfail(q, SM_ENOMEM, "box capacity exceeded");
  const int start = n_boxes(q);
  for (int b : todo)
    for (int c = 0; c < 4; ++c) {
      const int nb = n_boxes(q);
      add_box(q, level + 1, 2 * q->ix[b] + (c & 1), 2 * q->iy[b] + (c >> 1), b);
      q->chl[4 * b + c] = nb;
    }
  if (n_new) *n_new = n_boxes(q) - start;
  if (n_dropped) *n_dropped = dropped;
  if (todo.empty()) return SM_OK;
  q->off[level + 2] = n_boxes(q);
  q->nlev = level + 2;
  set_neighbours(q, level + 1);
  drop_graphs(q);
  // the new boxes' fields start at zero
  for (int v = 0; v < NV; ++v)
    if (cudaMemsetAsync(q->var[v] + (size_t)start * QC, 0, sizeof(double) * QC * (size_t)(n_boxes(q) - start),
                        q->stream) != cudaSuccess)
      return qfail(q, SM_ECUDA, "memset");
  return upload_tables(q);
}

extern "C" int sm_quad_get_tables(const sm_quad *q, int *nb, int *nl, int32_t *level_offset, int32_t *level,
                                  int32_t *ij, uint64_t *morton, int32_t *parent, int32_t *child, int32_t *nbr) {
  if (!q) return SM_EINVAL;
  const int n = n_boxes(q);
  if (nb) *nb = n;
  if (nl) *nl = q->nlev;
  if (level_offset)
    for (int l = 0; l <= q->nlev; ++l) level_offset[l] = q->off[l];
  for (int b = 0; b < n; ++b) {
    if (level) level[b] = q->lev[b];
    if (ij) {
      ij[2 * b] = q->ix[b];
      ij[2 * b + 1] = q->iy[b];
    }
    if (morton) morton[b] = q->mort[b];
    if (parent) parent[b] = q->par[b];
    if (child)
      for (int c = 0; c < 4; ++c) child[4 * b + c] = q->chl[4 * b + c];
    if (nbr)
      for (int d = 0; d < 8; ++d) nbr[8 * b + d] = q->nbr8[8 * b + d];
  }
  return SM_OK;
}

extern "C" int sm_quad_var_ptr(sm_quad *q, int v, double **dev) {
  if (!q || !dev || v < 0 || v > V_RHO) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  *dev = q->var[v];
  return SM_OK;
}

extern "C" int sm_quad_upload(sm_quad *q, int v, const double *host) {
  if (!q || !host || v < 0 || v > V_RHO) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  if (cudaMemcpyAsync(q->var[v], host, sizeof(double) * QC * (size_t)n_boxes(q), cudaMemcpyHostToDevice,
                      q->stream) != cudaSuccess ||
      cudaStreamSynchronize(q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "upload");
  return SM_OK;
}

extern "C" int sm_quad_download(sm_quad *q, int v, double *host) {
  if (!q || !host || v < 0 || v > V_RHO) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  if (cudaMemcpyAsync(host, q->var[v], sizeof(double) * QC * (size_t)n_boxes(q), cudaMemcpyDeviceToHost,
                      q->stream) != cudaSuccess ||
      cudaStreamSynchronize(q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "download");
  return SM_OK;
}

extern "C" int sm_quad_set_table(sm_quad *q, int n, double e_max, const double *mu, const double *diff,
                                 const double *alpha) {
  if (!q || !mu || !diff || !alpha || n < 2 || n > 4096 || !(e_max > 0.0)) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  std::vector<double> t(3 * (size_t)n);
  std::memcpy(t.data(), mu, sizeof(double) * n);
  std::memcpy(t.data() + n, diff, sizeof(double) * n);
  std::memcpy(t.data() + 2 * n, alpha, sizeof(double) * n);
  if (cudaMemcpyAsync(q->lut, t.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, q->stream) != cudaSuccess ||
      cudaStreamSynchronize(q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "table upload");
  q->lut_n = n;
  q->lut_emax = e_max;
  return SM_OK;
}

extern "C" int sm_quad_charge_rhs(sm_quad *q, double c, double eps, int use_rho) {
  if (!q || !(eps > 0.0)) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  return charge(q, c, eps, use_rho);
}

extern "C" int sm_quad_fmg(sm_quad *q, double tol, int max_cycles, int *cycles, double *rel) {
  SM_RANGE();
  if (!q || max_cycles < 1 || !(tol >= 0.0)) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  const int top = q->nlev - 1;
  restrict_all(q, V_RHS);
  coarse_solve(q);
  for (int l = 1; l <= top; ++l) {
    const int n = level_count(q, l);
    k_q_prolong<<<blocks_for(n), QT, 0, q->stream>>>(q->off[l], n, l, q->var[V_PHI], q->var[V_OLD], 0, tabs(q),
                                                      q->bc, q->d_err);
    ++q->launches;
    if (int st = vcycle_g(q, l)) return st;
  }
  if (int st = check(q, "FMG")) return st;
  return solve_loop(q, tol, max_cycles, 1, cycles, rel);
}

extern "C" int sm_quad_solve(sm_quad *q, double tol, int max_cycles, int *cycles, double *rel) {
  SM_RANGE();
  if (!q || max_cycles < 1 || !(tol >= 0.0)) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  return solve_loop(q, tol, max_cycles, 0, cycles, rel);
}

extern "C" int sm_quad_vcycles(sm_quad *q, int n) {
  SM_RANGE();
  if (!q || n < 0) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  for (int c = 0; c < n; ++c)
    if (int st = vcycle_g(q, q->nlev - 1)) return st;
  return check(q, "V-cycle");
}

extern "C" int sm_quad_compute_field(sm_quad *q) {
  SM_RANGE();
  if (!q) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  return field(q);
}

extern "C" int sm_quad_dt_limit(sm_quad *q, double c, double eps, double *dt) {
  SM_RANGE();
  if (!q || !dt || !(eps > 0.0)) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  if (!q->lut_n) return qfail(q, SM_ESTATE, "no coefficient table");
  return dt_limit(q, c, eps, dt);
}

extern "C" int sm_quad_fluid_stage(sm_quad *q, double dt) {
  SM_RANGE();
  if (!q) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  if (!q->lut_n) return qfail(q, SM_ESTATE, "no coefficient table");
  restrict_all(q, V_NE);
  restrict_all(q, V_NI);
  if (int st = euler_stage(q, V_NE, V_NI, V_NE1, V_NI1, dt)) return st;
  const size_t bytes = sizeof(double) * QC * (size_t)n_boxes(q);
  if (cudaMemcpyAsync(q->var[V_NE], q->var[V_NE1], bytes, cudaMemcpyDeviceToDevice, q->stream) != cudaSuccess ||
      cudaMemcpyAsync(q->var[V_NI], q->var[V_NI1], bytes, cudaMemcpyDeviceToDevice, q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "copy");
  return SM_OK;
}

extern "C" int sm_quad_advance(sm_quad *q, double dt, double c, double eps, double tol, int max_cycles,
                               double *dt_next, int *cycles) {
  SM_RANGE();
  if (!q || !(eps > 0.0) || max_cycles < 1) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  if (!q->lut_n) return qfail(q, SM_ESTATE, "no coefficient table");
  const size_t bytes = sizeof(double) * QC * (size_t)n_boxes(q);
  const long long cells = (long long)n_boxes(q) * QC;
  restrict_all(q, V_NE);
  restrict_all(q, V_NI);
  if (cudaMemcpyAsync(q->var[V_NE0], q->var[V_NE], bytes, cudaMemcpyDeviceToDevice, q->stream) != cudaSuccess ||
      cudaMemcpyAsync(q->var[V_NI0], q->var[V_NI], bytes, cudaMemcpyDeviceToDevice, q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "copy");
  if (int st = euler_stage(q, V_NE0, V_NI0, V_NE, V_NI, dt)) return st;
  if (int st = charge(q, c, eps, 0)) return st;
  int c1 = 0, c2 = 0;
  const int st1 = solve_loop(q, tol, max_cycles, 0, &c1, nullptr);
  if (st1 && st1 != SM_ENOCONV) return st1;
  if (int st = field(q)) return st;
  double dtn = 0.0;
  if (int st = dt_limit(q, c, eps, &dtn)) return st;
  if (int st = euler_stage(q, V_NE, V_NI, V_NE1, V_NI1, dt)) return st;
  k_q_average<<<(int)((cells + 255) / 256), 256, 0, q->stream>>>(cells, q->var[V_NE], q->var[V_NE0], q->var[V_NE1]);
  k_q_average<<<(int)((cells + 255) / 256), 256, 0, q->stream>>>(cells, q->var[V_NI], q->var[V_NI0], q->var[V_NI1]);
  q->launches += 2;
  if (int st = charge(q, c, eps, 0)) return st;
  const int st2 = solve_loop(q, tol, max_cycles, 0, &c2, nullptr);
  if (st2 && st2 != SM_ENOCONV) return st2;
  if (int st = field(q)) return st;
  if (dt_next) *dt_next = dtn;
  if (cycles) {
    cycles[0] = c1;
    cycles[1] = c2;
  }
  if (cudaStreamSynchronize(q->stream) != cudaSuccess) return qfail(q, SM_ECUDA, "advance");
  return st1 ? st1 : st2;
}

// Eq. 8 with buffer and derefinement flags (the rules of the 3-D form on
// the quadtree): the per-cell test on the GPU, the buffer (same-level leaf
// neighbours within `buffer` cells, Chebyshev distance) on the host from
// the per-box masks
extern "C" int sm_quad_refine_flags(sm_quad *q, double c0, double c1, double c0_deref, double dx_deref, int buffer,
                                    int8_t *flags) {
  SM_RANGE();
  if (!q || !flags || buffer < 0 || buffer > QN) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  if (!q->lut_n) return qfail(q, SM_ESTATE, "no coefficient table");
  const int n = n_boxes(q);
  const double de = q->lut_emax / (q->lut_n - 1);
  qlaunch(q, k_q_refcrit, blocks_for(n), QT, n, (const double *)q->var[V_EMAG], tabs(q),
          (const double *)(q->lut + 2 * q->lut_n), q->lut_n, de, c1, c0 * c1, c0_deref * c1, dx_deref,
          (const double *)q->d_h, q->d_need, q->d_fine);
  std::vector<unsigned long long> need(n);
  std::vector<unsigned char> fine(n);
  if (cudaMemcpyAsync(need.data(), q->d_need, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, q->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(fine.data(), q->d_fine, n, cudaMemcpyDeviceToHost, q->stream) != cudaSuccess ||
      cudaStreamSynchronize(q->stream) != cudaSuccess)
    return qfail(q, SM_ECUDA, "refinement test");
  // cells of a neighbour in direction (dx, dy) within `buffer` cells of the box
  auto axis_ok = [&](int d, int i) { return d < 0 ? i >= QN - buffer : (d > 0 ? i <= buffer - 1 : true); };
  unsigned long long mask[8];
  for (int dy = -1, k = 0; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      if (!dx && !dy) continue;
      unsigned long long m = 0;
      for (int c = 0; c < QC; ++c)
        if (axis_ok(dx, c % QN) && axis_ok(dy, c / QN)) m |= 1ull << c;
      mask[k++] = m;
    }
  for (int b = 0; b < n; ++b) {
    flags[b] = 0;
    if (q->chl[4 * b] >= 0) continue;
    bool marked = need[b] != 0;
    for (int d = 0; d < 8 && !marked; ++d) {
      const int nb = q->nbr8[8 * b + d];
      if (nb >= 0 && q->chl[4 * nb] < 0 && (need[nb] & mask[d])) marked = true;
    }
    if (marked) {
      if (q->lev[b] < q->lmax) flags[b] = 1;
    } else if (fine[b] && q->lev[b] > q->lbase) {
      flags[b] = -1;
    }
  }
  return SM_OK;
}

// The new box set, its tables and the move descriptors are formed on the
// device (k_qrg_*); the host reads the request counts and per-level list
// sizes once, then the new tables for its own copy of the mesh.
extern "C" int sm_quad_regrid(sm_quad *q, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped) {
  SM_RANGE();
  if (!q || !flags) return SM_EINVAL;
  if (!q->arena) return qfail(q, SM_ESTATE, "no arena bound");
  const int n = n_boxes(q), M = q->max_boxes, L0 = q->nlev, T = 256;
  cudaStream_t s = q->stream;
  restrict_all(q, V_NE);
  restrict_all(q, V_NI);
  // scratch in the per-call work fields (V_OLD onwards: nothing there
  // outlives a call)
  char *wp = reinterpret_cast<char *>(q->var[V_OLD]);
  auto take = [&](size_t bytes) {
    char *p = wp;
    wp += (bytes + 255) & ~(size_t)255;
    return p;
  };
  int8_t *dflags = (int8_t *)take((size_t)n);
  int *refv = (int *)take(4 * (size_t)n), *keepv = (int *)take(4 * (size_t)n), *derv = (int *)take(4 * (size_t)n);
  int *ref_pos = (int *)take(4 * ((size_t)n + 1)), *keep_pos = (int *)take(4 * ((size_t)n + 1));
  uint64_t *ref_keys = (uint64_t *)take(8 * (size_t)n), *kept_keys = (uint64_t *)take(8 * (size_t)n);
  int *nlev = (int *)take(4 * (size_t)M);
  int2 *nij = (int2 *)take(8 * (size_t)M);
  uint64_t *nkey = (uint64_t *)take(8 * (size_t)M);
  int *cnt = (int *)take(8), *counts = (int *)take(4 * (2 * QMAXL + 8));
  const int gb = (n + T - 1) / T;
  if (cudaMemcpyAsync(dflags, flags, (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(cnt, 0, 8, s) != cudaSuccess)
    return qfail(q, SM_ECUDA, "regrid flags");
  k_qrg_refine<<<gb, T, 0, s>>>(n, q->d_lev, q->d_chl, q->d_nbr8, dflags, q->lmax, refv, cnt);
  k_qrg_derefine<<<gb, T, 0, s>>>(n, q->d_chl, q->d_par, q->d_nbr8, dflags, refv, derv, cnt);
  k_qrg_keep<<<gb, T, 0, s>>>(n, q->d_par, derv, keepv);
  k_qrg_scan2<<<dim3(1, 2), 1024, 0, s>>>(refv, ref_pos, keepv, keep_pos, n);
  QOffsets off{};
  for (int l = 0; l <= L0; ++l) off.v[l] = q->off[l];
  k_qrg_counts<<<1, 32, 0, s>>>(cnt, keep_pos, ref_pos, off, L0, counts);
  q->launches += 5;
  std::vector<int> hc(3 + 2 * L0 + 1);
  if (int st = check(q, "regrid decisions")) return st;
  if (cudaMemcpyAsync(hc.data(), counts, sizeof(int) * hc.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return qfail(q, SM_ECUDA, "regrid counts");
  const int *hk = &hc[2], *hr = &hc[3 + L0];
  const int nref = hr[L0], nder = hc[1];
  if (n_refined) *n_refined = nref;
  if (n_derefined) *n_derefined = nder;
  if (n_dropped) *n_dropped = hc[0];
  if (nref == 0 && nder == 0) return SM_OK;
  QRgLevels L{};
  int nlevels = 0, m = 0;
  for (int l = 0; l < QMAXL + 2; ++l) {
    const int kept = l < L0 ? hk[l + 1] - hk[l] : 0;
    const int born = (l >= 1 && l - 1 < L0) ? 4 * (hr[l] - hr[l - 1]) : 0;
    L.kept[l] = l <= L0 ? hk[l] : hk[L0];
    L.ref[l] = l <= L0 ? hr[l] : hr[L0];
    L.nw[l] = m;
    m += kept + born;
    if (kept + born > 0) nlevels = l + 1;
  }
  if (m > M) return qfail(q, SM_ENOMEM, "box capacity exceeded");
  k_qrg_keys<<<gb, T, 0, s>>>(n, q->d_ij, keepv, keep_pos, refv, ref_pos, kept_keys, ref_keys);
  k_qrg_place<<<(4 * n + T - 1) / T, T, 0, s>>>(n, q->d_lev, q->d_ij, q->d_nbr8, keepv, keep_pos, refv, ref_pos,
                                               kept_keys, ref_keys, L, nlev, nij, nkey, q->d_rg);
  q->launches += 2;
  // snapshot of the old fields (the move writes the same arrays)
  const int vars[6] = {V_PHI, V_NE, V_NI, V_RHS, V_EMAG, V_RHO};
  const size_t stride = (size_t)M * QC;
  for (int v = 0; v < 6; ++v)
    if (cudaMemcpyAsync(q->snap + v * stride, q->var[vars[v]], sizeof(double) * QC * (size_t)n,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return qfail(q, SM_ECUDA, "regrid snapshot");
  // the new tables in place of the old ones
  if (cudaMemcpyAsync(q->d_lev, nlev, sizeof(int) * m, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(q->d_ij, nij, sizeof(int2) * m, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return qfail(q, SM_ECUDA, "regrid tables");
  const int gm = (m + T - 1) / T, gm8 = (8 * m + T - 1) / T;
  k_qrg_links<<<gm, T, 0, s>>>(m, nlev, nkey, L, nlevels, q->d_par, q->d_chl);
  k_qrg_nbr<<<gm8, T, 0, s>>>(m, nlev, nij, nkey, L, q->d_nbr8);
  k_qrg_derived<<<gm8, T, 0, s>>>(m, q->dom.geometry == SM_AXISYMMETRIC, q->d_par, q->d_chl, q->d_nbr8, q->d_ij,
                                  q->d_pn, q->d_ref, q->d_w, q->d_wv);
  q->launches += 3;
  if (int st = check(q, "regrid tables")) return st;
  drop_graphs(q);
  k_q_regrid_move<<<blocks_for(m), QT, 0, s>>>(m, q->d_rg, q->snap, stride, q->var[V_PHI], q->var[V_NE],
                                               q->var[V_NI], q->var[V_RHS], q->var[V_EMAG], q->var[V_RHO], tabs(q),
                                               q->bc, q->d_err);
  ++q->launches;
  // the host's copy of the new mesh
  std::vector<int2> hij(m);
  q->lev.resize(m);
  q->par.resize(m);
  q->chl.resize(4 * (size_t)m);
  q->nbr8.resize(8 * (size_t)m);
  q->mort.resize(m);
  unsigned ev = 0;
  if (cudaMemcpyAsync(q->lev.data(), q->d_lev, sizeof(int) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hij.data(), q->d_ij, sizeof(int2) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(q->par.data(), q->d_par, sizeof(int) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(q->chl.data(), q->d_chl, sizeof(int) * 4 * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(q->nbr8.data(), q->d_nbr8, sizeof(int) * 8 * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(q->mort.data(), nkey, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&ev, q->d_err, sizeof(ev), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return qfail(q, SM_ECUDA, "regrid move");
  q->ix.resize(m);
  q->iy.resize(m);
  for (int b = 0; b < m; ++b) {
    q->ix[b] = hij[b].x;
    q->iy[b] = hij[b].y;
  }
  q->nlev = nlevels;
  for (int l = 0; l <= QMAXL + 1; ++l) q->off[l] = l <= nlevels ? L.nw[l] : m;
  if (ev) return qfail(q, SM_ESTATE, "a coarse box needed by the regrid prolongation is missing");
  return SM_OK;
}

extern "C" int sm_quad_set_graphs(sm_quad *q, int on) {
  if (!q) return SM_EINVAL;
  q->graphs = on != 0;
  return SM_OK;
}

extern "C" int sm_quad_set_pdl(sm_quad *q, int on) {
  if (!q) return SM_EINVAL;
  q->pdl = on != 0;
  drop_graphs(q);
  return SM_OK;
}

extern "C" int sm_quad_launch_count(const sm_quad *q, long long *n) {
  if (!q || !n) return SM_EINVAL;
  *n = q->launches;
  return SM_OK;
}

extern "C" const char *sm_quad_last_error(const sm_quad *q) { return q ? q->err.c_str() : "null context"; }
