// multigrid.cu -- geometric multigrid for Poisson's equation on the octree
// (Sec. 2.1.2, Eq. 1 and 5): full approximation scheme V-cycle and full
// multigrid, red-black Gauss-Seidel smoothing of the 7-point cell-centred
// Laplacian, 8-child averaging restriction, 4-point linear prolongation,
// coarse-to-fine ghost interpolation and an exact solve on level 0.
//
// The level kernels are templates on the value type: FP64 for the plain
// solve, FP32 for the error equation of the mixed-precision form, whose
// outer defect-correction loop (residual, accumulation, level-0 solve)
// stays in FP64.
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include "sm_internal.cuh"
#include "sm_nvtx.h"

using namespace sm;

// ---------------------------------------------------------------------------
// per-box work of the level operations
// ---------------------------------------------------------------------------
//
// Every level operation processes one 8^3 box with a group of GT threads.
// In the per-level kernels the group is the whole block (barrier 0); in the
// persistent kernel it is one of the PGROUPS groups of a block (named
// barriers 1..PGROUPS), each taking boxes in turn.

constexpr int GT = 128;             // threads of a box group
constexpr int CPT = CELLS / GT;     // cells per thread
constexpr int RPT = CELLS / 2 / GT; // cells of one colour per thread
constexpr int NSL = GT / 64;        // 64-thread slices of a group (one face cell each)
constexpr int FPS = 6 / NSL;        // faces per slice
constexpr int PGROUPS = 8;          // box groups per block of the persistent kernel
static_assert(CELLS % GT == 0 && 6 % NSL == 0, "group size");

struct Grp {
  int t;    // thread within the group
  int bar;  // hardware barrier of the group
  __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(GT) : "memory"); }
};

// position of interior cell c (i + 8j + 64k) in a 10^3 staging array
__device__ __forceinline__ int s10(int c) { return ((c & 7) + 1) + 10 * (((c >> 3) & 7) + 1) + 100 * ((c >> 6) + 1); }

// interior cell next to face f at face coordinates (u, w): u runs along
// axis (a+1)%3 and w along (a+2)%3 of the face axis a
__device__ __forceinline__ int face_cell(int f, int u, int w) {
  const int a = f >> 1, e = (f & 1) ? NC - 1 : 0;
  return a == 0 ? cidx(e, u, w) : (a == 1 ? cidx(w, e, u) : cidx(u, w, e));
}

// neighbour-table entries of the faces a thread fills while staging box b
// (face f belongs to the 64-thread slice f mod NSL); the tables do not
// change during a solve, so kernels read them before waiting on their
// predecessor
struct Nb {
  int v[FPS];
};

__device__ __forceinline__ Nb load_nb(const Grp &g, const int32_t *__restrict__ nbr6, int b) {
  Nb nb;
  const int slice = g.t >> 6;
#pragma unroll
  for (int f = 0; f < 6; ++f)
    if (f % NSL == slice) nb.v[f / NSL] = __ldg(nbr6 + 6 * b + f);
  return nb;
}

// Stage box b of variable v and its six face halos in s[1000] (10^3, one
// ghost layer).  Ghost values follow pot_ghost: the same-level neighbour
// cell, the physical-boundary ghost (Dirichlet 2g - inner, -inner when
// homogeneous, Neumann inner) or inner/3 + 2 phihat/3 at a refinement face.
// The neighbour-table, neighbour-cell and phihat loads are issued together
// with the interior loads; face f is filled by the 64-thread slice f mod NSL.
// With color >= 0 only the halo cells next to interior cells of that colour
// ((i+j+k) % 2 == color) are filled: a colour pass reads no others.
template <typename T>
__device__ __forceinline__ void stage_box(const Grp &g, T *s, const T *v, const Nb &nbv, const T *gh, int b,
                                          const Bc &bc, int homog, int color = -1) {
  const T *p = v + (size_t)b * CELLS;
  T x[CPT];
#pragma unroll
  for (int h = 0; h < CPT; ++h) x[h] = p[g.t + h * GT];
  const int slice = g.t >> 6, u = g.t & 7, w = (g.t >> 3) & 7;
  T hv[FPS];
  // colour of the interior face cell (u, w) of face f: u + w + (0 or 7)
  const int cw = (u + w) & 1;
  auto used = [&](int f) { return color < 0 || ((cw + ((f & 1) ? 1 : 0)) & 1) == color; };
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (f % NSL != slice || !used(f)) continue;
    const int r = f / NSL;
    const int nb = nbv.v[r];
    if (nb >= 0) hv[r] = v[(size_t)nb * CELLS + face_cell(f ^ 1, u, w)];
    else if (nb == -2) hv[r] = gh[(size_t)(6 * b + f) * FACE + u + NC * w];
    else hv[r] = T(0);
  }
  g.sync();  // earlier users of s are done
#pragma unroll
  for (int h = 0; h < CPT; ++h) s[s10(g.t + h * GT)] = x[h];
  g.sync();
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (f % NSL != slice || !used(f)) continue;
    const int r = f / NSL, a = f >> 1;
    const int q = s10(face_cell(f, u, w));
    const int stride = a == 0 ? 1 : (a == 1 ? 10 : 100);
    const T inner = s[q];
    T gv;
    if (nbv.v[r] >= 0) gv = hv[r];
    else if (nbv.v[r] == -1) gv = bc.type[f] ? (homog ? T(0) : bc_g2<T>(bc, f)) - inner : inner;
    else gv = inner * T(1.0 / 3.0) + T(2.0 / 3.0) * hv[r];
    s[q + ((f & 1) ? stride : -stride)] = gv;
  }
  g.sync();
}

// sum of the six neighbours from a staged box (order -x,+x,-y,+y,-z,+z)
template <typename T>
__device__ __forceinline__ T staged_sum(const T *s, int q) {
  return s[q - 1] + s[q + 1] + s[q - 10] + s[q + 10] + s[q - 100] + s[q + 100];
}

// One colour of a red-black Gauss-Seidel sweep on box b: phi = (sum of 6
// neighbours - h^2 f)/6 on the cells with (i+j+k) % 2 == color (level-global
// parity; box origins are multiples of 8).
// Gauss-Seidel value of staged cell c: (sum of 6 neighbours - h^2 f) / 6
template <typename T>
__device__ __forceinline__ T rbgs_value(const T *s, int c, T f, T h2) {
  return (staged_sum(s, s10(c)) - h2 * f) * T(1.0 / 6.0);
}

// natural index of the n-th cell of a colour in a box
__device__ __forceinline__ int colour_cell(int n, int color) {
  const int k = n >> 5, j = (n >> 2) & 7;
  return cidx(((n & 3) << 1) | ((j + k + color) & 1), j, k);
}

template <typename T>
__device__ __forceinline__ void rbgs_box(const Grp &g, T *s, int b, int color, T *phi, const T *rhs, const T *gh,
                                         const Nb &nb, const Bc &bc, T h2, int homog) {
  const size_t base = (size_t)b * CELLS;
  int c[RPT];
  T f[RPT];
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    c[h] = colour_cell(g.t + h * GT, color);
    f[h] = rhs[base + c[h]];
  }
  stage_box(g, s, phi, nb, gh, b, bc, homog, color);
#pragma unroll
  for (int h = 0; h < RPT; ++h) phi[base + c[h]] = rbgs_value(s, c[h], f[h], h2);
}

// parent of box b and the octant of the parent that b covers
struct Place {
  int P, ox, oy, oz;
};

__device__ __forceinline__ Place load_place(const int32_t *__restrict__ parent, const int32_t *__restrict__ ijk,
                                            int b) {
  return Place{__ldg(parent + b), __ldg(ijk + 3 * b) & 1, __ldg(ijk + 3 * b + 1) & 1, __ldg(ijk + 3 * b + 2) & 1};
}

// Residual r = f - L phi of box b (level l) and restriction: the 64 cells
// of the parent region get the 8-child averages of phi (into phi) and of r
// (into rhs, completed to the FAS right-hand side by fas_box).
template <typename T>
__device__ __forceinline__ void resid_restrict_box(const Grp &g, T *s, T *sr, int b, T *phi, T *rhs, const T *gh,
                                                   const Nb &nb, const Place &pl, const Bc &bc, T inv_h2,
                                                   int homog, T *old = nullptr) {
  const size_t base = (size_t)b * CELLS;
  T f[CPT];
#pragma unroll
  for (int h = 0; h < CPT; ++h) f[h] = rhs[base + g.t + h * GT];
  stage_box(g, s, phi, nb, gh, b, bc, homog);
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const int q = s10(g.t + h * GT);
    sr[g.t + h * GT] = f[h] - (staged_sum(s, q) - T(6) * s[q]) * inv_h2;
  }
  g.sync();
  if (g.t >= 64) return;
  const int ci = g.t & 3, cj = (g.t >> 2) & 3, ck = g.t >> 4;
  T ap = 0, ar = 0;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int c = cidx(2 * ci + di, 2 * cj + dj, 2 * ck + dk);
        ap += s[s10(c)];
        ar += sr[c];
      }
  const size_t cc = (size_t)pl.P * CELLS + cidx(4 * pl.ox + ci, 4 * pl.oy + cj, 4 * pl.oz + ck);
  const T v = ap * T(0.125);
  phi[cc] = v;
  if (old) old[cc] = v;
  rhs[cc] = ar * T(0.125);
}

// After restriction into box b (level l-1): keep a copy of phi, and on a
// refined box complete the FAS right-hand side f = avg(r_fine) + L phi.
// FAS step of a refined box already staged in s: old = phi, rhs += L phi
template <typename T>
__device__ __forceinline__ void fas_staged(const Grp &g, const T *s, int b, T *old, T *rhs, T inv_h2) {
  const size_t base = (size_t)b * CELLS;
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const int c = g.t + h * GT, q = s10(c);
    const T p = s[q];
    old[base + c] = p;
    rhs[base + c] += (staged_sum(s, q) - T(6) * p) * inv_h2;
  }
}

template <typename T>
__device__ __forceinline__ void fas_box(const Grp &g, T *s, int b, T *phi, T *old, T *rhs, const T *gh,
                                        const Nb &nb, bool refined, const Bc &bc, T inv_h2, int homog) {
  const size_t base = (size_t)b * CELLS;
  if (!refined) {
#pragma unroll
    for (int h = 0; h < CPT; ++h) old[base + g.t + h * GT] = phi[base + g.t + h * GT];
    return;
  }
  stage_box(g, s, phi, nb, gh, b, bc, homog);
  fas_staged(g, s, b, old, rhs, inv_h2);
}

// plain 8-child average of one or two variables from box b into its parent
template <typename T>
__device__ __forceinline__ void restrict1_box(const Grp &g, int b, const Place &pl, T *a, T *a2) {
  if (g.t >= 64) return;
  const int ci = g.t & 3, cj = (g.t >> 2) & 3, ck = g.t >> 4;
  const size_t fb = (size_t)b * CELLS;
  T s = 0, s2 = 0;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int c = cidx(2 * ci + di, 2 * cj + dj, 2 * ck + dk);
        s += a[fb + c];
        if (a2) s2 += a2[fb + c];
      }
  const size_t cc = (size_t)pl.P * CELLS + cidx(4 * pl.ox + ci, 4 * pl.oy + cj, 4 * pl.oz + ck);
  a[cc] = s * T(0.125);
  if (a2) a2[cc] = s2 * T(0.125);
}

// Value of a coarse-level quantity at local cell (q0,q1,q2) of box Q where
// the cell may lie one step outside the box along axis E (direction S):
// the neighbour box of the same level, or the physical-boundary ghost
// wall(f, ctr) of the cell `ctr` it left.  E and S are compile-time so that
// the boundary table is indexed by constants.
template <int E, int S, typename T, typename F, typename W>
__device__ __forceinline__ T coarse_at(F val, W wall, const int32_t *__restrict__ nbr6, int Q, int q0, int q1, int q2,
                                       T ctr, unsigned long long *err) {
  const int qe = E == 0 ? q0 : (E == 1 ? q1 : q2);
  if (qe >= 0 && qe < NC) return val(Q, cidx(q0, q1, q2));
  constexpr int f = 2 * E + (S > 0);
  const int Qn = __ldg(nbr6 + 6 * Q + f);
  if (Qn >= 0) {
    const int w = S > 0 ? 0 : NC - 1;
    return val(Qn, cidx(E == 0 ? w : q0, E == 1 ? w : q1, E == 2 ? w : q2));
  }
  if (Qn == -1) return wall(f, ctr);
  atomicOr(err, 1ull);  // nesting violated: no coarse box where one must be
  return ctr;
}

// coarse_at with a run-time direction s along compile-time axis E
template <int E, typename T, typename F, typename W>
__device__ __forceinline__ T coarse_step(F val, W wall, const int32_t *__restrict__ nbr6, int Q, int q0, int q1,
                                         int q2, int s, T ctr, unsigned long long *err) {
  if (s > 0)
    return coarse_at<E, 1, T>(val, wall, nbr6, Q, q0 + (E == 0), q1 + (E == 1), q2 + (E == 2), ctr, err);
  return coarse_at<E, -1, T>(val, wall, nbr6, Q, q0 - (E == 0), q1 - (E == 1), q2 - (E == 2), ctr, err);
}

// The three level l-1 values behind ghost cell (u,w) of refinement face F
// of box b (level l): the coarse cell c containing the ghost and its two
// tangential neighbours c1, c2 on the ghost's side.  False (error bit 2
// set) when the parent has no neighbour across F.
template <int F, typename T, typename V, typename W>
__device__ __forceinline__ bool cf_coarse3(V val, W wall, const int32_t *__restrict__ nbr6,
                                           const int32_t *__restrict__ parent, const int32_t *__restrict__ ijk, int b,
                                           int u, int w, unsigned long long *err, T &c, T &c1, T &c2) {
  constexpr int a = F >> 1, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  int G[3];
  G[a] = NC * __ldg(ijk + 3 * b + a) + ((F & 1) ? NC : -1);
  G[t1] = NC * __ldg(ijk + 3 * b + t1) + u;
  G[t2] = NC * __ldg(ijk + 3 * b + t2) + w;
  const int P = __ldg(parent + b);
  const int Q = __ldg(nbr6 + 6 * P + F);
  if (Q < 0) {
    atomicOr(err, 2ull);
    return false;
  }
  const int l0 = (G[0] >> 1) - NC * __ldg(ijk + 3 * Q), l1 = (G[1] >> 1) - NC * __ldg(ijk + 3 * Q + 1),
            l2 = (G[2] >> 1) - NC * __ldg(ijk + 3 * Q + 2);
  c = val(Q, cidx(l0, l1, l2));
  c1 = coarse_step<t1, T>(val, wall, nbr6, Q, l0, l1, l2, (G[t1] & 1) ? 1 : -1, c, err);
  c2 = coarse_step<t2, T>(val, wall, nbr6, Q, l0, l1, l2, (G[t2] & 1) ? 1 : -1, c, err);
  return true;
}

// phihat = c/2 + c_t1/4 + c_t2/4 for ghost cell (u,w) of refinement face F
// of box b (level l), from the level l-1 values of v
template <int F, typename T>
__device__ __forceinline__ void cf_value(const T *v, T *gh, const int32_t *__restrict__ nbr6,
                                         const int32_t *__restrict__ parent, const int32_t *__restrict__ ijk,
                                         const Bc &bc, int homog, int b, int u, int w, unsigned long long *err) {
  auto val = [&](int Q, int c) { return v[(size_t)Q * CELLS + c]; };
  auto wall = [&](int f, T ctr) { return bc.type[f] ? (homog ? T(0) : bc_g2<T>(bc, f)) - ctr : ctr; };
  T c, c1, c2;
  if (!cf_coarse3<F, T>(val, wall, nbr6, parent, ijk, b, u, w, err, c, c1, c2)) return;
  T ph = T(0.5) * c;
  ph += T(0.25) * c1;
  ph += T(0.25) * c2;
  gh[(size_t)(6 * b + F) * FACE + u + NC * w] = ph;
}

// coarse interpolation values of the refinement faces of box b, cells
// (u,w) = (e & 7, e >> 3) for the face-cell index e of this thread
template <typename T>
__device__ __forceinline__ void cf_faces_box(int e, int nthreads, const T *v, T *gh, const int32_t *__restrict__ nbr6,
                                             const int32_t *__restrict__ parent, const int32_t *__restrict__ ijk,
                                             const Bc &bc, int homog, int b, unsigned long long *err) {
  // thread e handles face cells e, e + nthreads, ... of the 6 x 64 list
  const int u = e & 7, w = (e >> 3) & 7, first = e >> 6, step = nthreads >> 6;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (f < first || (f - first) % step) continue;
    if (__ldg(nbr6 + 6 * b + f) != -2) continue;
    switch (f) {
      case 0: cf_value<0>(v, gh, nbr6, parent, ijk, bc, homog, b, u, w, err); break;
      case 1: cf_value<1>(v, gh, nbr6, parent, ijk, bc, homog, b, u, w, err); break;
      case 2: cf_value<2>(v, gh, nbr6, parent, ijk, bc, homog, b, u, w, err); break;
      case 3: cf_value<3>(v, gh, nbr6, parent, ijk, bc, homog, b, u, w, err); break;
      case 4: cf_value<4>(v, gh, nbr6, parent, ijk, bc, homog, b, u, w, err); break;
      default: cf_value<5>(v, gh, nbr6, parent, ijk, bc, homog, b, u, w, err); break;
    }
  }
}

// Prolongation into box b (level l) and the coarse interpolation values of
// its refinement faces (both read only level l-1): mode 0 adds the
// correction (phi - old) with homogeneous wall ghosts, mode 1 overwrites
// with the prolonged solution (FMG); gh interpolates phi itself.  homog:
// the variable is an error (homogeneous wall ghosts everywhere).
//
// The coarse values of the 4^3 cells under b and of their face neighbours
// (6^3 region without edges and corners) are staged once in sp[216]; each
// thread then forms four of the eight fine values of one coarse cell from
// the shared partial sums (c + c_x) and (c + c_x + c_y), which keeps the
// summation order ((c + c_x) + c_y) + c_z of the 4-point stencil.
template <typename T>
__device__ __forceinline__ void prolong_box(const Grp &g, T *sp, int b, int mode, T *phi, const T *old, T *gh,
                                            const int32_t *__restrict__ nbr6, const int32_t *__restrict__ parent,
                                            const int32_t *__restrict__ ijk, const Bc &bc, int homog,
                                            unsigned long long *err) {
  const int P = __ldg(parent + b);
  const int o[3] = {__ldg(ijk + 3 * b) & 1, __ldg(ijk + 3 * b + 1) & 1, __ldg(ijk + 3 * b + 2) & 1};
  auto val = [&](int Q, int c) {
    const size_t x = (size_t)Q * CELLS + c;
    return mode ? phi[x] : phi[x] - old[x];
  };
  const int hom = (mode && !homog) ? 0 : 1;
  auto reg = [](int x, int y, int z) { return x + 6 * y + 36 * z; };
  // interior of the region: the 64 coarse cells under b
  if (g.t < 64) {
    const int x = g.t & 3, y = (g.t >> 2) & 3, z = g.t >> 4;
    sp[reg(x + 1, y + 1, z + 1)] = val(P, cidx(4 * o[0] + x, 4 * o[1] + y, 4 * o[2] + z));
  }
  // face layers: 16 cells per face, face F by threads [slot, slot + 16)
#pragma unroll
  for (int F = 0; F < 6; ++F) {
    const int slot = F < 4 ? 64 + 16 * F : 16 * (F - 4);
    if (g.t < slot || g.t >= slot + 16) continue;
    const int E = F >> 1, S = (F & 1) ? 1 : -1;
    const int u = (g.t - slot) & 3, w = (g.t - slot) >> 2;
    // region coordinates: the layer along E, (u, w) along the other axes
    int rc[3], lc[3];
    rc[E] = S > 0 ? 5 : 0;
    rc[(E + 1) % 3] = u + 1;
    rc[(E + 2) % 3] = w + 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) lc[d] = 4 * o[d] - 1 + rc[d];
    T v;
    if (lc[E] >= 0 && lc[E] < NC) {
      v = val(P, cidx(lc[0], lc[1], lc[2]));
    } else {
      const int Qn = __ldg(nbr6 + 6 * P + F);
      if (Qn >= 0) {
        lc[E] = S > 0 ? 0 : NC - 1;
        v = val(Qn, cidx(lc[0], lc[1], lc[2]));
      } else {
        lc[E] -= S;  // the coarse cell inside P next to the boundary
        const T ctr = val(P, cidx(lc[0], lc[1], lc[2]));
        if (Qn == -1) {
          v = bc.type[F] ? (hom ? T(0) : bc_g2<T>(bc, F)) - ctr : ctr;
        } else {
          atomicOr(err, 1ull);  // nesting violated: no coarse box where one must be
          v = ctr;
        }
      }
    }
    sp[reg(rc[0], rc[1], rc[2])] = v;
  }
  g.sync();
  {
    const int cc = g.t >> 1, dx = g.t & 1;
    const int ci = cc & 3, cj = (cc >> 2) & 3, ck = cc >> 4;
    const int q = reg(ci + 1, cj + 1, ck + 1);
    const T A = sp[q] + sp[q + (dx ? 1 : -1)];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const T B = A + sp[q + (dy ? 6 : -6)];
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        const T sum = B + sp[q + (dz ? 36 : -36)];
        const size_t x = (size_t)b * CELLS + cidx(2 * ci + dx, 2 * cj + dy, 2 * ck + dz);
        if (mode) phi[x] = T(0.25) * sum;
        else phi[x] += T(0.25) * sum;
      }
    }
  }
  cf_faces_box(g.t, GT, phi, gh, nbr6, parent, ijk, bc, homog, b, err);
  g.sync();  // sp is free again
}

// Exact solve on level 0 (one 8^3 box), always in FP64: fold the Dirichlet
// boundary values into the right-hand side (not for the homogeneous error
// equation), transform to the separable eigenbasis, divide by the
// eigenvalues of the 7-point operator, transform back.  NT threads (t0 the
// thread's index, sync their barrier); sm: 2 x 512 + 216 doubles of shared
// memory.
template <int NT, typename Sync, typename In, typename Out>
__device__ __forceinline__ void coarse_box_io(int t0, Sync sync, double *sm, In rhs_of, Out store,
                                              const double *__restrict__ basis, const Bc &bc, double h2,
                                              double inv_h2, int homog) {
  double *x = sm, *y = sm + CELLS, *V = sm + 2 * CELLS, *lam = V + 192;
  for (int i = t0; i < 216; i += NT) {
    if (i < 192) V[i] = __ldg(basis + i);
    else lam[i - 192] = __ldg(basis + i);
  }
#pragma unroll
  for (int h = 0; h < CELLS / NT; ++h) {
    const int t = t0 + h * NT;
    const int c[3] = {t & 7, (t >> 3) & 7, t >> 6};
    double r = rhs_of(t);
    if (!homog) {
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const int q = c[f >> 1] + ((f & 1) ? 1 : -1);
        if ((q < 0 || q >= NC) && bc.type[f]) r -= 2.0 * bc.val[f] * inv_h2;
      }
    }
    x[t] = r;
  }
  sync();
  // forward: coefficients along x, then y, then z
#pragma unroll
  for (int h = 0; h < CELLS / NT; ++h) {
    const int t = t0 + h * NT, c0 = t & 7, c1 = (t >> 3) & 7, c2 = t >> 6;
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[0 * 64 + m * 8 + c0] * x[cidx(m, c1, c2)];
    y[t] = acc;
  }
  sync();
#pragma unroll
  for (int h = 0; h < CELLS / NT; ++h) {
    const int t = t0 + h * NT, c0 = t & 7, c1 = (t >> 3) & 7, c2 = t >> 6;
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[1 * 64 + m * 8 + c1] * y[cidx(c0, m, c2)];
    x[t] = acc;
  }
  sync();
#pragma unroll
  for (int h = 0; h < CELLS / NT; ++h) {
    const int t = t0 + h * NT, c0 = t & 7, c1 = (t >> 3) & 7, c2 = t >> 6;
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[2 * 64 + m * 8 + c2] * x[cidx(c0, c1, m)];
    y[t] = acc * h2 / (lam[c0] + lam[8 + c1] + lam[16 + c2]);
  }
  sync();
  // backward
#pragma unroll
  for (int h = 0; h < CELLS / NT; ++h) {
    const int t = t0 + h * NT, c0 = t & 7, c1 = (t >> 3) & 7, c2 = t >> 6;
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[0 * 64 + c0 * 8 + m] * y[cidx(m, c1, c2)];
    x[t] = acc;
  }
  sync();
#pragma unroll
  for (int h = 0; h < CELLS / NT; ++h) {
    const int t = t0 + h * NT, c0 = t & 7, c1 = (t >> 3) & 7, c2 = t >> 6;
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[1 * 64 + c1 * 8 + m] * x[cidx(c0, m, c2)];
    y[t] = acc;
  }
  sync();
#pragma unroll
  for (int h = 0; h < CELLS / NT; ++h) {
    const int t = t0 + h * NT, c0 = t & 7, c1 = (t >> 3) & 7, c2 = t >> 6;
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[2 * 64 + c2 * 8 + m] * y[cidx(c0, c1, m)];
    store(t, acc);
  }
  sync();  // sm is free again
}

// the level-0 solve on arrays of the value type T (FP64 or FP32 in memory)
template <int NT, typename T, typename Sync>
__device__ __forceinline__ void coarse_box(int t0, Sync sync, double *sm, T *phi, const T *rhs,
                                           const double *__restrict__ basis, const Bc &bc, double h2,
                                           double inv_h2, int homog) {
  coarse_box_io<NT>(
      t0, sync, sm, [&](int t) { return (double)rhs[t]; }, [&](int t, double v) { phi[t] = (T)v; }, basis, bc, h2,
      inv_h2, homog);
}

// FP64 residual f - L v of the cells of this thread in leaf box b; the
// largest magnitude is returned, r is stored to r32 when given
__device__ __forceinline__ double resid_box(const Grp &g, double *s, int b, const double *v, const double *rhs,
                                            const double *gh, const Nb &nb, const Bc &bc, double inv_h2,
                                            float *r32) {
  const size_t base = (size_t)b * CELLS;
  double f[CPT];
#pragma unroll
  for (int h = 0; h < CPT; ++h) f[h] = rhs[base + g.t + h * GT];
  stage_box(g, s, v, nb, gh, b, bc, 0);
  double m = 0.0;
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const int q = s10(g.t + h * GT);
    const double r = f[h] - (staged_sum(s, q) - 6.0 * s[q]) * inv_h2;
    if (r32) r32[base + g.t + h * GT] = cvt_f64_f32_rn(r);
    m = fmax(m, fabs(r));
  }
  return m;
}

// max over a box group, pushed to *slot by thread 0 (red: GT/32 doubles
// of shared memory of the group)
__device__ __forceinline__ void group_max_to(const Grp &g, unsigned long long *slot, double v, double *red) {
  v = warp_max(v);
  if ((g.t & 31) == 0) red[g.t >> 5] = v;
  g.sync();
  if (g.t == 0) {
    double x = red[0];
#pragma unroll
    for (int i = 1; i < GT / 32; ++i) x = fmax(x, red[i]);
    atomic_max_pos(slot, x);
  }
  g.sync();
}

// ---------------------------------------------------------------------------
// per-level kernels: one box per block of GT threads
// ---------------------------------------------------------------------------
//
// Each kernel reads its table entries (neighbours, parent, children: fixed
// during a solve) before waiting on its predecessor.  None of them triggers
// its dependent early: dependent blocks scheduled while a level kernel still
// runs slowed the V-cycle down by a third.

__device__ __forceinline__ Grp block_grp() { return Grp{(int)threadIdx.x, 0}; }

template <typename T>
__global__ void __launch_bounds__(GT) k_rbgs(int lo, int color, T *__restrict__ phi, const T *__restrict__ rhs,
                                             const T *__restrict__ gh, const int32_t *__restrict__ nbr6, Bc bc, T h2,
                                             int homog) {
  __shared__ T s[1000];
  const Grp g = block_grp();
  const int b = lo + blockIdx.x;
  const Nb nb = load_nb(g, nbr6, b);
  pdl_wait();
  rbgs_box(g, s, b, color, phi, rhs, gh, nb, bc, h2, homog);
}

// Three levels of the 8-child average chain in one launch.  A block takes a
// box b and writes its restriction into up to `depth` (1-3) ancestors: the
// 4^3 cells of its parent region, then the 2^3 cells of the grandparent that
// those 64 values cover, then the one cell of the great-grandparent that
// those 8 cover, each an 8-value sum in the order of restrict1_box times
// 1/8, so that every value equals the one the level-by-level chain writes.
// Blocks [0, nb) take the boxes lo.. of the group's finest level (depth
// d0), the next nl1 blocks the leaves leaf[lo1..] of the level below (depth
// d0 - 1) and the last nl2 the leaves leaf[lo2..] of the level below that
// (depth d0 - 2): every refined box of the three levels below the finest is
// then complete, from values complete before the launch.
template <typename T>
__global__ void __launch_bounds__(64) k_restrict3(int lo, int nb, int lo1, int nl1, int lo2, int d0,
                                                  const int32_t *__restrict__ leaf,
                                                  const int32_t *__restrict__ parent,
                                                  const int32_t *__restrict__ ijk, T *__restrict__ a,
                                                  T *__restrict__ a2) {
  __shared__ T sp[2][64], sg[2][8];
  const int blk = blockIdx.x, t = threadIdx.x;
  int b, depth;
  if (blk < nb) {
    b = lo + blk;
    depth = d0;
  } else if (blk < nb + nl1) {
    b = __ldg(leaf + lo1 + blk - nb);
    depth = d0 - 1;
  } else {
    b = __ldg(leaf + lo2 + blk - nb - nl1);
    depth = d0 - 2;
  }
  // ancestors and octants: P of b, G of P, Q of G
  const int P = __ldg(parent + b);
  const int ob[3] = {__ldg(ijk + 3 * b) & 1, __ldg(ijk + 3 * b + 1) & 1, __ldg(ijk + 3 * b + 2) & 1};
  int G = -1, Q = -1, op[3] = {0, 0, 0}, og[3] = {0, 0, 0};
  if (depth >= 2) {
    G = __ldg(parent + P);
    for (int d = 0; d < 3; ++d) op[d] = __ldg(ijk + 3 * P + d) & 1;
  }
  if (depth >= 3) {
    Q = __ldg(parent + G);
    for (int d = 0; d < 3; ++d) og[d] = __ldg(ijk + 3 * G + d) & 1;
  }
  pdl_wait();
  const int ci = t & 3, cj = (t >> 2) & 3, ck = t >> 4;
  const size_t fb = (size_t)b * CELLS;
  T s = 0, s2 = 0;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int c = cidx(2 * ci + di, 2 * cj + dj, 2 * ck + dk);
        s += a[fb + c];
        if (a2) s2 += a2[fb + c];
      }
  const T v = s * T(0.125), v2 = s2 * T(0.125);
  const size_t pc = (size_t)P * CELLS + cidx(4 * ob[0] + ci, 4 * ob[1] + cj, 4 * ob[2] + ck);
  a[pc] = v;
  if (a2) a2[pc] = v2;
  if (depth < 2) return;  // uniform per block
  sp[0][t] = v;
  sp[1][t] = v2;
  __syncthreads();
  if (t < 8) {
    const int ei = t & 1, ej = (t >> 1) & 1, ek = t >> 2;
    T g = 0, g2 = 0;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
          const int c = (2 * ei + di) + 4 * (2 * ej + dj) + 16 * (2 * ek + dk);
          g += sp[0][c];
          g2 += sp[1][c];
        }
    const T w = g * T(0.125), w2 = g2 * T(0.125);
    const size_t gc = (size_t)G * CELLS + cidx(4 * op[0] + 2 * ob[0] + ei, 4 * op[1] + 2 * ob[1] + ej,
                                               4 * op[2] + 2 * ob[2] + ek);
    a[gc] = w;
    if (a2) a2[gc] = w2;
    sg[0][t] = w;
    sg[1][t] = w2;
  }
  if (depth < 3) return;
  __syncthreads();
  if (t == 0) {
    T q = 0, q2 = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {  // e = di + 2 dj + 4 dk: the restrict1_box order
      q += sg[0][e];
      q2 += sg[1][e];
    }
    const size_t qc = (size_t)Q * CELLS + cidx(4 * og[0] + 2 * op[0] + ob[0], 4 * og[1] + 2 * op[1] + ob[1],
                                               4 * og[2] + 2 * op[2] + ob[2]);
    a[qc] = q * T(0.125);
    if (a2) a2[qc] = q2 * T(0.125);
  }
}

template <typename T>
__global__ void __launch_bounds__(GT) k_fas(int lo, T *__restrict__ phi, T *__restrict__ old, T *__restrict__ rhs,
                                            const T *__restrict__ gh, const int32_t *__restrict__ nbr6,
                                            const int32_t *__restrict__ child, Bc bc, T inv_h2, int homog) {
  __shared__ T s[1000];
  const Grp g = block_grp();
  const int b = lo + blockIdx.x;
  const Nb nb = load_nb(g, nbr6, b);
  const bool refined = __ldg(child + 8 * b) >= 0;
  pdl_wait();
  fas_box(g, s, b, phi, old, rhs, gh, nb, refined, bc, inv_h2, homog);
}

template <typename T>
// Blocks [0, n) take the boxes lo.. of level l.  With old != nullptr the
// restricted values also go to old, and blocks [n, n + nl) copy the leaf
// boxes leaf[0, nl) of the level below into old (for k_fas_rbgs0).
__global__ void __launch_bounds__(GT) k_resid_restrict(int lo, int n, T *__restrict__ phi, T *__restrict__ rhs,
                                                       const T *__restrict__ gh, const int32_t *__restrict__ nbr6,
                                                       const int32_t *__restrict__ parent,
                                                       const int32_t *__restrict__ ijk, Bc bc, T inv_h2,
                                                       int homog, T *__restrict__ old, const int32_t *__restrict__ leaf) {
  __shared__ T s[1000], sr[CELLS];
  const Grp g = block_grp();
  if ((int)blockIdx.x >= n) {
    const int b = __ldg(leaf + blockIdx.x - n);
    pdl_wait();
    const size_t base = (size_t)b * CELLS;
#pragma unroll
    for (int h = 0; h < CPT; ++h) old[base + g.t + h * GT] = phi[base + g.t + h * GT];
    return;
  }
  const int b = lo + blockIdx.x;
  const Nb nb = load_nb(g, nbr6, b);
  const Place pl = load_place(parent, ijk, b);
  pdl_wait();
  resid_restrict_box(g, s, sr, b, phi, rhs, gh, nb, pl, bc, inv_h2, homog, old);
}

// k_fas fused with the first colour pass (colour 0) of the smoothing that
// follows it on the same level.  The FAS term of a box reads its
// neighbours' face cells, whose colour-0 values the neighbours' own blocks
// of this launch overwrite; so every value is staged from old, which the
// restriction launch before (k_resid_restrict with old) filled with the
// whole level as it is now and which nothing in this launch writes.  The
// box's new rhs is read back after the block barrier.  The same operations
// as k_fas followed by k_rbgs with colour 0.
template <typename T>
__global__ void __launch_bounds__(GT) k_fas_rbgs0(int lo, T *__restrict__ phi, const T *__restrict__ old,
                                                  T *__restrict__ rhs, const T *__restrict__ gh,
                                                  const int32_t *__restrict__ nbr6, const int32_t *__restrict__ child,
                                                  Bc bc, T inv_h2, T h2, int homog) {
  __shared__ T s[1000];
  const Grp g = block_grp();
  const int b = lo + blockIdx.x;
  const Nb nb = load_nb(g, nbr6, b);
  const bool refined = __ldg(child + 8 * b) >= 0;
  pdl_wait();
  const size_t base = (size_t)b * CELLS;
  stage_box(g, s, old, nb, gh, b, bc, homog);
  if (refined) {
#pragma unroll
    for (int h = 0; h < CPT; ++h) {
      const int c = g.t + h * GT, q = s10(c);
      rhs[base + c] += (staged_sum(s, q) - T(6) * s[q]) * inv_h2;
    }
  }
  g.sync();
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    const int c = colour_cell(g.t + h * GT, 0);
    phi[base + c] = rbgs_value(s, c, rhs[base + c], h2);
  }
}

// leaf boxes of one level whose FP64 residual norm a prolongation launch
// computes in extra blocks (n = 0: none)
struct LeafNorm {
  const int32_t *leaf;  // leaf list segment of the level
  int n;
  const double *v, *rhs, *gh;
  double inv_h2;
  unsigned long long *slot;
};

// Blocks [0, n) prolong into the boxes [lo, lo + n) of level l; blocks
// beyond add the residual max of the leaf boxes of level l-1, which no
// later operation of the V-cycle changes, to ln.slot.
template <typename T>
__global__ void __launch_bounds__(GT) k_prolong_cf(int lo, int n, int mode, T *__restrict__ phi,
                                                   const T *__restrict__ old, T *__restrict__ gh,
                                                   const int32_t *__restrict__ nbr6,
                                                   const int32_t *__restrict__ parent,
                                                   const int32_t *__restrict__ ijk, Bc bc, int homog,
                                                   unsigned long long *err, LeafNorm ln) {
  __shared__ T sp[216];
  __shared__ double rs[1000 + GT / 32];
  const Grp g = block_grp();
  if ((int)blockIdx.x >= n) {
    const int b = __ldg(ln.leaf + blockIdx.x - n);
    const Nb nb = load_nb(g, nbr6, b);
    pdl_wait();
    const double m = resid_box(g, rs, b, ln.v, ln.rhs, ln.gh, nb, bc, ln.inv_h2, nullptr);
    group_max_to(g, ln.slot, m, rs + 1000);
    return;
  }
  pdl_wait();
  prolong_box(g, sp, lo + blockIdx.x, mode, phi, old, gh, nbr6, parent, ijk, bc, homog, err);
}

// coarse interpolation values of the refinement faces of the boxes
// [lo, lo+grid), 64 threads per box
template <typename T>
__global__ void __launch_bounds__(64) k_fill_cf(int lo, const T *__restrict__ v, T *__restrict__ gh,
                                                const int32_t *__restrict__ nbr6,
                                                const int32_t *__restrict__ parent,
                                                const int32_t *__restrict__ ijk, Bc bc, int homog,
                                                unsigned long long *err) {
  pdl_wait();
  cf_faces_box((int)threadIdx.x, 64, v, gh, nbr6, parent, ijk, bc, homog, lo + blockIdx.x, err);
}

template <typename T>
__global__ void __launch_bounds__(CELLS) k_coarse_solve(T *__restrict__ phi, const T *__restrict__ rhs,
                                                        const double *__restrict__ basis, Bc bc, double h2,
                                                        double inv_h2, int homog) {
  __shared__ double sm[2 * CELLS + 216];
  pdl_wait();
  coarse_box<CELLS>((int)threadIdx.x, [] { __syncthreads(); }, sm, phi, rhs, basis, bc, h2, inv_h2, homog);
}

// Orthonormal eigenvectors and (h^2-scaled) eigenvalues of the 1-D
// cell-centred 3-point operator on n cells with Neumann (ghost = inner) or
// Dirichlet (ghost = -inner) ends: cosine (NN), sine (DD) and quarter-wave
// sine (DN, ND) families.  basis[a*64 + i*8 + m] = component i of vector m.
__global__ void k_coarse_basis(double *basis, Bc bc, int n) {
  pdl_wait();
  int t = threadIdx.x;
  if (t >= 3 * n) return;
  int a = t / n, m = t % n;
  int lo = bc.type[2 * a], hi = bc.type[2 * a + 1];
  double v[NC], nrm = 0.0, mu;
  for (int i = 0; i < n; ++i) {
    double x = (i + 0.5) / n;
    if (!lo && !hi) v[i] = cospi(m * x);
    else if (lo && hi) v[i] = sinpi((m + 1) * x);
    else if (lo) v[i] = sinpi((m + 0.5) * x);
    else v[i] = sinpi((m + 0.5) * (n - i - 0.5) / n);
    nrm += v[i] * v[i];
  }
  double th = (!lo && !hi) ? m : ((lo && hi) ? m + 1 : m + 0.5);
  double sn = sinpi(th / (2.0 * n));
  mu = -4.0 * sn * sn;
  nrm = rsqrt(nrm);
  for (int i = 0; i < n; ++i) basis[a * 64 + i * 8 + m] = v[i] * nrm;
  basis[192 + a * 8 + m] = mu;
}

// max over leaf cells of |f - L v| into *slot (one leaf box per block); with
// f32 given, also the residual rounded to FP32 (right-hand side of the
// error equation of the mixed-precision solve)
__global__ void __launch_bounds__(GT) k_resnorm(const int32_t *__restrict__ leaf, const int32_t *__restrict__ level,
                                                const double *__restrict__ v, const double *__restrict__ rhs,
                                                const double *__restrict__ gh, const int32_t *__restrict__ nbr6,
                                                Bc bc, LevelH lh, float *__restrict__ f32,
                                                unsigned long long *slot) {
  __shared__ double s[1000], red[GT / 32];
  pdl_wait();
  const Grp g = block_grp();
  const int b = __ldg(leaf + blockIdx.x);
  const double m = resid_box(g, s, b, v, rhs, gh, load_nb(g, nbr6, b), bc, lh.inv_h2[__ldg(level + b)], f32);
  group_max_to(g, slot, m, red);
}

// FP64 accumulation of the FP32 correction on leaf cells
__global__ void __launch_bounds__(GT) k_add_corr(const int32_t *__restrict__ leaf, double *__restrict__ phi,
                                                 const float *__restrict__ e32) {
  pdl_wait();
  const size_t x = (size_t)__ldg(leaf + blockIdx.x) * CELLS + threadIdx.x;
#pragma unroll
  for (int h = 0; h < CPT; ++h) phi[x + h * GT] += cvt_f32_f64(e32[x + h * GT]);
}

// Stopping test of the device-side cycle loop: relative residual of the
// last norm, cycle count (+inc), and the loop condition
// rel > tol && cycles < max; the relative residual of cycle c also goes to
// hist[c - 1] (the first SM_HIST cycles).
__global__ void k_loop_check(cudaGraphConditionalHandle h, unsigned long long *sc, int inc, double *hist) {
  pdl_wait();
  double num = __longlong_as_double((long long)sc[SC_NORM]);
  double den = __longlong_as_double((long long)sc[SC_DEN]);
  double rel = den > 0.0 ? num / den : num;
  unsigned long long c = sc[SC_CYC] + (unsigned long long)inc;
  sc[SC_CYC] = c;
  sc[SC_REL] = (unsigned long long)__double_as_longlong(rel);
  if (c >= 1 && c <= (unsigned long long)SM_HIST) hist[c - 1] = rel;
  double tol = __longlong_as_double((long long)sc[SC_TOL]);
  const bool ovf = (sc[SC_ERR] & 8ull) != 0;  // fixed-point range left: the host runs the solve again
  cudaGraphSetConditional(h, (rel > tol && c < sc[SC_MAXC] && !ovf) ? 1u : 0u);
}

#include "mgfix.cuh"

// ---------------------------------------------------------------------------
// persistent V-cycle kernel
// ---------------------------------------------------------------------------
//
// One cooperative launch (every block resident) runs the phases of one or
// more V-cycles: each phase is one level operation over all boxes of a
// level, spread over the box groups of all blocks, and ends with a grid
// barrier.  The barrier waits are bounded: after PERSIST_SPIN polls a block
// sets error bit 4 and returns, and so do the others at their next wait.

constexpr unsigned long long ERR_BARRIER = 4ull;
constexpr long long PERSIST_SPIN = 1ll << 21;  // about a second of polling

template <typename T>
struct PArgs {
  T *phi, *rhs, *old, *gh;
  const int32_t *nbr6, *parent, *ijk, *child, *leaf, *level;
  const double *basis;
  double *phi64, *rhs64, *gh64;  // FP64 potential, rhs, interpolation values (residual test)
  unsigned long long *sc;
  Bc bc;
  LevelH lh;
  int level_off[MAXL + 1];
  int n_levels, n_leaves, top, nu1, nu2, homog;
  int fmg;   // run the FMG ladder first (restricted rhs, level-0 solve, one V-cycle per finer level)
  int loop;  // after that (or from the start): V-cycles with the residual test until converged
  int bar_extra;  // arrivals a barrier waits for beyond the grid (0; 1 only in the timeout self-test)
};

// shared memory of one box group of the persistent kernel (bytes)
template <typename T>
__host__ __device__ constexpr size_t persist_group_smem() {
  return 1512 * sizeof(T) > (2 * CELLS + 216) * sizeof(double) ? 1512 * sizeof(T)
                                                                 : (2 * CELLS + 216) * sizeof(double);
}
static_assert(1000 + GT / 32 <= 2 * CELLS + 216, "residual staging fits the FP64 scratch");

struct GridBar {
  unsigned int *cnt;
  unsigned int epoch;
  unsigned int extra;  // see PArgs::bar_extra
  int *flag;  // shared: barrier outcome for the block
  unsigned long long *err;
  // all blocks arrive; false when the wait ran out (the caller returns)
  __device__ __forceinline__ bool sync() {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int target = ++epoch * (gridDim.x + extra);
      __threadfence();
      atomicAdd(cnt, 1u);
      int ok = 1;
      long long it = 0;
      unsigned int v;
      while (true) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
        if (v >= target) break;
        if (++it > PERSIST_SPIN) {
          atomicOr(err, ERR_BARRIER);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
      *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
  }
};

template <typename T>
struct Persist {
  const PArgs<T> &a;
  Grp g;
  int gi, ng;  // group index over the grid, number of groups
  T *s, *sr;
  double *sd;  // FP64 scratch of the group (coarse solve, residual staging)
  GridBar bar;

  __device__ int lo(int l) const { return a.level_off[l]; }
  __device__ int hi(int l) const { return a.level_off[l + 1]; }
  __device__ bool empty(int l) const { return hi(l) == lo(l); }

  __device__ bool smooth(int l, int nu) {
    if (empty(l)) return true;
    const T h2 = (T)a.lh.h2[l];
    for (int it = 0; it < nu; ++it)
      for (int color = 0; color < 2; ++color) {
        for (int b = lo(l) + gi; b < hi(l); b += ng)
          rbgs_box(g, s, b, color, a.phi, a.rhs, a.gh, load_nb(g, a.nbr6, b), a.bc, h2, a.homog);
        if (!bar.sync()) return false;
      }
    return true;
  }

  __device__ bool coarse() {
    if (gi == 0)
      coarse_box<GT>(g.t, [&] { g.sync(); }, sd, a.phi, a.rhs, a.basis, a.bc, a.lh.h2[0], a.lh.inv_h2[0], a.homog);
    return bar.sync();
  }

  __device__ bool prolong(int l, int mode) {
    if (empty(l)) return true;
    for (int b = lo(l) + gi; b < hi(l); b += ng)
      prolong_box(g, s, b, mode, a.phi, a.old, a.gh, a.nbr6, a.parent, a.ijk, a.bc, a.homog, a.sc + SC_ERR);
    return bar.sync();
  }

  __device__ bool vcycle(int top) {
    for (int l = top; l >= 1; --l) {
      if (!smooth(l, a.nu1)) return false;
      if (!empty(l)) {
        const T ih2 = (T)a.lh.inv_h2[l];
        for (int b = lo(l) + gi; b < hi(l); b += ng)
          resid_restrict_box(g, s, sr, b, a.phi, a.rhs, a.gh, load_nb(g, a.nbr6, b), load_place(a.parent, a.ijk, b),
                             a.bc, ih2, a.homog);
        if (!bar.sync()) return false;
      }
      const T ih2c = (T)a.lh.inv_h2[l - 1];
      for (int b = lo(l - 1) + gi; b < hi(l - 1); b += ng)
        fas_box(g, s, b, a.phi, a.old, a.rhs, a.gh, load_nb(g, a.nbr6, b), __ldg(a.child + 8 * b) >= 0, a.bc, ih2c,
                a.homog);
      if (!bar.sync()) return false;
    }
    if (!coarse()) return false;
    for (int l = 1; l <= top; ++l) {
      if (!prolong(l, 0)) return false;
      if (!smooth(l, a.nu2)) return false;
    }
    return true;
  }

  __device__ bool ladder() {
    for (int l = a.n_levels - 1; l >= 1; --l) {
      for (int b = lo(l) + gi; b < hi(l); b += ng)
        restrict1_box<T>(g, b, load_place(a.parent, a.ijk, b), a.rhs, nullptr);
      if (!bar.sync()) return false;
    }
    if (!coarse()) return false;
    for (int l = 1; l < a.n_levels; ++l) {
      if (!prolong(l, 1)) return false;
      if (!vcycle(l)) return false;
    }
    return true;
  }

  // max_leaf |f - L phi| (FP64) into slot; true when the wait succeeded
  __device__ bool resnorm(unsigned long long *slot) {
    double m = 0.0;
    for (int i = gi; i < a.n_leaves; i += ng) {
      const int b = __ldg(a.leaf + i);
      m = fmax(m, resid_box(g, sd, b, a.phi64, a.rhs64, a.gh64, load_nb(g, a.nbr6, b), a.bc,
                            a.lh.inv_h2[__ldg(a.level + b)], nullptr));
    }
    group_max_to(g, slot, m, sd + 1000);
    return bar.sync();
  }
};

template <typename T>
__global__ void __launch_bounds__(PGROUPS *GT, 1) k_persist(const __grid_constant__ PArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int flag;
  const int q = threadIdx.x / GT;
  // one region per group, used by one phase at a time: T staging s[1000]
  // and sr[512], or FP64 scratch (level-0 solve 2 x 512 + 216 doubles,
  // residual staging 1000 + GT/32 doubles)
  unsigned char *base = smem + (size_t)q * persist_group_smem<T>();
  Persist<T> p{a, Grp{(int)threadIdx.x % GT, 1 + q}, q * (int)gridDim.x + (int)blockIdx.x,
               PGROUPS * (int)gridDim.x, nullptr, nullptr, nullptr,
               GridBar{(unsigned int *)(a.sc + SC_BAR), 0u, (unsigned int)a.bar_extra, &flag, a.sc + SC_ERR}};
  p.sd = (double *)base;
  p.s = (T *)base;
  p.sr = p.s + 1000;
  int cyc = 0;
  double rel = 0.0, num = 0.0;
  const double den = __longlong_as_double((long long)a.sc[SC_DEN]);
  const double tol = __longlong_as_double((long long)a.sc[SC_TOL]);
  const unsigned long long maxc = a.sc[SC_MAXC];
  int pass = 0;  // residual passes: slot SC_PN0 + (pass & 1)
  auto test = [&]() -> int {  // 1 = go on, 0 = converged or limit, -1 = barrier wait ran out
    unsigned long long *slot = a.sc + SC_PN0 + (pass & 1);
    if (!p.resnorm(slot)) return -1;
    unsigned long long bits;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(bits) : "l"(slot) : "memory");
    num = __longlong_as_double((long long)bits);
    rel = den > 0.0 ? num / den : num;
    ++cyc;
    ++pass;
    return (rel > tol && (unsigned long long)cyc < maxc) ? 1 : 0;
  };
  // each residual slot is cleared one full cycle before its next use
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.sc[SC_PN0] = 0ull;
    a.sc[SC_PN1] = 0ull;
  }
  if (!p.bar.sync()) return;
  int go = 1;
  if (a.fmg) {
    if (!p.ladder()) return;
    if (a.loop) {
      go = test();
      if (go < 0) return;
    } else {
      go = 0;
    }
  }
  while (go) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && pass > 0) a.sc[SC_PN0 + (pass & 1)] = 0ull;
    if (!p.vcycle(a.top)) return;
    if (!a.loop) break;
    go = test();
    if (go < 0) return;
  }
  if (a.loop && blockIdx.x == 0 && threadIdx.x == 0) {
    a.sc[SC_NORM] = (unsigned long long)__double_as_longlong(num);
    a.sc[SC_REL] = (unsigned long long)__double_as_longlong(rel);
    a.sc[SC_CYC] = (unsigned long long)cyc;
  }
}

template <typename T>
constexpr size_t persist_smem() {
  return (size_t)PGROUPS * persist_group_smem<T>();
}

// The persistent kernel of the FP64 solve: the fixed-point phases of
// mgfix.cuh between grid barriers (bit-identical to the per-level launches).
struct PArgsX {
  long long *phx, *gx, *oldx, *ghx;
  const double *rhs;
  const int32_t *nbr6, *parent, *ijk, *child, *leaf, *level;
  const double *basis;
  unsigned long long *sc;
  Bc bc;
  LevelH lh;
  int level_off[MAXL + 1];
  int n_levels, n_leaves, top, nu1, nu2;
  int fmg, loop, bar_extra;  // as PArgs (the rhs restriction of FMG is done before the launch)
};

// shared memory of one box group: 10^3 staging plus 512 sums, or the
// FP64 scratch of the level-0 solve, then GT/32 reduction words (bytes)
constexpr size_t PX_STAGE = (1000 + CELLS) * sizeof(long long);
static_assert((2 * CELLS + 216) * sizeof(double) <= PX_STAGE, "level-0 scratch fits");
__host__ __device__ constexpr size_t persistx_group_smem() {
  return PX_STAGE + (GT / 32) * sizeof(unsigned long long);
}

struct PersistX {
  const PArgsX &a;
  Grp g;
  int gi, ng;
  long long *s;
  unsigned long long *red;
  GridBar bar;

  __device__ int lo(int l) const { return a.level_off[l]; }
  __device__ int hi(int l) const { return a.level_off[l + 1]; }
  __device__ bool empty(int l) const { return hi(l) == lo(l); }

  __device__ bool smooth(int l, int nu) {
    if (empty(l)) return true;
    for (int it = 0; it < nu; ++it)
      for (int color = 0; color < 2; ++color) {
        for (int b = lo(l) + gi; b < hi(l); b += ng) {
          const bool bad = fx::fx_color_box(g, s, b, color, a.phx, a.gx, a.ghx, load_nb(g, a.nbr6, b), a.bc, a.sc);
          fx::fx_flag(bad, a.sc);
        }
        if (!bar.sync()) return false;
      }
    return true;
  }

  __device__ bool coarse() {
    if (gi == 0) {
      const int E = fx::fx_E(a.sc);
      const double cf = -6.0 * fx::fx_q(E) * a.lh.inv_h2[0];
      bool bad = false;
      coarse_box_io<GT>(
          g.t, [&] { g.sync(); }, (double *)s, [&](int t) { return __ll2double_rn(a.gx[fx::xsplit(t)]) * cf; },
          [&](int t, double v) { a.phx[fx::xsplit(t)] = fx::fx_of(v, E, bad); }, a.basis, a.bc, a.lh.h2[0],
          a.lh.inv_h2[0], 0);
      fx::fx_flag(bad, a.sc);
    }
    return bar.sync();
  }

  __device__ bool prolong(int l, int mode) {
    if (empty(l)) return true;
    for (int b = lo(l) + gi; b < hi(l); b += ng) {
      const bool bad = fx::fx_prolong_box(g, s, b, mode, a.phx, a.oldx, a.ghx, a.nbr6, a.parent, a.ijk, a.bc, a.sc,
                                          a.sc + SC_ERR);
      fx::fx_flag(bad, a.sc);
    }
    return bar.sync();
  }

  __device__ bool vcycle(int top) {
    for (int l = top; l >= 1; --l) {
      if (!smooth(l, a.nu1)) return false;
      if (!empty(l)) {
        for (int b = lo(l) + gi; b < hi(l); b += ng)
          fx::fx_resid_restrict_box(g, s, s + 1000, b, a.phx, a.gx, a.ghx, load_nb(g, a.nbr6, b),
                                    load_place(a.parent, a.ijk, b), a.bc, a.sc);
        if (!bar.sync()) return false;
      }
      for (int b = lo(l - 1) + gi; b < hi(l - 1); b += ng) {
        const bool bad = fx::fx_fas_box(g, s, b, a.phx, a.oldx, a.gx, a.ghx, load_nb(g, a.nbr6, b),
                                        __ldg(a.child + 8 * b) >= 0, a.bc, a.sc);
        fx::fx_flag(bad, a.sc);
      }
      if (!bar.sync()) return false;
    }
    if (!coarse()) return false;
    for (int l = 1; l <= top; ++l) {
      if (!prolong(l, 0)) return false;
      if (!smooth(l, a.nu2)) return false;
    }
    return true;
  }

  __device__ bool ladder() {
    if (!coarse()) return false;
    for (int l = 1; l < a.n_levels; ++l) {
      if (!prolong(l, 1)) return false;
      if (!vcycle(l)) return false;
    }
    return true;
  }

  // max_leaf |f - L phi| into slot; true when the wait succeeded
  __device__ bool resnorm(unsigned long long *slot) {
    unsigned long long m = 0;
    const double q = fx::fx_q(fx::fx_E(a.sc));
    for (int i = gi; i < a.n_leaves; i += ng) {
      const int b = __ldg(a.leaf + i);
      const unsigned long long r = fx::fx_resid_max_box(g, s, b, a.phx, a.rhs, a.ghx, load_nb(g, a.nbr6, b), a.bc,
                                                        a.sc, -q * a.lh.inv_h2[__ldg(a.level + b)]);
      m = r > m ? r : m;
    }
    fx::group_umax_to(g, slot, m, red);
    return bar.sync();
  }
};

__global__ void __launch_bounds__(PGROUPS *GT, 1) k_persistx(const __grid_constant__ PArgsX a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int flag;
  const int q = threadIdx.x / GT;
  unsigned char *base = smem + (size_t)q * persistx_group_smem();
  PersistX p{a, Grp{(int)threadIdx.x % GT, 1 + q}, q * (int)gridDim.x + (int)blockIdx.x, PGROUPS * (int)gridDim.x,
             (long long *)base, (unsigned long long *)(base + PX_STAGE),
             GridBar{(unsigned int *)(a.sc + SC_BAR), 0u, (unsigned int)a.bar_extra, &flag, a.sc + SC_ERR}};
  int cyc = 0;
  double rel = 0.0, num = 0.0;
  const double den = __longlong_as_double((long long)a.sc[SC_DEN]);
  const double tol = __longlong_as_double((long long)a.sc[SC_TOL]);
  const unsigned long long maxc = a.sc[SC_MAXC];
  int pass = 0;
  auto test = [&]() -> int {  // 1 = go on, 0 = converged, limit or range left, -1 = barrier wait ran out
    unsigned long long *slot = a.sc + SC_PN0 + (pass & 1);
    if (!p.resnorm(slot)) return -1;
    unsigned long long bits, err;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(bits) : "l"(slot) : "memory");
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(err) : "l"(a.sc + SC_ERR) : "memory");
    num = __longlong_as_double((long long)bits);
    rel = den > 0.0 ? num / den : num;
    ++cyc;
    ++pass;
    return (rel > tol && (unsigned long long)cyc < maxc && !(err & fx::FX_ERR_OVF)) ? 1 : 0;
  };
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.sc[SC_PN0] = 0ull;
    a.sc[SC_PN1] = 0ull;
  }
  if (!p.bar.sync()) return;
  int go = 1;
  if (a.fmg) {
    if (!p.ladder()) return;
    if (a.loop) {
      go = test();
      if (go < 0) return;
    } else {
      go = 0;
    }
  }
  while (go) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && pass > 0) a.sc[SC_PN0 + (pass & 1)] = 0ull;
    if (!p.vcycle(a.top)) return;
    if (!a.loop) break;
    go = test();
    if (go < 0) return;
  }
  if (a.loop && blockIdx.x == 0 && threadIdx.x == 0) {
    a.sc[SC_NORM] = (unsigned long long)__double_as_longlong(num);
    a.sc[SC_REL] = (unsigned long long)__double_as_longlong(rel);
    a.sc[SC_CYC] = (unsigned long long)cyc;
  }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
static int lvl_n(const sm_ctx *ctx, int l) { return ctx->level_off[l + 1] - ctx->level_off[l]; }

// the arrays one multigrid cycle works on
template <typename T>
struct MG {
  T *phi, *rhs, *old, *gh;
  int homog;  // error equation: homogeneous physical ghosts
};

static MG<float> mg32(sm_ctx *ctx) { return {ctx->e32, ctx->f32, ctx->old32, ctx->gh32, 1}; }

int sm_mg_fill_cf(sm_ctx *ctx, double *var, int l, int homog) {
  if (l <= ctx->lbase || l >= ctx->n_levels) return SM_OK;  // uniform levels: no refinement faces
  int n = lvl_n(ctx, l);
  if (n == 0) return SM_OK;
  sm_launch(ctx, k_fill_cf<double>, n, 64, 0, ctx->level_off[l], var, ctx->gh, ctx->nbr6, ctx->parent,
            ctx->ijk, ctx->bc, homog, ctx->dscal + SC_ERR);
  SM_CKL("fill_cf");
  return SM_OK;
}

// every level at once: each level's values come from the level below only
int sm_fill_all_cf(sm_ctx *ctx, double *var) {
  if (ctx->lbase + 1 >= ctx->n_levels) return SM_OK;
  const int lo = ctx->level_off[ctx->lbase + 1], n = ctx->n_boxes - lo;
  if (n <= 0) return SM_OK;
  sm_launch(ctx, k_fill_cf<double>, n, 64, 0, lo, var, ctx->gh, ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc, 0,
            ctx->dscal + SC_ERR);
  SM_CKL("fill_cf");
  return SM_OK;
}

template <typename T>
static int restrict_chain(sm_ctx *ctx, T *a, T *a2) {
  // groups of three levels, finest first (k_restrict3)
  for (int l = ctx->n_levels - 1; l >= 1; l -= 3) {
    const int d0 = l < 3 ? l : 3;
    const int nb = lvl_n(ctx, l);
    const int lo1 = d0 >= 2 ? ctx->leaf_level_off[l - 1] : 0, nl1 = d0 >= 2 ? ctx->leaf_level_off[l] - lo1 : 0;
    const int lo2 = d0 >= 3 ? ctx->leaf_level_off[l - 2] : 0, nl2 = d0 >= 3 ? ctx->leaf_level_off[l - 1] - lo2 : 0;
    if (nb + nl1 + nl2 == 0) continue;
    sm_launch(ctx, k_restrict3<T>, nb + nl1 + nl2, 64, 0, ctx->level_off[l], nb, lo1, nl1, lo2, d0, ctx->leaf,
              ctx->parent, ctx->ijk, a, a2);
  }
  SM_CKL("restrict");
  return SM_OK;
}

// a = avg8 of children (and a2 likewise), finest level first
int sm_restrict_pair(sm_ctx *ctx, double *a, double *a2) { return restrict_chain(ctx, a, a2); }

template <typename T>
static int rbgs_pass(sm_ctx *ctx, const MG<T> &m, int l, int color) {
  sm_launch(ctx, k_rbgs<T>, lvl_n(ctx, l), GT, 0, ctx->level_off[l], color, m.phi, m.rhs, m.gh, ctx->nbr6,
            ctx->bc, (T)ctx->lh.h2[l], m.homog);
  return SM_OK;
}

// nu red-black sweeps of level l; with skip_first the first colour pass has
// already run (k_fas_rbgs0)
template <typename T>
static int smooth(sm_ctx *ctx, const MG<T> &m, int l, int nu, bool skip_first = false) {
  if (!lvl_n(ctx, l)) return SM_OK;
  for (int s = 0; s < nu; ++s)
    for (int color = 0; color < 2; ++color)
      if (!(skip_first && s == 0 && color == 0)) rbgs_pass(ctx, m, l, color);
  SM_CKL("rbgs");
  return SM_OK;
}

static int ensure_basis(sm_ctx *ctx) {
  if (!ctx->basis_ready) {
    sm_launch(ctx, k_coarse_basis, 1, 32, 0, ctx->basis, ctx->bc, NC);
    SM_CKL("coarse basis");
    ctx->basis_ready = true;
  }
  return SM_OK;
}

template <typename T>
static int coarse_solve(sm_ctx *ctx, const MG<T> &m) {
  int st = ensure_basis(ctx);
  if (st) return st;
  sm_launch(ctx, k_coarse_solve<T>, 1, CELLS, 0, m.phi, m.rhs, ctx->basis, ctx->bc, ctx->lh.h2[0],
            ctx->lh.inv_h2[0], m.homog);
  SM_CKL("coarse solve");
  return SM_OK;
}

// leaf segment of level l for a residual-norm role (none when slot < 0)
static LeafNorm leaf_norm_of(sm_ctx *ctx, int l, int slot) {
  LeafNorm ln = {};
  if (slot < 0 || l < 0) return ln;
  ln.leaf = ctx->leaf + ctx->leaf_level_off[l];
  ln.n = ctx->leaf_level_off[l + 1] - ctx->leaf_level_off[l];
  ln.v = ctx->phi;
  ln.rhs = ctx->rhs;
  ln.gh = ctx->gh;
  ln.inv_h2 = ctx->lh.inv_h2[l];
  ln.slot = ctx->dscal + slot;
  return ln;
}

template <typename T>
static int prolong_cf(sm_ctx *ctx, const MG<T> &m, int l, int mode, LeafNorm ln = LeafNorm{}) {
  sm_launch(ctx, k_prolong_cf<T>, lvl_n(ctx, l) + ln.n, GT, 0, ctx->level_off[l], lvl_n(ctx, l), mode, m.phi, m.old,
            m.gh, ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc, m.homog, ctx->dscal + SC_ERR, ln);
  SM_CKL("prolong");
  return SM_OK;
}

// FAS V-cycle with `top` as finest level.  On entry the coarse
// interpolation values gh of every level <= top must match the current
// values of the level below (the solve prologue and every up-sweep leave
// them so); the down-sweep changes no level below the one it smooths
// before that level is visited again, so it needs no refill.
// With norm_slot >= 0 (FP64 arrays, top the finest level) the cycle also
// leaves max_leaf |f - L phi| in that slot: the leaves of level l-1 are
// measured by extra blocks of the prolongation into level l, those of the
// top level after its post-smoothing.
template <typename T>
static int vcycle(sm_ctx *ctx, const MG<T> &m, int top, int norm_slot = -1) {
  int st;
  if (norm_slot >= 0)
    SM_CK(cudaMemsetAsync(ctx->dscal + norm_slot, 0, sizeof(unsigned long long), ctx->stream));
  bool fused = false;  // the first colour pass of level l has run (k_fas_rbgs0)
  for (int l = top; l >= 1; --l) {
    if ((st = smooth(ctx, m, l, ctx->cfg.nu1, fused))) return st;
    // on a level of one partial wave below another (above level 0) the FAS
    // step also runs the level's first colour pass; the restriction then
    // copies the whole level below into old first
    fused = l - 1 >= 1 && ctx->cfg.nu1 > 0 && lvl_n(ctx, l) < ctx->rows_min && lvl_n(ctx, l - 1) < ctx->rows_min;
    const int nl = fused ? ctx->leaf_level_off[l] - ctx->leaf_level_off[l - 1] : 0;
    sm_launch(ctx, k_resid_restrict<T>, lvl_n(ctx, l) + nl, GT, 0, ctx->level_off[l], lvl_n(ctx, l), m.phi, m.rhs,
              m.gh, ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc, (T)ctx->lh.inv_h2[l], m.homog,
              fused ? m.old : nullptr, ctx->leaf + ctx->leaf_level_off[l - 1]);
    if (fused)
      sm_launch(ctx, k_fas_rbgs0<T>, lvl_n(ctx, l - 1), GT, 0, ctx->level_off[l - 1], m.phi, (const T *)m.old, m.rhs,
                m.gh, ctx->nbr6, ctx->child, ctx->bc, (T)ctx->lh.inv_h2[l - 1], (T)ctx->lh.h2[l - 1], m.homog);
    else
      sm_launch(ctx, k_fas<T>, lvl_n(ctx, l - 1), GT, 0, ctx->level_off[l - 1], m.phi, m.old, m.rhs, m.gh,
                ctx->nbr6, ctx->child, ctx->bc,
                (T)ctx->lh.inv_h2[l - 1], m.homog);
    SM_CKL("vcycle down");
  }
  if ((st = coarse_solve(ctx, m))) return st;
  for (int l = 1; l <= top; ++l) {
    if ((st = prolong_cf(ctx, m, l, 0, leaf_norm_of(ctx, norm_slot >= 0 ? l - 1 : -1, norm_slot)))) return st;
    if ((st = smooth(ctx, m, l, ctx->cfg.nu2))) return st;
  }
  if (norm_slot >= 0) {
    const LeafNorm ln = leaf_norm_of(ctx, top, norm_slot);
    if (ln.n > 0)
      sm_launch(ctx, k_resnorm, ln.n, GT, 0, ln.leaf, ctx->level, ctx->phi, ctx->rhs, ctx->gh, ctx->nbr6, ctx->bc,
                ctx->lh, (float *)nullptr, ln.slot);
    SM_CKL("resnorm");
  }
  return SM_OK;
}

// Blocks of the persistent kernel that fit on the device at once (its
// launches are cooperative, so all of them are resident together).
// Blocks of a persistent kernel that fit on the device at once (its
// launches are cooperative, so all of them are resident together); idx 0:
// the fixed-point FP64 kernel, 1: the FP32 kernel of the mixed form.
template <typename K>
static int persist_prepare_k(sm_ctx *ctx, K kernel, size_t smem, int idx) {
  if (ctx->persist_grid[idx]) return SM_OK;
  SM_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, sms = 0, coop = 0;
  SM_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  if (!coop) return sm_fail(ctx, SM_ECUDA, "device has no cooperative launch");
  SM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, PGROUPS * GT, smem));
  SM_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  if (per_sm < 1) return sm_fail(ctx, SM_ECUDA, "persistent kernel does not fit on one SM");
  ctx->persist_grid[idx] = per_sm * sms;
  return SM_OK;
}

static int persist_prepare32(sm_ctx *ctx) {
  return persist_prepare_k(ctx, k_persist<float>, persist_smem<float>(), 1);
}
static int persistx_prepare(sm_ctx *ctx) {
  return persist_prepare_k(ctx, k_persistx, (size_t)PGROUPS * persistx_group_smem(), 0);
}

template <typename A, typename K>
static int persist_coop_launch(sm_ctx *ctx, K kernel, const A &a, size_t smem, int idx) {
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_BAR, 0, sizeof(unsigned long long), ctx->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctx->persist_grid[idx]);
  cfg.blockDim = dim3(PGROUPS * GT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++ctx->n_launch;
  SM_CK(cudaLaunchKernelEx(&cfg, kernel, a));
  return SM_OK;
}

// One cooperative launch of the FP32 persistent kernel (error equation of
// the mixed form): the FMG ladder (fmg) or one V-cycle with `top` as
// finest level.
static int persist_launch(sm_ctx *ctx, const MG<float> &m, int top, int fmg, int loop, int bar_extra = 0) {
  int st = persist_prepare32(ctx);
  if (st) return st;
  PArgs<float> a;
  memset(&a, 0, sizeof a);
  a.phi = m.phi;
  a.rhs = m.rhs;
  a.old = m.old;
  a.gh = m.gh;
  a.nbr6 = ctx->nbr6;
  a.parent = ctx->parent;
  a.ijk = ctx->ijk;
  a.child = ctx->child;
  a.leaf = ctx->leaf;
  a.level = ctx->level;
  a.basis = ctx->basis;
  a.phi64 = ctx->phi;
  a.rhs64 = ctx->rhs;
  a.gh64 = ctx->gh;
  a.sc = ctx->dscal;
  a.bc = ctx->bc;
  a.lh = ctx->lh;
  for (int l = 0; l <= MAXL; ++l) a.level_off[l] = ctx->level_off[l];
  a.n_levels = ctx->n_levels;
  a.n_leaves = ctx->n_leaves;
  a.top = top;
  a.nu1 = ctx->cfg.nu1;
  a.nu2 = ctx->cfg.nu2;
  a.homog = m.homog;
  a.fmg = fmg;
  a.loop = loop;
  a.bar_extra = bar_extra;
  return persist_coop_launch(ctx, k_persist<float>, a, persist_smem<float>(), 1);
}

// One cooperative launch of the fixed-point FP64 persistent kernel: the
// FMG ladder (fmg; rhs already restricted), V-cycles with `top` as finest
// level, and with loop set the residual test after each cycle until
// SC_TOL or SC_MAXC is reached (SC_NORM, SC_REL, SC_CYC written at the
// end).  Without loop one V-cycle runs (or only the ladder when fmg is set).
static int persistx_launch(sm_ctx *ctx, int top, int fmg, int loop, int bar_extra = 0) {
  int st = persistx_prepare(ctx);
  if (st) return st;
  PArgsX a;
  memset(&a, 0, sizeof a);
  a.phx = ctx->phx;
  a.gx = ctx->gx;
  a.oldx = (long long *)ctx->old;
  a.ghx = ctx->ghx;
  a.rhs = ctx->rhs;
  a.nbr6 = ctx->nbr6;
  a.parent = ctx->parent;
  a.ijk = ctx->ijk;
  a.child = ctx->child;
  a.leaf = ctx->leaf;
  a.level = ctx->level;
  a.basis = ctx->basis;
  a.sc = ctx->dscal;
  a.bc = ctx->bc;
  a.lh = ctx->lh;
  for (int l = 0; l <= MAXL; ++l) a.level_off[l] = ctx->level_off[l];
  a.n_levels = ctx->n_levels;
  a.n_leaves = ctx->n_leaves;
  a.top = top;
  a.nu1 = ctx->cfg.nu1;
  a.nu2 = ctx->cfg.nu2;
  a.fmg = fmg;
  a.loop = loop;
  a.bar_extra = bar_extra;
  return persist_coop_launch(ctx, k_persistx, a, (size_t)PGROUPS * persistx_group_smem(), 0);
}

static int leaf_norm(sm_ctx *ctx, double *v, int slot);

// FMG ladder: restrict f, exact level-0 solve, then for each finer level
// prolong the solution (and its interpolation values) and run one V-cycle
// with that level on top; with norm_slot >= 0 (FP64) the residual max of
// the result is left in that slot
template <typename T>
static int fmg_ladder(sm_ctx *ctx, const MG<T> &m, int norm_slot = -1) {
  int st;
  if ((st = restrict_chain<T>(ctx, m.rhs, nullptr))) return st;
  if ((st = coarse_solve(ctx, m))) return st;
  for (int l = 1; l < ctx->n_levels; ++l) {
    if ((st = prolong_cf(ctx, m, l, 1))) return st;
    if ((st = vcycle(ctx, m, l, l == ctx->n_levels - 1 ? norm_slot : -1))) return st;
  }
  if (norm_slot >= 0 && ctx->n_levels == 1) return leaf_norm(ctx, ctx->phi, norm_slot);
  return SM_OK;
}

// max_leaf |f - L v| into slot (v's refinement ghosts must be current)
static int leaf_norm(sm_ctx *ctx, double *v, int slot) {
  SM_CK(cudaMemsetAsync(ctx->dscal + slot, 0, sizeof(unsigned long long), ctx->stream));
  sm_launch(ctx, k_resnorm, ctx->n_leaves, GT, 0, ctx->leaf, ctx->level, v, ctx->rhs, ctx->gh, ctx->nbr6, ctx->bc,
            ctx->lh, (float *)nullptr, ctx->dscal + slot);
  SM_CKL("resnorm");
  return SM_OK;
}

// outer FP64 residual of the mixed form: norm into SC_NORM, f32 = (float) r
static int leaf_resid32(sm_ctx *ctx) {
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_NORM, 0, sizeof(unsigned long long), ctx->stream));
  sm_launch(ctx, k_resnorm, ctx->n_leaves, GT, 0, ctx->leaf, ctx->level, ctx->phi, ctx->rhs, ctx->gh, ctx->nbr6,
            ctx->bc, ctx->lh, ctx->f32, ctx->dscal + SC_NORM);
  SM_CKL("resid32");
  return SM_OK;
}

// One defect-correction step of the mixed form, after leaf_resid32: solve
// the error equation A e = r in FP32 from e = 0 (one V-cycle, or the FMG
// ladder for the first step of an FMG solve), add e to phi in FP64 on leaf
// cells, re-average refined boxes, refresh the coarse interpolation values
// and the outer residual.
static int mixed_correction(sm_ctx *ctx, int ladder) {
  int st;
  size_t nc = (size_t)CELLS * ctx->n_boxes;
  SM_CK(cudaMemsetAsync(ctx->e32, 0, sizeof(float) * nc, ctx->stream));
  SM_CK(cudaMemsetAsync(ctx->gh32, 0, sizeof(float) * 6 * FACE * (size_t)ctx->n_boxes, ctx->stream));
  MG<float> m = mg32(ctx);
  if (ctx->persist) st = persist_launch(ctx, m, ctx->n_levels - 1, ladder, 0);
  else if (ladder) st = fmg_ladder(ctx, m);
  else st = vcycle(ctx, m, ctx->n_levels - 1);
  if (st) return st;
  sm_launch(ctx, k_add_corr, ctx->n_leaves, GT, 0, ctx->leaf, ctx->phi, ctx->e32);
  SM_CKL("add correction");
  if ((st = restrict_chain<double>(ctx, ctx->phi, nullptr))) return st;
  if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
  return leaf_resid32(ctx);
}

// internal status: a fixed-point solve left its range (never returned by
// an entry point: the solve runs again with a larger margin)
constexpr int SM_FX_RETRY = 100;

static int read_scalars(sm_ctx *ctx) {
  SM_CK(cudaMemcpyAsync(ctx->hscal, ctx->dscal, sizeof(double) * SC_N, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  unsigned long long e;
  memcpy(&e, &ctx->hscal[SC_ERR], sizeof e);
  if (e & ERR_BARRIER) return sm_fail(ctx, SM_ETIMEOUT, "grid barrier of the persistent kernel timed out");
  if (e & ~fx::FX_ERR_OVF) return sm_fail(ctx, SM_ESTATE, "device consistency check failed (flags 0x%llx)", e);
  if (e) return SM_FX_RETRY;
  return SM_OK;
}

// denominator of the relative residual, max_leaf |f - L 0| (old serves as
// the zero field), then the coarse interpolation values of phi restored
static int solve_prologue(sm_ctx *ctx) {
  int st;
  SM_CK(cudaMemsetAsync(ctx->old, 0, sizeof(double) * CELLS * (size_t)ctx->n_boxes, ctx->stream));
  if ((st = sm_fill_all_cf(ctx, ctx->old))) return st;
  if ((st = leaf_norm(ctx, ctx->old, SC_DEN))) return st;
  if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_CYC, 0, sizeof(unsigned long long), ctx->stream));
  return SM_OK;
}

static int rel_residual(sm_ctx *ctx, double *rel) {
  int st;
  if ((st = leaf_norm(ctx, ctx->phi, SC_NORM))) return st;
  if ((st = read_scalars(ctx))) return st;
  double num = ctx->hscal[SC_NORM], den = ctx->hscal[SC_DEN];
  *rel = den > 0.0 ? num / den : num;
  return SM_OK;
}

static int check_ready(sm_ctx *ctx) {
  if (!ctx) return SM_EINVAL;
  if (!ctx->arena || ctx->n_levels == 0) return sm_fail(ctx, SM_ESTATE, "octree not built");
  return SM_OK;
}

// ---- the FP64 solve in fixed point (kernels in mgfix.cuh) -----------------

static fx::FxLev fx_levels(const sm_ctx *ctx) {
  fx::FxLev fl;
  for (int l = 0; l < MAXL; ++l) {
    int e = 0;
    frexp(ctx->lh.h2[l], &e);  // h^2 < 2^e
    fl.eh[l] = e;
    fl.mh6[l] = -ctx->lh.h2[l] / 6.0;
  }
  return fl;
}

// the exponent margin of the next solve's scale (host value, not captured)
static int fx_set_margin(sm_ctx *ctx) {
  const unsigned long long m = (unsigned long long)ctx->fx_margin;
  memcpy(&ctx->hscal[SC_FXM], &m, sizeof m);
  SM_CK(cudaMemcpyAsync(ctx->dscal + SC_FXM, ctx->hscal + SC_FXM, sizeof(double), cudaMemcpyHostToDevice,
                        ctx->stream));
  return SM_OK;
}

// Ghat of every refinement face (each level from the level below)
static int fx_fill_cf(sm_ctx *ctx) {
  if (ctx->lbase + 1 >= ctx->n_levels) return SM_OK;
  const int lo = ctx->level_off[ctx->lbase + 1], n = ctx->n_boxes - lo;
  if (n <= 0) return SM_OK;
  sm_launch(ctx, fx::k_ffill_cf, n, 64, 0, lo, ctx->phx, ctx->ghx, ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc,
            ctx->dscal);
  SM_CKL("fill Ghat");
  return SM_OK;
}

// scale of the solve (from phi, every h^2 f and 2g), the potential and G
// of every box in quanta with the residual norm of the zero potential in
// SC_DEN, and (ghat) the refinement-face sums
static int fx_prologue(sm_ctx *ctx, bool ghat) {
  const fx::FxLev fl = fx_levels(ctx);
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_FXI, 0, sizeof(unsigned long long), ctx->stream));
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_DEN, 0, sizeof(unsigned long long), ctx->stream));
  const int grid = ctx->n_boxes < 608 ? 2 * ctx->n_boxes : 1216;
  sm_launch(ctx, fx::k_fx_expo, grid, 256, 0, ctx->n_boxes, ctx->level, ctx->phi, ctx->rhs, fl, ctx->dscal);
  sm_launch(ctx, fx::k_fx_scale, 1, 1, 0, ctx->bc, ctx->dscal);
  sm_launch(ctx, fx::k_fx_init, ctx->n_boxes, GT, 0, ctx->level, ctx->child, ctx->nbr6, ctx->phi, ctx->rhs,
            ctx->phx, ctx->gx, fl, ctx->bc, ctx->lh, ctx->dscal, ctx->dscal + SC_DEN);
  SM_CKL("fixed-point prologue");
  return ghat ? fx_fill_cf(ctx) : SM_OK;
}

// phi from the fixed-point potential (skipped on the device when the solve
// left its range), then the FP64 interpolation values of phi
static int fx_epilogue(sm_ctx *ctx) {
  sm_launch(ctx, fx::k_fx_final, ctx->n_boxes, GT, 0, ctx->phx, ctx->phi, ctx->dscal);
  SM_CKL("fixed-point epilogue");
  return sm_fill_all_cf(ctx, ctx->phi);
}

// nu red-black sweeps of level l (two colour passes each, in place); with
// skip_first the first colour pass has already run (k_ffas_color0).  A
// level of at least ctx->rows_min boxes runs the row kernel (4 cells and
// 16-byte row loads per thread, fewer instructions per cell); a level that
// is one partial wave of blocks runs the half-row kernel (2 cells per
// thread, twice the warps to hide its load latency).  Both give the bits
// of the box kernel (fx_color_box, which the persistent kernel runs).
static int fx_smooth(sm_ctx *ctx, int l, int nu, bool skip_first = false) {
  const int n = lvl_n(ctx, l);
  if (!n) return SM_OK;
  for (int s = 0; s < nu; ++s)
    for (int color = 0; color < 2; ++color) {
      if (skip_first && s == 0 && color == 0) continue;
      if (n >= ctx->rows_min)
        sm_launch(ctx, fx::k_fcolor_rows, (n + fx::RBOX - 1) / fx::RBOX, 64 * fx::RBOX, 0, ctx->level_off[l], n,
                  color, ctx->phx, ctx->gx, ctx->ghx, ctx->nbr6, ctx->bc, ctx->dscal);
      else
        sm_launch(ctx, fx::k_fcolor_half, n, 128, 0, ctx->level_off[l], color, ctx->phx, ctx->gx, ctx->ghx,
                  ctx->nbr6, ctx->bc, ctx->dscal);
    }
  SM_CKL("rbgs");
  return SM_OK;
}

// level-0 solve; fas: complete level 0's FAS right-hand side first (the
// down leg of a V-cycle has restricted into it)
static int fx_coarse(sm_ctx *ctx, bool fas = false) {
  int st = ensure_basis(ctx);
  if (st) return st;
  sm_launch(ctx, fx::k_fcoarse8, 8, 64, 0, ctx->phx, ctx->gx, (long long *)ctx->old, ctx->basis, ctx->bc,
            ctx->lh.h2[0], ctx->lh.inv_h2[0], (int)fas, ctx->dscal);
  SM_CKL("coarse solve");
  return SM_OK;
}

// leaves of level l whose residual norm goes to slot (none when slot < 0)
static fx::FxNorm fx_norm_of(sm_ctx *ctx, int l, int slot) {
  fx::FxNorm nm = {};
  if (slot < 0 || l < 0) return nm;
  nm.leaf = ctx->leaf + ctx->leaf_level_off[l];
  nm.n = ctx->leaf_level_off[l + 1] - ctx->leaf_level_off[l];
  nm.rhs = ctx->rhs;
  nm.inv_h2 = ctx->lh.inv_h2[l];
  nm.slot = ctx->dscal + slot;
  return nm;
}

static int fx_prolong(sm_ctx *ctx, int l, int mode, fx::FxNorm nm) {
  const int n = lvl_n(ctx, l);
  if (n >= ctx->rows_min)
    sm_launch(ctx, fx::k_fprolong_rows, (n + 1) / 2 + nm.n, 128, 0, ctx->level_off[l], n, mode, ctx->phx,
              (const long long *)ctx->old, ctx->ghx, ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc, ctx->dscal, nm);
  else
    sm_launch(ctx, fx::k_fprolong_half, n + nm.n, GT, 0, ctx->level_off[l], n, mode, ctx->phx,
              (const long long *)ctx->old, ctx->ghx, ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc, ctx->dscal, nm);
  SM_CKL("prolong");
  return SM_OK;
}

// residual max of the leaves listed at [off, off + n) into slot
static int fx_leaf_norm(sm_ctx *ctx, int off, int n, int slot) {
  if (n <= 0) return SM_OK;
  sm_launch(ctx, fx::k_fresnorm, n, GT, 0, ctx->leaf + off, ctx->level, ctx->phx, ctx->rhs, ctx->ghx, ctx->nbr6,
            ctx->bc, ctx->lh, ctx->dscal, ctx->dscal + slot);
  SM_CKL("resnorm");
  return SM_OK;
}

// FAS V-cycle in fixed point with `top` as finest level; with norm_slot >= 0
// (top the finest level) max_leaf |f - L phi| is left in that slot.  The
// Ghat values of every level <= top must match the level below on entry
// (the prologue and every up-sweep leave them so).
static int fx_vcycle(sm_ctx *ctx, int top, int norm_slot = -1) {
  int st;
  if (norm_slot >= 0)
    SM_CK(cudaMemsetAsync(ctx->dscal + norm_slot, 0, sizeof(unsigned long long), ctx->stream));
  bool fused = false;  // the first colour pass of level l has run (k_ffas_color0)
  for (int l = top; l >= 1; --l) {
    if ((st = fx_smooth(ctx, l, ctx->cfg.nu1, fused))) return st;
    // on a level of one partial wave below another, the FAS completion also
    // runs the level's first colour pass; the restriction then copies the
    // whole level below into old first
    fused = l - 1 >= 1 && ctx->cfg.nu1 > 0 && lvl_n(ctx, l) < ctx->rows_min && lvl_n(ctx, l - 1) < ctx->rows_min;
    if (lvl_n(ctx, l) >= ctx->rows_min) {
      sm_launch(ctx, fx::k_fresid_restrict_rows, lvl_n(ctx, l), 64, 0, ctx->level_off[l], ctx->phx, ctx->gx,
                ctx->ghx, ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc, ctx->dscal);
    } else {
      const int nl = fused ? ctx->leaf_level_off[l] - ctx->leaf_level_off[l - 1] : 0;
      sm_launch(ctx, fx::k_fresid_restrict, lvl_n(ctx, l) + nl, GT, 0, ctx->level_off[l], lvl_n(ctx, l), ctx->phx,
                ctx->gx, ctx->ghx, ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc, ctx->dscal,
                fused ? (long long *)ctx->old : nullptr, ctx->leaf + ctx->leaf_level_off[l - 1]);
    }
    if (fused)
      sm_launch(ctx, fx::k_ffas_color0, lvl_n(ctx, l - 1), GT, 0, ctx->level_off[l - 1], ctx->phx,
                (const long long *)ctx->old, ctx->gx, ctx->ghx, ctx->nbr6, ctx->child, ctx->bc, ctx->dscal);
    else if (l - 1 >= 1)  // level 0's FAS completion runs in the level-0 solve
      sm_launch(ctx, fx::k_ffas, lvl_n(ctx, l - 1), GT, 0, ctx->level_off[l - 1], ctx->phx, (long long *)ctx->old,
                ctx->gx, ctx->ghx, ctx->nbr6, ctx->child, ctx->bc, ctx->dscal);
    SM_CKL("vcycle down");
  }
  if ((st = fx_coarse(ctx, top >= 1))) return st;
  for (int l = 1; l <= top; ++l) {
    if ((st = fx_prolong(ctx, l, 0, fx_norm_of(ctx, norm_slot >= 0 ? l - 1 : -1, norm_slot)))) return st;
    if ((st = fx_smooth(ctx, l, ctx->cfg.nu2))) return st;
  }
  if (norm_slot >= 0) {
    const int off = ctx->leaf_level_off[top];
    return fx_leaf_norm(ctx, off, ctx->leaf_level_off[top + 1] - off, norm_slot);
  }
  return SM_OK;
}

// FMG ladder on the restricted right-hand side: level-0 solve, then for
// each finer level the prolonged solution and one V-cycle with that level
// on top (the residual of the result in norm_slot)
static int fx_fmg_ladder(sm_ctx *ctx, int norm_slot) {
  int st;
  if ((st = fx_coarse(ctx))) return st;
  for (int l = 1; l < ctx->n_levels; ++l) {
    if ((st = fx_prolong(ctx, l, 1, fx::FxNorm{}))) return st;
    if ((st = fx_vcycle(ctx, l, l == ctx->n_levels - 1 ? norm_slot : -1))) return st;
  }
  if (ctx->n_levels == 1) {
    SM_CK(cudaMemsetAsync(ctx->dscal + norm_slot, 0, sizeof(unsigned long long), ctx->stream));
    return fx_leaf_norm(ctx, 0, ctx->n_leaves, norm_slot);
  }
  return SM_OK;
}

// Work of an FP64 solve before its cycle loop: the restricted rhs of FMG,
// the fixed-point scale and arrays with the residual norm of phi = 0 (the
// denominator); FMG then runs its ladder (leaving the residual of its
// result in SC_NORM) unless the persistent kernel will.
static int fx_solve_prefix(sm_ctx *ctx, int fmg, bool ladder) {
  int st;
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_CYC, 0, sizeof(unsigned long long), ctx->stream));
  if (fmg && (st = restrict_chain<double>(ctx, ctx->rhs, nullptr))) return st;
  if ((st = fx_prologue(ctx, !fmg))) return st;
  if (fmg && ladder) return fx_fmg_ladder(ctx, SC_NORM);
  return SM_OK;
}

// ---- solve bodies shared by the graph and the direct paths ----------------
//
// kind 0: FP64 solve (warm start), 1: FP64 FMG, 2: mixed solve, 3: mixed FMG.
// prefix(): work before the cycle loop; for kinds 1 and 3 it ends with the
// residual of the FMG result.  body(): one loop iteration up to and
// including the residual it leaves in SC_NORM.

static int solve_prefix(sm_ctx *ctx, int kind) {
  int st;
  switch (kind) {
    case 0:
    case 1:
      return fx_solve_prefix(ctx, kind, true);
    case 2:
      if ((st = solve_prologue(ctx))) return st;
      return leaf_resid32(ctx);
    default:
      // phi = 0: its outer residual is the denominator itself
      SM_CK(cudaMemsetAsync(ctx->phi, 0, sizeof(double) * CELLS * (size_t)ctx->n_boxes, ctx->stream));
      if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
      SM_CK(cudaMemsetAsync(ctx->dscal + SC_CYC, 0, sizeof(unsigned long long), ctx->stream));
      if ((st = leaf_resid32(ctx))) return st;
      SM_CK(cudaMemcpyAsync(ctx->dscal + SC_DEN, ctx->dscal + SC_NORM, sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, ctx->stream));
      return mixed_correction(ctx, 1);
  }
}

static int solve_body(sm_ctx *ctx, int kind) {
  if (kind >= 2) return mixed_correction(ctx, 0);
  return fx_vcycle(ctx, ctx->n_levels - 1, SC_NORM);
}

// work after the cycle loop: the FP64 kinds convert the fixed-point result
static int solve_suffix(sm_ctx *ctx, int kind) { return kind < 2 ? fx_epilogue(ctx) : SM_OK; }

// ---- graph-captured solves with a device-side cycle loop ------------------

static sm_graph *graph_of(sm_ctx *ctx, int kind) {
  switch (kind) {
    case 0: return &ctx->g_solve;
    case 1: return &ctx->g_fmg;
    case 2: return &ctx->g_solve32;
    default: return &ctx->g_fmg32;
  }
}

void sm_drop_graphs(sm_ctx *ctx) {
  for (auto *g : {&ctx->g_solve, &ctx->g_fmg, &ctx->g_solve32, &ctx->g_fmg32}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
}

static int end_captures(sm_ctx *ctx, cudaStream_t saved, int st) {
  cudaGraph_t tmp = nullptr;
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(ctx->cap2, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaStreamEndCapture(ctx->cap2, &tmp);
    if (tmp) cudaGraphDestroy(tmp);
  }
  tmp = nullptr;
  if (cudaStreamIsCapturing(ctx->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaStreamEndCapture(ctx->cap, &tmp);
    if (tmp) cudaGraphDestroy(tmp);
  }
  ctx->stream = saved;
  cudaGetLastError();
  return st;
}

// Capture prefix + WHILE(cond){ body; check } into an executable graph.
// FMG kinds check once after the prefix (the FMG result counts as cycle
// 1); the others run the body at least once.
static int capture_solve(sm_ctx *ctx, int kind, sm_graph *out) {
  cudaStream_t saved = ctx->stream;
  if (!ctx->cap) SM_CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
  if (!ctx->cap2) SM_CK(cudaStreamCreateWithFlags(&ctx->cap2, cudaStreamNonBlocking));
  {
    int st = ensure_basis(ctx);  // once per context, outside any graph
    if (st) return st;
  }
  const int fmg = kind == 1 || kind == 3;
  if (ctx->persist) {
    int st = kind < 2 ? persistx_prepare(ctx) : persist_prepare32(ctx);
    if (st) return st;
  }
  if (ctx->persist && kind < 2) {
    // prefix + one persistent launch holding the FMG ladder and the cycle
    // loop + the conversion of the result
    SM_CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    ctx->stream = ctx->cap;
    long long n0 = ctx->n_launch;
    int st = fx_solve_prefix(ctx, fmg, false);
    if (!st) st = persistx_launch(ctx, ctx->n_levels - 1, fmg, 1);
    if (!st) st = fx_epilogue(ctx);
    if (st) return end_captures(ctx, saved, st);
    out->prefix_launches = ctx->n_launch - n0;
    out->body_launches = 0;
    cudaGraph_t whole = nullptr;
    if (cudaStreamEndCapture(ctx->cap, &whole) != cudaSuccess)
      return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "end capture"));
    ctx->stream = saved;
    cudaError_t e = cudaGraphInstantiate(&out->exec, whole, 0);
    cudaGraphDestroy(whole);
    if (e != cudaSuccess) return sm_cuda_check(ctx, e, "graph instantiate");
    ctx->n_launch -= out->prefix_launches;
    return SM_OK;
  }
  SM_CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
  ctx->stream = ctx->cap;
  int st = SM_OK;
  cudaGraph_t g = nullptr, body = nullptr, whole = nullptr;
  cudaStreamCaptureStatus cs;
  cudaGraphConditionalHandle h;
  cudaGraphNode_t node;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  // the node-parameter union has no default constructor: zeroed raw storage
  alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
  memset(pbuf, 0, sizeof pbuf);
  cudaGraphNodeParams &p = *reinterpret_cast<cudaGraphNodeParams *>(pbuf);
  long long n0;
  if (cudaStreamGetCaptureInfo(ctx->cap, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "capture info"));
  if (cudaGraphConditionalHandleCreate(&h, g, fmg ? 0u : 1u, cudaGraphCondAssignDefault) != cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "conditional handle"));
  n0 = ctx->n_launch;
  if ((st = solve_prefix(ctx, kind))) return end_captures(ctx, saved, st);
  if (fmg) {
    sm_launch(ctx, k_loop_check, 1, 1, 0, h, ctx->dscal, 1, ctx->hist);
  }
  out->prefix_launches = ctx->n_launch - n0;
  if (cudaStreamGetCaptureInfo(ctx->cap, &cs, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "capture deps"));
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &p) != cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "while node"));
  body = p.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(ctx->cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
      cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "capture deps update"));
  if (cudaStreamBeginCaptureToGraph(ctx->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "body capture"));
  ctx->stream = ctx->cap2;
  n0 = ctx->n_launch;
  if ((st = solve_body(ctx, kind))) return end_captures(ctx, saved, st);
  sm_launch(ctx, k_loop_check, 1, 1, 0, h, ctx->dscal, 1, ctx->hist);
  out->body_launches = ctx->n_launch - n0;
  if (cudaStreamEndCapture(ctx->cap2, &body) != cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "end body capture"));
  ctx->stream = ctx->cap;
  n0 = ctx->n_launch;
  if ((st = solve_suffix(ctx, kind))) return end_captures(ctx, saved, st);
  out->prefix_launches += ctx->n_launch - n0;
  if (cudaStreamEndCapture(ctx->cap, &whole) != cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "end capture"));
  ctx->stream = saved;
  cudaError_t e = cudaGraphInstantiate(&out->exec, whole, 0);
  cudaGraphDestroy(whole);
  if (e != cudaSuccess) return sm_cuda_check(ctx, e, "graph instantiate");
  // captured launches are counted when the graph runs
  ctx->n_launch -= out->prefix_launches + out->body_launches;
  return SM_OK;
}

// One attempt of a solve: SM_OK with the cycle count and relative
// residual, SM_FX_RETRY when the fixed-point potential left its range (phi
// is then unchanged), or an error.
static int run_solve_once(sm_ctx *ctx, int kind, double tol, int max_cycles, int *cycles, double *rel_res) {
  int st;
  int c = 0;
  double rel = 0.0;
  const int fmg = kind & 1;
  if (kind < 2 && (st = fx_set_margin(ctx))) return st;
  if (ctx->graphs) {
    sm_graph *g = graph_of(ctx, kind);
    if (!g->exec && (st = capture_solve(ctx, kind, g))) return st;
    SM_CK(cudaGraphLaunch(g->exec, ctx->stream));
    st = read_scalars(ctx);
    unsigned long long cc;
    memcpy(&cc, &ctx->hscal[SC_CYC], sizeof cc);
    c = (int)cc;
    rel = ctx->hscal[SC_REL];
    ctx->n_launch += g->prefix_launches + g->body_launches * (long long)(fmg ? c - 1 : c);
    if (st) return st;
  } else if (ctx->persist && kind < 2) {
    if ((st = ensure_basis(ctx))) return st;
    if ((st = fx_solve_prefix(ctx, fmg, false))) return st;
    if ((st = persistx_launch(ctx, ctx->n_levels - 1, fmg, 1))) return st;
    if ((st = fx_epilogue(ctx))) return st;
    if ((st = read_scalars(ctx))) return st;
    unsigned long long cc;
    memcpy(&cc, &ctx->hscal[SC_CYC], sizeof cc);
    c = (int)cc;
    rel = ctx->hscal[SC_REL];
  } else {
    if ((st = ensure_basis(ctx))) return st;
    if ((st = solve_prefix(ctx, kind))) return st;
    bool go = true;
    ctx->hhist.clear();
    if (fmg) {
      c = 1;
      if ((st = read_scalars(ctx))) return st;
      double num = ctx->hscal[SC_NORM], den = ctx->hscal[SC_DEN];
      rel = den > 0.0 ? num / den : num;
      ctx->hhist.push_back(rel);
      go = rel > tol && c < max_cycles;
    }
    while (go) {
      if ((st = solve_body(ctx, kind))) return st;
      ++c;
      if ((st = read_scalars(ctx))) return st;
      double num = ctx->hscal[SC_NORM], den = ctx->hscal[SC_DEN];
      rel = den > 0.0 ? num / den : num;
      ctx->hhist.push_back(rel);
      go = rel > tol && c < max_cycles;
    }
    if ((st = solve_suffix(ctx, kind))) return st;
  }
  *cycles = c;
  *rel_res = rel;
  return SM_OK;
}

// after an attempt that left the fixed-point range: clear the flag and
// widen the scale (false when the margin is exhausted)
static int fx_widen(sm_ctx *ctx, bool *again) {
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_ERR, 0, sizeof(unsigned long long), ctx->stream));
  *again = ctx->fx_margin < 5 + 4 * 8;
  if (*again) ctx->fx_margin += 8;
  return SM_OK;
}

static void vcycle_model(const sm_ctx *ctx, int top, bool fixed, double *bytes, double *ops);

static void json_num(FILE *f, double v) {
  if (v == v && v - v == 0.0) fprintf(f, "%.17g", v);
  else fputs("null", f);
}

// one JSON line of the metrics log for the solve that just ended (its
// stream synchronised): cycles, relative residual after each cycle, time
// from the events around the call (retries of a widened fixed-point scale
// included), algorithmic bytes of the V-cycles (the per-level model of
// sm_kernel_bench class 2 times the cycle count; an FMG ladder counts as
// one cycle) and the bandwidth they imply
static int log_solve(sm_ctx *ctx, int fmg, int kind, double tol, int c, double rel, int st) {
  SM_CK(cudaEventRecord(ctx->mlog_ev[1], ctx->stream));
  SM_CK(cudaEventSynchronize(ctx->mlog_ev[1]));
  float ms = 0.0f;
  SM_CK(cudaEventElapsedTime(&ms, ctx->mlog_ev[0], ctx->mlog_ev[1]));
  std::vector<double> hist;
  const char *path = "persistent";
  if (ctx->graphs) {
    path = "graph";
    hist.resize((size_t)std::max(0, std::min(c, SM_HIST)));
    if (!hist.empty())
      SM_CK(cudaMemcpy(hist.data(), ctx->hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost));
  } else if (!(ctx->persist && kind < 2)) {
    path = "host";
    hist = ctx->hhist;
  }
  double by = 0.0, ops = 0.0;
  if (ctx->n_levels > 1) vcycle_model(ctx, ctx->n_levels - 1, kind < 2, &by, &ops);
  const double bytes = by * c, gbs = ms > 0.0f ? bytes / (ms * 1e-3) / 1e9 : 0.0;
  FILE *f = ctx->mlog;
  fprintf(f, "{\"seq\": %lld, \"call\": \"%s\", \"precision\": \"%s\", \"path\": \"%s\", ",
          ++ctx->mlog_seq, fmg ? "fmg" : "solve", kind < 2 ? "fp64" : "mixed", path);
  fprintf(f, "\"boxes\": %d, \"levels\": %d, \"leaf_cells\": %lld, \"tol\": ", ctx->n_boxes, ctx->n_levels,
          (long long)ctx->n_leaves * CELLS);
  json_num(f, tol);
  fprintf(f, ", \"status\": %d, \"cycles\": %d, \"rel\": ", st, c);
  json_num(f, rel);
  fputs(", \"residual_history\": [", f);
  for (size_t i = 0; i < hist.size(); ++i) {
    if (i) fputs(", ", f);
    json_num(f, hist[i]);
  }
  fputs("], \"ms\": ", f);
  json_num(f, ms);
  fputs(", \"vcycle_bytes\": ", f);
  json_num(f, by);
  fputs(", \"bytes\": ", f);
  json_num(f, bytes);
  fputs(", \"gbs\": ", f);
  json_num(f, gbs);
  fputs(", \"hbm_frac\": ", f);
  if (ctx->mlog_peak > 0.0) json_num(f, gbs / ctx->mlog_peak);
  else fputs("null", f);
  fputs("}\n", f);
  fflush(f);
  return SM_OK;
}

static int run_solve_logged(sm_ctx *ctx, int fmg, double tol, int max_cycles, int *cycles, double *rel_res);

static int run_solve(sm_ctx *ctx, int fmg, double tol, int max_cycles, int *cycles, double *rel_res) {
  if (!ctx->mlog) return run_solve_logged(ctx, fmg, tol, max_cycles, cycles, rel_res);
  SM_CK(cudaEventRecord(ctx->mlog_ev[0], ctx->stream));
  int c = 0;
  double rel = 0.0;
  const int st = run_solve_logged(ctx, fmg, tol, max_cycles, &c, &rel);
  if (st == SM_OK || st == SM_ENOCONV) {
    const int kind = (ctx->cfg.precision == SM_MIXED ? 2 : 0) + (fmg ? 1 : 0);
    const int lst = log_solve(ctx, fmg, kind, tol, c, rel, st);
    if (lst) return lst;
  }
  if (cycles) *cycles = c;
  if (rel_res) *rel_res = rel;
  return st;
}

// the solve itself (run_solve adds the metrics line when a log is open)
static int run_solve_logged(sm_ctx *ctx, int fmg, double tol, int max_cycles, int *cycles, double *rel_res) {
  int st;
  int c = 0;
  double rel = 0.0;
  const int kind = (ctx->cfg.precision == SM_MIXED ? 2 : 0) + (fmg ? 1 : 0);
  // stopping parameters of the device-side loops
  ctx->hscal[SC_TOL] = tol;
  unsigned long long mc = (unsigned long long)max_cycles;
  memcpy(&ctx->hscal[SC_MAXC], &mc, sizeof mc);
  SM_CK(cudaMemcpyAsync(ctx->dscal + SC_TOL, ctx->hscal + SC_TOL, 2 * sizeof(double), cudaMemcpyHostToDevice,
                        ctx->stream));
  while ((st = run_solve_once(ctx, kind, tol, max_cycles, &c, &rel)) == SM_FX_RETRY) {
    bool again = false;
    if ((st = fx_widen(ctx, &again))) return st;
    if (!again)
      return sm_fail(ctx, SM_ENOCONV, "potential or right-hand side not finite or beyond 2^%d of its scale",
                     ctx->fx_margin);
  }
  if (st) return st;
  if (cycles) *cycles = c;
  if (rel_res) *rel_res = rel;
  return rel <= tol ? SM_OK : sm_fail(ctx, SM_ENOCONV, "residual %.3e > tol %.3e after %d cycles", rel, tol, c);
}

extern "C" int sm_set_metrics_log(sm_ctx *ctx, const char *path, double hbm_peak_gbs) {
  if (!ctx) return SM_EINVAL;
  if (ctx->mlog) {
    fclose(ctx->mlog);
    ctx->mlog = nullptr;
  }
  if (!path || !*path) return SM_OK;
  if (!ctx->mlog_ev[0]) {
    SM_CK(cudaEventCreate(&ctx->mlog_ev[0]));
    SM_CK(cudaEventCreate(&ctx->mlog_ev[1]));
  }
  ctx->mlog = fopen(path, "a");
  if (!ctx->mlog) return sm_fail(ctx, SM_EINVAL, "cannot open the metrics log %s", path);
  ctx->mlog_peak = hbm_peak_gbs > 0.0 ? hbm_peak_gbs : 0.0;
  return SM_OK;
}

// relative residual of the current potential (denominator recomputed);
// leaves the coarse interpolation values of phi current
int sm_rel_residual_now(sm_ctx *ctx, double *rel) {
  int st = solve_prologue(ctx);
  if (st) return st;
  return rel_residual(ctx, rel);
}

extern "C" int sm_fill_ghosts_range(sm_ctx *ctx, int var, int level_lo, int level_hi) {
  int st = check_ready(ctx);
  if (st) return st;
  if (var != SM_PHI || level_lo < 0 || level_hi >= ctx->n_levels || level_lo > level_hi) return SM_EINVAL;
  for (int l = level_lo; l <= level_hi; ++l)
    if ((st = sm_mg_fill_cf(ctx, ctx->phi, l, 0))) return st;
  return SM_OK;
}

extern "C" int sm_get_ghosts(sm_ctx *ctx, int var, double *host, int n_boxes) {
  int st = check_ready(ctx);
  if (st) return st;
  if (var != SM_PHI || !host || n_boxes < 0 || n_boxes > ctx->n_boxes) return SM_EINVAL;
  SM_CK(cudaMemcpyAsync(host, ctx->gh, sizeof(double) * 6 * FACE * (size_t)n_boxes, cudaMemcpyDeviceToHost,
                        ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  return SM_OK;
}

extern "C" int sm_fill_ghosts(sm_ctx *ctx, int var, int level) {
  int st = check_ready(ctx);
  if (st) return st;
  if (var != SM_PHI || level < 0 || level >= ctx->n_levels) return SM_EINVAL;
  return sm_mg_fill_cf(ctx, ctx->phi, level, 0);
}

extern "C" int sm_mg_vcycle(sm_ctx *ctx, int n_cycles, double *rel_res) {
  SM_RANGE();
  int st = check_ready(ctx);
  if (st) return st;
  if (n_cycles < 0) return SM_EINVAL;
  if ((st = ensure_basis(ctx))) return st;
  const int top = ctx->n_levels - 1;
  for (;;) {
    if ((st = fx_set_margin(ctx))) return st;
    if ((st = fx_solve_prefix(ctx, 0, false))) return st;
    for (int c = 0; c < n_cycles; ++c)
      if ((st = ctx->persist ? persistx_launch(ctx, top, 0, 0) : fx_vcycle(ctx, top))) return st;
    if ((st = fx_epilogue(ctx))) return st;
    if ((st = read_scalars(ctx)) != SM_FX_RETRY) break;
    bool again = false;
    if ((st = fx_widen(ctx, &again))) return st;
    if (!again) return sm_fail(ctx, SM_ENOCONV, "potential or right-hand side beyond the fixed-point range");
  }
  if (st) return st;
  double rel = 0.0;
  if ((st = rel_residual(ctx, &rel))) return st;
  if (rel_res) *rel_res = rel;
  return SM_OK;
}

extern "C" int sm_mg_solve(sm_ctx *ctx, double tol, int max_cycles, int *cycles, double *rel_res) {
  SM_RANGE();
  int st = check_ready(ctx);
  if (st) return st;
  if (max_cycles < 1) return SM_EINVAL;
  return run_solve(ctx, 0, tol, max_cycles, cycles, rel_res);
}

extern "C" int sm_mg_fmg(sm_ctx *ctx, double tol, int max_cycles, int *cycles, double *rel_res) {
  SM_RANGE();
  int st = check_ready(ctx);
  if (st) return st;
  if (max_cycles < 1) return SM_EINVAL;
  return run_solve(ctx, 1, tol, max_cycles, cycles, rel_res);
}

extern "C" int sm_set_graphs(sm_ctx *ctx, int enable) {
  if (!ctx) return SM_EINVAL;
  ctx->graphs = enable != 0;
  return SM_OK;
}

extern "C" int sm_persist_barrier_selftest(sm_ctx *ctx) {
  int st = check_ready(ctx);
  if (st) return st;
  if (ctx->n_levels < 2) return SM_EINVAL;
  if ((st = ensure_basis(ctx))) return st;
  if ((st = read_scalars(ctx))) return st;  // no earlier error may be pending
  // every barrier waits for one block more than the grid holds
  if ((st = persistx_launch(ctx, ctx->n_levels - 1, 0, 0, 1))) return st;
  st = read_scalars(ctx);
  // the launch ended by itself: clear its flag so the context stays usable
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_ERR, 0, sizeof(unsigned long long), ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  return st;
}

extern "C" int sm_set_persistent(sm_ctx *ctx, int enable) {
  if (!ctx) return SM_EINVAL;
  if (ctx->persist != (enable != 0)) sm_drop_graphs(ctx);
  ctx->persist = enable != 0;
  return SM_OK;
}

extern "C" int sm_set_row_kernels(sm_ctx *ctx, int min_boxes) {
  if (!ctx || min_boxes < 0) return SM_EINVAL;
  if (ctx->rows_min != min_boxes) sm_drop_graphs(ctx);
  ctx->rows_min = min_boxes;
  return SM_OK;
}

extern "C" int sm_set_pdl(sm_ctx *ctx, int enable) {
  if (!ctx) return SM_EINVAL;
  if (ctx->pdl != (enable != 0)) sm_drop_graphs(ctx);
  ctx->pdl = enable != 0;
  return SM_OK;
}

// Algorithmic bytes and FP64 instructions of one V-cycle from `top` (the
// per-level model stated with sm_kernel_bench).  fixed: the FP64 solve's
// fixed-point cycle (colour passes of 12 B per cell in its colour-split
// layout, no FP64 work outside the level-0 solve); otherwise the FP32
// cycle of the mixed form (colour passes of 8 B per cell).
static void vcycle_model(const sm_ctx *ctx, int top, bool fixed, double *bytes, double *ops) {
  double by = 16.0 * CELLS, op = 60.0 * CELLS;  // level-0 solve
  const double sweeps = ctx->cfg.nu1 + ctx->cfg.nu2;
  for (int l = 1; l <= top; ++l) {
    const double n = (double)CELLS * lvl_n(ctx, l), nc = (double)CELLS * lvl_n(ctx, l - 1);
    const double refined = n / 8.0;  // cells of the refined boxes of level l-1
    if (fixed) {
      by += sweeps * 24.0 * n + 18.0 * n + 16.0 * nc + 16.0 * refined + 18.0 * n;
    } else {
      by += 0.5 * (sweeps * 2.0 * 16.0 * n + 18.0 * n + 16.0 * nc + 16.0 * refined + 18.0 * n);
    }
  }
  *bytes = by;
  *ops = fixed ? op : 0.0;
}

// Average launch duration of a kernel class (see the header for the
// classes and their algorithmic bytes and operations).
extern "C" int sm_kernel_bench(sm_ctx *ctx, int kclass, int reps, double *us_per_launch, long long *launches,
                               double *bytes_per_launch, double *flops_per_launch) {
  int st = check_ready(ctx);
  if (st) return st;
  if (kclass < 0 || kclass >= K_NCLASS || reps < 1) return SM_EINVAL;
  int top = ctx->n_levels - 1;
  if (top < 1) return SM_EINVAL;
  if (kclass != K_VCYCLE32) {
    // the fixed-point arrays and scale of the current potential
    if ((st = ensure_basis(ctx))) return st;
    if ((st = fx_set_margin(ctx))) return st;
    if ((st = fx_solve_prefix(ctx, 0, false))) return st;
  }
  if (kclass == K_PERSIST) {
    if ((st = persistx_launch(ctx, top, 0, 0))) return st;  // warm
    cudaEvent_t a, b;
    SM_CK(cudaEventCreate(&a));
    SM_CK(cudaEventCreate(&b));
    SM_CK(cudaEventRecord(a, ctx->stream));
    for (int r = 0; r < reps && !st; ++r) st = persistx_launch(ctx, top, 0, 0);
    SM_CK(cudaEventRecord(b, ctx->stream));
    SM_CK(cudaEventSynchronize(b));
    float ms = 0.f;
    SM_CK(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) return st;
    if ((st = read_scalars(ctx)) && st != SM_FX_RETRY) return st;
    if (st == SM_FX_RETRY) SM_CK(cudaMemsetAsync(ctx->dscal + SC_ERR, 0, sizeof(unsigned long long), ctx->stream));
    double by, fl;
    vcycle_model(ctx, top, true, &by, &fl);
    if (us_per_launch) *us_per_launch = 1e3 * ms / reps;
    if (launches) *launches = reps;
    if (bytes_per_launch) *bytes_per_launch = by;
    if (flops_per_launch) *flops_per_launch = fl;
    return SM_OK;
  }
  const bool whole = kclass == K_VCYCLE || kclass == K_VCYCLE32;
  if (kclass == K_VCYCLE32 && ctx->cfg.precision != SM_MIXED)
    return sm_fail(ctx, SM_EINVAL, "class 3 needs a mixed-precision context");
  if (kclass == K_VCYCLE32) {
    if ((st = ensure_basis(ctx))) return st;
    if ((st = solve_prologue(ctx))) return st;
    if ((st = leaf_resid32(ctx))) return st;
  }
  cudaStream_t saved = ctx->stream;
  if (!ctx->cap) SM_CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
  SM_CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
  ctx->stream = ctx->cap;
  long long n = 0, n0 = ctx->n_launch;
  double bytes = 0.0;
  for (int r = 0; r < reps; ++r) {
    if (kclass == K_VCYCLE) {
      if ((st = fx_vcycle(ctx, top))) break;
      ++n;
      continue;
    }
    if (kclass == K_VCYCLE32) {
      if ((st = vcycle(ctx, mg32(ctx), top))) break;
      ++n;
      continue;
    }
    // one red-black sweep (two colour passes) per level
    for (int l = top; l >= 1; --l) {
      if ((st = fx_smooth(ctx, l, 1))) break;
      n += 2;
      bytes += 2.0 * (double)lvl_n(ctx, l) * CELLS * 12.0;
    }
    if (st) break;
  }
  const long long kernels = ctx->n_launch - n0;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
  ctx->stream = saved;
  ctx->n_launch -= kernels;
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return sm_cuda_check(ctx, e, "bench capture");
  cudaGraphExec_t x;
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return sm_cuda_check(ctx, e, "bench instantiate");
  cudaEvent_t a, b;
  SM_CK(cudaEventCreate(&a));
  SM_CK(cudaEventCreate(&b));
  SM_CK(cudaGraphLaunch(x, ctx->stream));  // warm
  SM_CK(cudaEventRecord(a, ctx->stream));
  SM_CK(cudaGraphLaunch(x, ctx->stream));
  SM_CK(cudaEventRecord(b, ctx->stream));
  SM_CK(cudaEventSynchronize(b));
  float ms = 0.f;
  SM_CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaGraphExecDestroy(x);
  ctx->n_launch += 2 * kernels;
  if (us_per_launch) *us_per_launch = 1e3 * ms / n;
  if (launches) *launches = n;
  if (whole) {
    double by, fl;
    vcycle_model(ctx, top, kclass == K_VCYCLE, &by, &fl);
    if (bytes_per_launch) *bytes_per_launch = by;
    if (flops_per_launch) *flops_per_launch = fl;
    return SM_OK;
  }
  if (bytes_per_launch) *bytes_per_launch = bytes / n;
  if (flops_per_launch) *flops_per_launch = 0.0;  // integer arithmetic only
  return SM_OK;
}
