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
#include <math.h>
#include <string.h>

#include "sm_internal.cuh"

using namespace sm;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// position of interior cell c (i + 8j + 64k) in a 10^3 staging array
__device__ __forceinline__ int s10(int c) { return ((c & 7) + 1) + 10 * (((c >> 3) & 7) + 1) + 100 * ((c >> 6) + 1); }

// Stage box b of variable v and its six face halos (ghost values by the
// rules of pot_ghost, evaluated from the staged interior) in s[1000].
// Blocks of NT threads (a multiple of 64); face f is filled by the 64-thread
// group f mod (NT/64), the face loop unrolled so that f is a constant.
template <int NT, typename T>
__device__ __forceinline__ void stage_box(T *s, const T *__restrict__ v, const int32_t *__restrict__ nbr6,
                                          const T *__restrict__ gh, int b, const Bc &bc, int homog) {
  const T *p = v + (size_t)b * CELLS;
#pragma unroll
  for (int c = threadIdx.x; c < CELLS; c += NT) s[s10(c)] = p[c];
  __syncthreads();
  const int grp = threadIdx.x >> 6, u = threadIdx.x & 7, w = (threadIdx.x >> 3) & 7;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (grp != f % (NT / 64)) continue;
    const int a = f >> 1;
    const int i = a == 0 ? ((f & 1) ? NC - 1 : 0) : (a == 1 ? w : u);
    const int j = a == 1 ? ((f & 1) ? NC - 1 : 0) : (a == 2 ? w : u);
    const int k = a == 2 ? ((f & 1) ? NC - 1 : 0) : (a == 0 ? w : u);
    const int q = s10(cidx(i, j, k));
    const int stride = a == 0 ? 1 : (a == 1 ? 10 : 100);
    s[q + ((f & 1) ? stride : -stride)] = pot_ghost(v, nbr6, gh, b, f, i, j, k, s[q], bc, homog);
  }
  __syncthreads();
}

// sum of the six neighbours from a staged box (order -x,+x,-y,+y,-z,+z)
template <typename T>
__device__ __forceinline__ T staged_sum(const T *s, int q) {
  return s[q - 1] + s[q + 1] + s[q - 10] + s[q + 10] + s[q - 100] + s[q + 100];
}

// One colour of a Gauss-Seidel red-black sweep over the boxes [lo, lo+grid)
// of one level: phi = (sum of 6 neighbours - h^2 f)/6 on cells with
// (i+j+k) % 2 == color (level-global parity; box origins are multiples of
// 8).  One block of 256 threads per box: the box and its face halos are
// staged in shared memory, then one thread per cell of the colour.
template <typename T>
__global__ void __launch_bounds__(256) k_rbgs(int lo, int color, T *__restrict__ phi, const T *__restrict__ rhs,
                                              const T *__restrict__ gh, const int32_t *__restrict__ nbr6, Bc bc,
                                              T h2, int homog) {
  __shared__ T s[1000];
  pdl_wait();
  int b = lo + blockIdx.x;
  stage_box<256>(s, phi, nbr6, gh, b, bc, homog);
  int t = threadIdx.x;
  int k = t >> 5, j = (t >> 2) & 7;
  int i = ((t & 3) << 1) | ((j + k + color) & 1);
  int c = cidx(i, j, k);
  size_t base = (size_t)b * CELLS;
  T sum = staged_sum(s, s10(c));
  phi[base + c] = (sum - h2 * rhs[base + c]) * T(1.0 / 6.0);
}

// plain 8-child average of one or two variables (FMG right-hand side,
// densities, potential after a mixed-precision correction)
template <typename T>
__global__ void __launch_bounds__(64) k_restrict1(int lo, const int32_t *__restrict__ parent,
                                                  const int32_t *__restrict__ ijk, T *__restrict__ a,
                                                  T *__restrict__ a2) {
  pdl_wait();
  int b = lo + blockIdx.x;
  int t = threadIdx.x;
  int ci = t & 3, cj = (t >> 2) & 3, ck = t >> 4;
  int P = parent[b];
  int o[3] = {ijk[3 * b] & 1, ijk[3 * b + 1] & 1, ijk[3 * b + 2] & 1};
  size_t fb = (size_t)b * CELLS;
  T s = 0, s2 = 0;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        int c = cidx(2 * ci + di, 2 * cj + dj, 2 * ck + dk);
        s += a[fb + c];
        if (a2) s2 += a2[fb + c];
      }
  size_t cc = (size_t)P * CELLS + cidx(4 * o[0] + ci, 4 * o[1] + cj, 4 * o[2] + ck);
  a[cc] = s * T(0.125);
  if (a2) a2[cc] = s2 * T(0.125);
}

// After restriction into level l-1 (boxes [lo, lo+grid)): keep a copy of
// phi, and on refined boxes complete the FAS right-hand side
// f = avg(r_fine) + L phi_restricted.
template <typename T>
__global__ void __launch_bounds__(512) k_fas(int lo, T *__restrict__ phi, T *__restrict__ old, T *__restrict__ rhs,
                                             const T *__restrict__ gh, const int32_t *__restrict__ nbr6,
                                             const int32_t *__restrict__ child, Bc bc, T inv_h2, int homog) {
  pdl_wait();
  int b = lo + blockIdx.x;
  int t = threadIdx.x;
  size_t base = (size_t)b * CELLS;
  T p = phi[base + t];
  old[base + t] = p;
  if (child[8 * b] < 0) return;
  int i = t & 7, j = (t >> 3) & 7, k = t >> 6;
  T s = nb_sum(phi, nbr6, gh, b, i, j, k, p, bc, homog);
  rhs[base + t] += (s - T(6) * p) * inv_h2;
}

// value of a coarse-level quantity at local cell q of box Q, where q may
// leave the box by one step along axis e (sign s): the neighbour box of the
// same level, or the physical-boundary ghost of the cell `ctr` it left.
template <typename T, typename F>
__device__ __forceinline__ T coarse_at(F val, const int32_t *__restrict__ nbr6, int Q, int q[3], int e, int s,
                                       T ctr, const Bc &bc, int homog, unsigned long long *err) {
  if (q[e] >= 0 && q[e] < NC) return val(Q, cidx(q[0], q[1], q[2]));
  int f = 2 * e + (s > 0);
  int Qn = __ldg(nbr6 + 6 * Q + f);
  if (Qn >= 0) {
    q[e] = s > 0 ? 0 : NC - 1;
    return val(Qn, cidx(q[0], q[1], q[2]));
  }
  if (Qn == -1) {
    if (bc.type[f]) return (homog ? T(0) : T(2.0 * bc.val[f])) - ctr;
    return ctr;
  }
  atomicOr(err, 1ull);  // nesting violated: no coarse box where one must be
  return ctr;
}

// phihat = c/2 + c_t1/4 + c_t2/4 for ghost cell (u,w) of refinement face f
// of box b (level l), from the level l-1 values of v
template <typename T>
__device__ __forceinline__ void cf_value(const T *__restrict__ v, T *__restrict__ gh,
                                         const int32_t *__restrict__ nbr6, const int32_t *__restrict__ parent,
                                         const int32_t *__restrict__ ijk, const Bc &bc, int homog, int b, int f,
                                         int u, int w, unsigned long long *err) {
  auto val = [&](int Q, int c) { return v[(size_t)Q * CELLS + c]; };
  int a = f >> 1, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  int G[3];
  G[a] = NC * ijk[3 * b + a] + ((f & 1) ? NC : -1);
  G[t1] = NC * ijk[3 * b + t1] + u;
  G[t2] = NC * ijk[3 * b + t2] + w;
  int P = parent[b];
  int Q = nbr6[6 * P + f];
  if (Q < 0) {
    atomicOr(err, 2ull);
    return;
  }
  int lc[3];
  for (int d = 0; d < 3; ++d) lc[d] = (G[d] >> 1) - NC * ijk[3 * Q + d];
  T c = val(Q, cidx(lc[0], lc[1], lc[2]));
  T ph = T(0.5) * c;
  int ts[2] = {t1, t2};
  for (int e2 = 0; e2 < 2; ++e2) {
    int e = ts[e2];
    int s = (G[e] & 1) ? 1 : -1;
    int q[3] = {lc[0], lc[1], lc[2]};
    q[e] += s;
    ph += T(0.25) * coarse_at<T>(val, nbr6, Q, q, e, s, c, bc, homog, err);
  }
  gh[(size_t)(6 * b + f) * FACE + u + NC * w] = ph;
}

// Coarse interpolation values for the refinement-boundary faces of the
// boxes [lo, lo+grid), 64 threads per box, one per face cell.
template <typename T>
__global__ void __launch_bounds__(64) k_fill_cf(int lo, const T *__restrict__ v, T *__restrict__ gh,
                                                const int32_t *__restrict__ nbr6,
                                                const int32_t *__restrict__ parent,
                                                const int32_t *__restrict__ ijk, Bc bc, int homog,
                                                unsigned long long *err) {
  pdl_wait();
  int b = lo + blockIdx.x;
  int u = threadIdx.x & 7, w = threadIdx.x >> 3;
  for (int f = 0; f < 6; ++f) {
    if (__ldg(nbr6 + 6 * b + f) != -2) continue;
    cf_value(v, gh, nbr6, parent, ijk, bc, homog, b, f, u, w, err);
  }
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

// Exact solve on level 0 (one 8^3 box), always in FP64: fold the Dirichlet
// boundary values into the right-hand side (not for the homogeneous error
// equation), transform to the separable eigenbasis, divide by the
// eigenvalues of the 7-point operator, transform back.
template <typename T>
__global__ void __launch_bounds__(512) k_coarse_solve(T *__restrict__ phi, const T *__restrict__ rhs,
                                                      const double *__restrict__ basis, Bc bc, double h2,
                                                      double inv_h2, int homog) {
  pdl_wait();
  __shared__ double x[CELLS], y[CELLS], V[3][64], lam[3][8];
  int t = threadIdx.x;
  if (t < 192) V[t / 64][t % 64] = basis[t];
  if (t < 24) lam[t / 8][t % 8] = basis[192 + t];
  int c[3] = {t & 7, (t >> 3) & 7, t >> 6};
  double r = (double)rhs[t];
  if (!homog)
    for (int f = 0; f < 6; ++f) {
      int q = c[f >> 1] + ((f & 1) ? 1 : -1);
      if ((q < 0 || q >= NC) && bc.type[f]) r -= 2.0 * bc.val[f] * inv_h2;
    }
  x[t] = r;
  __syncthreads();
  // forward: coefficients along x, then y, then z
  double acc = 0.0;
  for (int m = 0; m < NC; ++m) acc += V[0][m * 8 + c[0]] * x[cidx(m, c[1], c[2])];
  y[t] = acc;
  __syncthreads();
  acc = 0.0;
  for (int m = 0; m < NC; ++m) acc += V[1][m * 8 + c[1]] * y[cidx(c[0], m, c[2])];
  x[t] = acc;
  __syncthreads();
  acc = 0.0;
  for (int m = 0; m < NC; ++m) acc += V[2][m * 8 + c[2]] * x[cidx(c[0], c[1], m)];
  y[t] = acc * h2 / (lam[0][c[0]] + lam[1][c[1]] + lam[2][c[2]]);
  __syncthreads();
  // backward
  acc = 0.0;
  for (int m = 0; m < NC; ++m) acc += V[0][c[0] * 8 + m] * y[cidx(m, c[1], c[2])];
  x[t] = acc;
  __syncthreads();
  acc = 0.0;
  for (int m = 0; m < NC; ++m) acc += V[1][c[1] * 8 + m] * x[cidx(c[0], m, c[2])];
  y[t] = acc;
  __syncthreads();
  acc = 0.0;
  for (int m = 0; m < NC; ++m) acc += V[2][c[2] * 8 + m] * y[cidx(c[0], c[1], m)];
  phi[t] = (T)acc;
}

// max over leaf cells of |f - L v| into *slot (one block per leaf box)
__global__ void __launch_bounds__(512) k_resnorm(const int32_t *__restrict__ leaf,
                                                 const int32_t *__restrict__ level,
                                                 const double *__restrict__ v, const double *__restrict__ rhs,
                                                 const double *__restrict__ gh,
                                                 const int32_t *__restrict__ nbr6, Bc bc, LevelH lh,
                                                 unsigned long long *slot) {
  pdl_wait();
  __shared__ double red[16];
  int b = leaf[blockIdx.x];
  int t = threadIdx.x;
  int i = t & 7, j = (t >> 3) & 7, k = t >> 6;
  size_t base = (size_t)b * CELLS;
  double p = v[base + t];
  double s = nb_sum(v, nbr6, gh, b, i, j, k, p, bc, 0);
  double r = rhs[base + t] - (s - 6.0 * p) * lh.inv_h2[level[b]];
  block_max_to(slot, fabs(r), red);
}

// Outer FP64 residual of the mixed-precision solve on leaf cells: the max
// norm into *slot and the residual rounded to FP32 as the right-hand side
// of the error equation.
__global__ void __launch_bounds__(512) k_resid_to32(const int32_t *__restrict__ leaf,
                                                    const int32_t *__restrict__ level,
                                                    const double *__restrict__ v, const double *__restrict__ rhs,
                                                    const double *__restrict__ gh,
                                                    const int32_t *__restrict__ nbr6, Bc bc, LevelH lh,
                                                    float *__restrict__ f32, unsigned long long *slot) {
  pdl_wait();
  __shared__ double red[16];
  int b = leaf[blockIdx.x];
  int t = threadIdx.x;
  int i = t & 7, j = (t >> 3) & 7, k = t >> 6;
  size_t base = (size_t)b * CELLS;
  double p = v[base + t];
  double s = nb_sum(v, nbr6, gh, b, i, j, k, p, bc, 0);
  double r = rhs[base + t] - (s - 6.0 * p) * lh.inv_h2[level[b]];
  f32[base + t] = (float)r;
  block_max_to(slot, fabs(r), red);
}

// FP64 accumulation of the FP32 correction on leaf cells
__global__ void __launch_bounds__(512) k_add_corr(const int32_t *__restrict__ leaf, double *__restrict__ phi,
                                                  const float *__restrict__ e32) {
  pdl_wait();
  size_t x = (size_t)leaf[blockIdx.x] * CELLS + threadIdx.x;
  phi[x] += (double)e32[x];
}

// Residual and restriction fused: one block per fine box of level l
// computes r = f - L phi for its 512 cells (box staged with its face
// halos), then its 64 parent cells get the 8-child averages of phi (into
// phi) and of r (into rhs, completed to the FAS right-hand side by k_fas).
template <typename T>
__global__ void __launch_bounds__(512) k_resid_restrict(int lo, T *__restrict__ phi, T *__restrict__ rhs,
                                                        const T *__restrict__ gh,
                                                        const int32_t *__restrict__ nbr6,
                                                        const int32_t *__restrict__ parent,
                                                        const int32_t *__restrict__ ijk, Bc bc, T inv_h2,
                                                        int homog) {
  __shared__ T s[1000], sr[CELLS];
  pdl_wait();
  int b = lo + blockIdx.x;
  stage_box<512>(s, phi, nbr6, gh, b, bc, homog);
  int t = threadIdx.x;
  size_t base = (size_t)b * CELLS;
  int q = s10(t);
  T p = s[q];
  sr[t] = rhs[base + t] - (staged_sum(s, q) - T(6) * p) * inv_h2;
  __syncthreads();
  if (t >= 64) return;
  int ci = t & 3, cj = (t >> 2) & 3, ck = t >> 4;
  int P = parent[b];
  int o[3] = {ijk[3 * b] & 1, ijk[3 * b + 1] & 1, ijk[3 * b + 2] & 1};
  T ap = 0, ar = 0;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        int c = cidx(2 * ci + di, 2 * cj + dj, 2 * ck + dk);
        ap += s[s10(c)];
        ar += sr[c];
      }
  size_t cc = (size_t)P * CELLS + cidx(4 * o[0] + ci, 4 * o[1] + cj, 4 * o[2] + ck);
  phi[cc] = ap * T(0.125);
  rhs[cc] = ar * T(0.125);
}

// Prolongation into the boxes of level l fused with the coarse
// interpolation values of their refinement faces (both read only level
// l-1): mode 0 adds the correction (phi - old) with homogeneous wall
// ghosts, mode 1 overwrites with the prolonged solution (FMG); gh
// interpolates phi itself.  homog: the variable is an error (homogeneous
// wall ghosts everywhere).
template <typename T>
__global__ void __launch_bounds__(512) k_prolong_cf(int lo, int mode, T *__restrict__ phi,
                                                    const T *__restrict__ old, T *__restrict__ gh,
                                                    const int32_t *__restrict__ nbr6,
                                                    const int32_t *__restrict__ parent,
                                                    const int32_t *__restrict__ ijk, Bc bc, int homog,
                                                    unsigned long long *err) {
  pdl_wait();
  int b = lo + blockIdx.x;
  int t = threadIdx.x;
  int P = parent[b];
  {
    int loc[3] = {t & 7, (t >> 3) & 7, t >> 6};
    int G[3], lc[3];
    for (int d = 0; d < 3; ++d) {
      G[d] = NC * ijk[3 * b + d] + loc[d];
      lc[d] = (G[d] >> 1) - NC * ijk[3 * P + d];
    }
    auto val = [&](int Q, int c) {
      size_t x = (size_t)Q * CELLS + c;
      return mode ? phi[x] : phi[x] - old[x];
    };
    T c0 = val(P, cidx(lc[0], lc[1], lc[2]));
    T sum = c0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      int s = (G[e] & 1) ? 1 : -1;
      int q[3] = {lc[0], lc[1], lc[2]};
      q[e] += s;
      sum += coarse_at<T>(val, nbr6, P, q, e, s, c0, bc, (mode && !homog) ? 0 : 1, err);
    }
    size_t x = (size_t)b * CELLS + t;
    if (mode) phi[x] = T(0.25) * sum;
    else phi[x] += T(0.25) * sum;
  }
  if (t >= 6 * FACE) return;
  int f = t >> 6, u = t & 7, w = (t >> 3) & 7;
  if (__ldg(nbr6 + 6 * b + f) != -2) return;
  cf_value(phi, gh, nbr6, parent, ijk, bc, homog, b, f, u, w, err);
}

// Stopping test of the device-side cycle loop: relative residual of the
// last norm, cycle count (+inc), and the loop condition
// rel > tol && cycles < max.
__global__ void k_loop_check(cudaGraphConditionalHandle h, unsigned long long *sc, int inc) {
  pdl_wait();
  double num = __longlong_as_double((long long)sc[SC_NORM]);
  double den = __longlong_as_double((long long)sc[SC_DEN]);
  double rel = den > 0.0 ? num / den : num;
  unsigned long long c = sc[SC_CYC] + (unsigned long long)inc;
  sc[SC_CYC] = c;
  sc[SC_REL] = (unsigned long long)__double_as_longlong(rel);
  double tol = __longlong_as_double((long long)sc[SC_TOL]);
  cudaGraphSetConditional(h, (rel > tol && c < sc[SC_MAXC]) ? 1u : 0u);
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

static MG<double> mg64(sm_ctx *ctx) { return {ctx->phi, ctx->rhs, ctx->old, ctx->gh, 0}; }
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

int sm_fill_all_cf(sm_ctx *ctx, double *var) {
  for (int l = ctx->lbase + 1; l < ctx->n_levels; ++l) {
    int st = sm_mg_fill_cf(ctx, var, l, 0);
    if (st) return st;
  }
  return SM_OK;
}

template <typename T>
static int restrict_chain(sm_ctx *ctx, T *a, T *a2) {
  for (int l = ctx->n_levels - 1; l >= 1; --l) {
    int n = lvl_n(ctx, l);
    if (!n) continue;
    sm_launch(ctx, k_restrict1<T>, n, 64, 0, ctx->level_off[l], ctx->parent, ctx->ijk, a, a2);
  }
  SM_CKL("restrict");
  return SM_OK;
}

// a = avg8 of children (and a2 likewise), finest level first
int sm_restrict_pair(sm_ctx *ctx, double *a, double *a2) { return restrict_chain(ctx, a, a2); }

template <typename T>
static int rbgs_pass(sm_ctx *ctx, const MG<T> &m, int l, int color) {
  sm_launch(ctx, k_rbgs<T>, lvl_n(ctx, l), 256, 0, ctx->level_off[l], color, m.phi, m.rhs, m.gh, ctx->nbr6,
            ctx->bc, (T)ctx->lh.h2[l], m.homog);
  return SM_OK;
}

template <typename T>
static int smooth(sm_ctx *ctx, const MG<T> &m, int l, int nu) {
  if (!lvl_n(ctx, l)) return SM_OK;
  for (int s = 0; s < nu; ++s)
    for (int color = 0; color < 2; ++color) rbgs_pass(ctx, m, l, color);
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
  sm_launch(ctx, k_coarse_solve<T>, 1, 512, 0, m.phi, m.rhs, ctx->basis, ctx->bc, ctx->lh.h2[0],
            ctx->lh.inv_h2[0], m.homog);
  SM_CKL("coarse solve");
  return SM_OK;
}

template <typename T>
static int prolong_cf(sm_ctx *ctx, const MG<T> &m, int l, int mode) {
  sm_launch(ctx, k_prolong_cf<T>, lvl_n(ctx, l), 512, 0, ctx->level_off[l], mode, m.phi, m.old, m.gh,
            ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc, m.homog,
            ctx->dscal + SC_ERR);
  SM_CKL("prolong");
  return SM_OK;
}

// FAS V-cycle with `top` as finest level.  On entry the coarse
// interpolation values gh of every level <= top must match the current
// values of the level below (the solve prologue and every up-sweep leave
// them so); the down-sweep changes no level below the one it smooths
// before that level is visited again, so it needs no refill.
template <typename T>
static int vcycle(sm_ctx *ctx, const MG<T> &m, int top) {
  int st;
  for (int l = top; l >= 1; --l) {
    if ((st = smooth(ctx, m, l, ctx->cfg.nu1))) return st;
    sm_launch(ctx, k_resid_restrict<T>, lvl_n(ctx, l), 512, 0, ctx->level_off[l], m.phi, m.rhs, m.gh,
              ctx->nbr6, ctx->parent, ctx->ijk, ctx->bc,
              (T)ctx->lh.inv_h2[l], m.homog);
    sm_launch(ctx, k_fas<T>, lvl_n(ctx, l - 1), 512, 0, ctx->level_off[l - 1], m.phi, m.old, m.rhs, m.gh,
              ctx->nbr6, ctx->child, ctx->bc,
              (T)ctx->lh.inv_h2[l - 1], m.homog);
    SM_CKL("vcycle down");
  }
  if ((st = coarse_solve(ctx, m))) return st;
  for (int l = 1; l <= top; ++l) {
    if ((st = prolong_cf(ctx, m, l, 0))) return st;
    if ((st = smooth(ctx, m, l, ctx->cfg.nu2))) return st;
  }
  return SM_OK;
}

// FMG ladder: restrict f, exact level-0 solve, then for each finer level
// prolong the solution (and its interpolation values) and run one V-cycle
// with that level on top
template <typename T>
static int fmg_ladder(sm_ctx *ctx, const MG<T> &m) {
  int st;
  if ((st = restrict_chain<T>(ctx, m.rhs, nullptr))) return st;
  if ((st = coarse_solve(ctx, m))) return st;
  for (int l = 1; l < ctx->n_levels; ++l) {
    if ((st = prolong_cf(ctx, m, l, 1))) return st;
    if ((st = vcycle(ctx, m, l))) return st;
  }
  return SM_OK;
}

// max_leaf |f - L v| into slot (v's refinement ghosts must be current)
static int leaf_norm(sm_ctx *ctx, double *v, int slot) {
  SM_CK(cudaMemsetAsync(ctx->dscal + slot, 0, sizeof(unsigned long long), ctx->stream));
  sm_launch(ctx, k_resnorm, ctx->n_leaves, 512, 0, ctx->leaf, ctx->level, v, ctx->rhs, ctx->gh, ctx->nbr6,
            ctx->bc, ctx->lh, ctx->dscal + slot);
  SM_CKL("resnorm");
  return SM_OK;
}

// outer FP64 residual of the mixed form: norm into SC_NORM, f32 = (float) r
static int leaf_resid32(sm_ctx *ctx) {
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_NORM, 0, sizeof(unsigned long long), ctx->stream));
  sm_launch(ctx, k_resid_to32, ctx->n_leaves, 512, 0, ctx->leaf, ctx->level, ctx->phi, ctx->rhs, ctx->gh,
            ctx->nbr6, ctx->bc, ctx->lh, ctx->f32,
            ctx->dscal + SC_NORM);
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
  if (ladder) st = fmg_ladder(ctx, m);
  else st = vcycle(ctx, m, ctx->n_levels - 1);
  if (st) return st;
  sm_launch(ctx, k_add_corr, ctx->n_leaves, 512, 0, ctx->leaf, ctx->phi, ctx->e32);
  SM_CKL("add correction");
  if ((st = restrict_chain<double>(ctx, ctx->phi, nullptr))) return st;
  if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
  return leaf_resid32(ctx);
}

static int read_scalars(sm_ctx *ctx) {
  SM_CK(cudaMemcpyAsync(ctx->hscal, ctx->dscal, sizeof(double) * SC_N, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  unsigned long long e;
  memcpy(&e, &ctx->hscal[SC_ERR], sizeof e);
  if (e) return sm_fail(ctx, SM_ESTATE, "device consistency check failed (flags 0x%llx)", e);
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
      return solve_prologue(ctx);
    case 1:
      if ((st = solve_prologue(ctx))) return st;
      if ((st = fmg_ladder(ctx, mg64(ctx)))) return st;
      return leaf_norm(ctx, ctx->phi, SC_NORM);
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
  int st;
  if (kind >= 2) return mixed_correction(ctx, 0);
  if ((st = vcycle(ctx, mg64(ctx), ctx->n_levels - 1))) return st;
  return leaf_norm(ctx, ctx->phi, SC_NORM);
}

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
    sm_launch(ctx, k_loop_check, 1, 1, 0, h, ctx->dscal, 1);
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
  sm_launch(ctx, k_loop_check, 1, 1, 0, h, ctx->dscal, 1);
  out->body_launches = ctx->n_launch - n0;
  if (cudaStreamEndCapture(ctx->cap2, &body) != cudaSuccess)
    return end_captures(ctx, saved, sm_fail(ctx, SM_ECUDA, "end body capture"));
  ctx->stream = ctx->cap;
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

static int run_solve(sm_ctx *ctx, int fmg, double tol, int max_cycles, int *cycles, double *rel_res) {
  int st;
  int c = 0;
  double rel = 0.0;
  const int kind = (ctx->cfg.precision == SM_MIXED ? 2 : 0) + (fmg ? 1 : 0);
  if (ctx->graphs) {
    sm_graph *g = graph_of(ctx, kind);
    if (!g->exec && (st = capture_solve(ctx, kind, g))) return st;
    ctx->hscal[SC_TOL] = tol;
    unsigned long long mc = (unsigned long long)max_cycles;
    memcpy(&ctx->hscal[SC_MAXC], &mc, sizeof mc);
    SM_CK(cudaMemcpyAsync(ctx->dscal + SC_TOL, ctx->hscal + SC_TOL, 2 * sizeof(double), cudaMemcpyHostToDevice,
                          ctx->stream));
    SM_CK(cudaGraphLaunch(g->exec, ctx->stream));
    if ((st = read_scalars(ctx))) return st;
    unsigned long long cc;
    memcpy(&cc, &ctx->hscal[SC_CYC], sizeof cc);
    c = (int)cc;
    rel = ctx->hscal[SC_REL];
    ctx->n_launch += g->prefix_launches + g->body_launches * (long long)(fmg ? c - 1 : c);
  } else {
    if ((st = ensure_basis(ctx))) return st;
    if ((st = solve_prefix(ctx, kind))) return st;
    bool go = true;
    if (fmg) {
      c = 1;
      if ((st = read_scalars(ctx))) return st;
      double num = ctx->hscal[SC_NORM], den = ctx->hscal[SC_DEN];
      rel = den > 0.0 ? num / den : num;
      go = rel > tol && c < max_cycles;
    }
    while (go) {
      if ((st = solve_body(ctx, kind))) return st;
      ++c;
      if ((st = read_scalars(ctx))) return st;
      double num = ctx->hscal[SC_NORM], den = ctx->hscal[SC_DEN];
      rel = den > 0.0 ? num / den : num;
      go = rel > tol && c < max_cycles;
    }
  }
  if (cycles) *cycles = c;
  if (rel_res) *rel_res = rel;
  return rel <= tol ? SM_OK : sm_fail(ctx, SM_ENOCONV, "residual %.3e > tol %.3e after %d cycles", rel, tol, c);
}

// relative residual of the current potential (denominator recomputed);
// leaves the coarse interpolation values of phi current
int sm_rel_residual_now(sm_ctx *ctx, double *rel) {
  int st = solve_prologue(ctx);
  if (st) return st;
  return rel_residual(ctx, rel);
}

extern "C" int sm_fill_ghosts(sm_ctx *ctx, int var, int level) {
  int st = check_ready(ctx);
  if (st) return st;
  if (var != SM_PHI || level < 0 || level >= ctx->n_levels) return SM_EINVAL;
  return sm_mg_fill_cf(ctx, ctx->phi, level, 0);
}

extern "C" int sm_mg_vcycle(sm_ctx *ctx, int n_cycles, double *rel_res) {
  int st = check_ready(ctx);
  if (st) return st;
  if (n_cycles < 0) return SM_EINVAL;
  if ((st = ensure_basis(ctx))) return st;
  if ((st = solve_prologue(ctx))) return st;
  for (int c = 0; c < n_cycles; ++c)
    if ((st = vcycle(ctx, mg64(ctx), ctx->n_levels - 1))) return st;
  double rel = 0.0;
  if ((st = rel_residual(ctx, &rel))) return st;
  if (rel_res) *rel_res = rel;
  return SM_OK;
}

extern "C" int sm_mg_solve(sm_ctx *ctx, double tol, int max_cycles, int *cycles, double *rel_res) {
  int st = check_ready(ctx);
  if (st) return st;
  if (max_cycles < 1) return SM_EINVAL;
  return run_solve(ctx, 0, tol, max_cycles, cycles, rel_res);
}

extern "C" int sm_mg_fmg(sm_ctx *ctx, double tol, int max_cycles, int *cycles, double *rel_res) {
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

extern "C" int sm_set_pdl(sm_ctx *ctx, int enable) {
  if (!ctx) return SM_EINVAL;
  if (ctx->pdl != (enable != 0)) sm_drop_graphs(ctx);
  ctx->pdl = enable != 0;
  return SM_OK;
}

// Average launch duration of a kernel class in the launch mix of a V-cycle,
// timed with CUDA events around one graph of `reps` repetitions.
extern "C" int sm_kernel_bench(sm_ctx *ctx, int kclass, int reps, double *us_per_launch, long long *launches,
                               double *bytes_per_launch) {
  int st = check_ready(ctx);
  if (st) return st;
  if (kclass != K_SMOOTH || reps < 1) return SM_EINVAL;
  int top = ctx->n_levels - 1;
  if (top < 1) return SM_EINVAL;
  cudaStream_t saved = ctx->stream;
  if (!ctx->cap) SM_CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
  SM_CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
  ctx->stream = ctx->cap;
  long long n = 0;
  double bytes = 0.0;
  MG<double> m = mg64(ctx);
  for (int r = 0; r < reps; ++r)
    for (int l = top; l >= 1; --l)
      for (int color = 0; color < 2; ++color) {
        rbgs_pass(ctx, m, l, color);
        ++n;
        bytes += (double)lvl_n(ctx, l) * CELLS * 16.0;
      }
  cudaGraph_t g;
  cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
  ctx->stream = saved;
  ctx->n_launch -= n;
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
  ctx->n_launch += 2 * n;
  if (us_per_launch) *us_per_launch = 1e3 * ms / n;
  if (launches) *launches = n;
  if (bytes_per_launch) *bytes_per_launch = bytes / n;
  return SM_OK;
}
