// fluid.cu -- field and drift-diffusion-reaction step (Sec. 2.2-2.4):
// cell |E| from the potential, Eq. 5 right-hand side, Koren-limited upwind
// advective flux (Eq. 6-7) plus central diffusive flux with coefficients
// from a lookup table, refinement-boundary ghosts and flux averaging,
// forward-Euler stages combined into the explicit trapezoidal (Heun) step,
// and the time-step limits reduced by block/atomic maxima.
#include <math.h>
#include <string.h>

#include "sm_internal.cuh"
#include "sm_nvtx.h"

using namespace sm;

int sm_mg_solve_internal(sm_ctx *ctx, double tol, int max_cycles, int *cycles);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

// Non-negative doubles (no NaN) order as their bit patterns: clamps and
// minima of such values are integer operations, off the FP64 pipe (2 FP64
// instructions per clock and SM on this GPU).
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double dabs(double x) { return __longlong_as_double(dbits(x) & 0x7fffffffffffffffll); }

// floor(x) and x - floor(x) of a finite 0 < x < 2^30, exactly, from the bit
// fields: the integer part is the significand shifted by the exponent, the
// fraction the remaining significand bits renormalised (never subnormal:
// at least 2^-52)
__device__ __forceinline__ void split_frac(double x, int &i, double &w) {
  const unsigned long long b = (unsigned long long)dbits(x);
  const int e = (int)(b >> 52) - 1023;
  if (e < 0) {
    i = 0;
    w = x;
    return;
  }
  const unsigned long long m = (b & 0x000fffffffffffffull) | (1ull << 52);
  const int sh = 52 - e;
  i = (int)(m >> sh);
  const unsigned long long fm = m & ((1ull << sh) - 1ull);
  if (fm == 0ull) {
    w = 0.0;
    return;
  }
  const int top = 63 - __clzll((long long)fm);  // value fm 2^(e-52) = 1.f 2^(top + e - 52)
  w = __longlong_as_double((long long)(((unsigned long long)(top + e - 52 + 1023) << 52) |
                                       ((fm << (52 - top)) & 0x000fffffffffffffull)));
}

// Linear interpolation in two tables sampled at E_k = k e_max/(n-1) at
// x = e (n-1)/e_max (given), clamped at both ends (Sec. 2.3): the index and
// weight come from the bits of x; the interpolation a0 + w (a1 - a0) is one
// FP64 FMA each, with the slope a1 - a0 stored beside the table (sa, sb).
__device__ __forceinline__ void lookup2x(const double *__restrict__ ta, const double *__restrict__ sa,
                                         const double *__restrict__ tb, const double *__restrict__ sb, int n,
                                         long long xmax, double x, double &va, double &vb) {
  const long long bx = dbits(x);
  if (bx <= 0) {  // x <= 0 (or -0)
    va = __ldg(ta);
    vb = __ldg(tb);
    return;
  }
  if (bx >= xmax) {  // x >= n - 1
    va = __ldg(ta + n - 1);
    vb = __ldg(tb + n - 1);
    return;
  }
  int i;
  double w;
  split_frac(x, i, w);
  va = fma(w, __ldg(sa + i), __ldg(ta + i));
  vb = fma(w, __ldg(sb + i), __ldg(tb + i));
}

// psi(a/b) b for the Koren limiter psi(x) = max(0, min(1, (2+x)/6, x)),
// without the division: 0 when a b <= 0 (a or b is +-0, or their signs
// differ: tested on the bits, with no product), else
// sign(b) min(|b|, (2|b| + |a|)/6, |a|) with the minimum taken on the bit
// patterns
__device__ __forceinline__ double koren(double a, double b) {
  const long long ba = dbits(a), bb = dbits(b);
  if ((ba ^ bb) < 0 || (ba << 1) == 0 || (bb << 1) == 0) return 0.0;
  const double ab = dabs(b), aa = dabs(a);
  long long m = dbits(ab);
  m = min(m, dbits(fma(2.0, ab, aa) * (1.0 / 6.0)));
  m = min(m, dbits(aa));
  return __longlong_as_double(m | (dbits(b) & (long long)0x8000000000000000ull));
}

// dx times the flux through the face between cells L and R (positive
// toward R): v = -mu(E*) E_face with E_face = (p_L - p_R)/dx,
// E* = (|E|_L + |E|_R)/2 at table index x; advective part by Eq. 7 when
// v >= 0 and Eq. 6 when v < 0; diffusive part -D(E*) (n_R - n_L)/dx.
// Written as -mu dp n_f - D dn: v < 0 exactly when mu dp > 0.
__device__ __forceinline__ double face_flux_h(double nL2, double nL, double nR, double nR2, double pL, double pR,
                                              double x, const Table &tb) {
  double mu, dc;
  lookup2x(tb.mu, tb.dmu, tb.diff, tb.ddiff, tb.n, tb.xmax, x, mu, dc);
  const double t1 = mu * (pL - pR);
  const double dn = nR - nL;
  const bool up = dbits(t1) > 0;  // v < 0: the upwind cell is R
  // the operands are selected first, so each path costs one FP64 operation
  const double k = koren((up ? nR2 : nL) - (up ? nR : nL2), dn);
  const double nf = (up ? nR : nL) + __longlong_as_double(dbits(k) ^ (up ? (long long)0x8000000000000000ull : 0ll));
  return fma(-t1, nf, -dc * dn);
}

// 2 x, exactly, on the integer pipe, for 0 <= x < 2^1023 (not NaN):
// doubling adds one to the exponent field of a normal value and shifts the
// bits of a subnormal one (a carry into the exponent field is the result)
__device__ __forceinline__ double twice(double x) {
  const long long b = dbits(x);
  return __longlong_as_double((b >> 52) ? b + (1ll << 52) : b << 1);
}

// Density ghost (depth t = 1 or 2) across refinement face f of fine box b
// at face cell (u,w): linear prolongation (c + c_sx + c_sy + c_sz)/4 of the
// coarse cell c that contains the ghost, limited to 2c (Sec. 2.3).
__device__ double density_cf_ghost(const double *__restrict__ n, const int32_t *__restrict__ nbr6,
                                   const int32_t *__restrict__ parent, const int32_t *__restrict__ ijk, int b,
                                   int f, int t, int u, int w, unsigned long long *err) {
  int a = f >> 1, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  int G[3];
  G[a] = NC * ijk[3 * b + a] + ((f & 1) ? NC - 1 + t : -t);
  G[t1] = NC * ijk[3 * b + t1] + u;
  G[t2] = NC * ijk[3 * b + t2] + w;
  int P = parent[b];
  int Q = nbr6[6 * P + f];
  if (Q < 0) {
    atomicOr(err, 4ull);
    return 0.0;
  }
  int lc[3];
  for (int d = 0; d < 3; ++d) lc[d] = (G[d] >> 1) - NC * ijk[3 * Q + d];
  double c = n[(size_t)Q * CELLS + cidx(lc[0], lc[1], lc[2])];
  double sum = c;
  for (int d = 0; d < 3; ++d) {
    int s = (G[d] & 1) ? 1 : -1;
    int q[3] = {lc[0], lc[1], lc[2]};
    q[d] += s;
    double v;
    if (q[d] >= 0 && q[d] < NC) {
      v = n[(size_t)Q * CELLS + cidx(q[0], q[1], q[2])];
    } else {
      int Qn = nbr6[6 * Q + 2 * d + (s > 0)];
      if (Qn >= 0) {
        q[d] = s > 0 ? 0 : NC - 1;
        v = n[(size_t)Qn * CELLS + cidx(q[0], q[1], q[2])];
      } else {
        if (Qn == -2) atomicOr(err, 8ull);
        v = c;  // Neumann wall: mirror of c
      }
    }
    sum += v;
  }
  double g = 0.25 * sum;
  return g > 2.0 * c ? 2.0 * c : g;
}

// |E| ghost at a refinement face: the coarse cell containing the ghost
__device__ double emag_cf_ghost(const double *__restrict__ em, const int32_t *__restrict__ nbr6,
                                const int32_t *__restrict__ parent, const int32_t *__restrict__ ijk, int b, int f,
                                int u, int w) {
  int a = f >> 1, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  int G[3];
  G[a] = NC * ijk[3 * b + a] + ((f & 1) ? NC : -1);
  G[t1] = NC * ijk[3 * b + t1] + u;
  G[t2] = NC * ijk[3 * b + t2] + w;
  int Q = nbr6[6 * parent[b] + f];
  if (Q < 0) return 0.0;
  int lc[3];
  for (int d = 0; d < 3; ++d) lc[d] = (G[d] >> 1) - NC * ijk[3 * Q + d];
  return em[(size_t)Q * CELLS + cidx(lc[0], lc[1], lc[2])];
}

// local cell (i,j,k) of face f at depth dep (0 = next to the face)
__device__ __forceinline__ void face_loc(int f, int dep, int u, int w, int c[3]) {
  int a = f >> 1;
  c[a] = (f & 1) ? NC - 1 - dep : dep;
  c[(a + 1) % 3] = u;
  c[(a + 2) % 3] = w;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// |E| on leaf cells: cell component = mean of the two face fields
// (phi_{i-1} - phi_i)/dx and (phi_i - phi_{i+1})/dx
__global__ void __launch_bounds__(512) k_field(const int32_t *__restrict__ leaf, const int32_t *__restrict__ level,
                                               const double *__restrict__ phi, const double *__restrict__ gh,
                                               const int32_t *__restrict__ nbr6, Bc bc, LevelH lh,
                                               double *__restrict__ emag) {
  int b = leaf[blockIdx.x];
  int t = threadIdx.x;
  int c[3] = {t & 7, (t >> 3) & 7, t >> 6};
  double ih = lh.inv_h[level[b]];
  const double *p = phi + (size_t)b * CELLS;
  double pc = p[t];
  const int stride[3] = {1, NC, FACE};
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double pm = c[a] > 0 ? p[t - stride[a]] : pot_ghost(phi, nbr6, gh, b, 2 * a, c[0], c[1], c[2], pc, bc, 0);
    double pp = c[a] < NC - 1 ? p[t + stride[a]]
                              : pot_ghost(phi, nbr6, gh, b, 2 * a + 1, c[0], c[1], c[2], pc, bc, 0);
    d[a] = pm - pp;
  }
  // |E| = |(p_-d - p_+d)| / (2 dx) summed in quadrature: each component is
  // the mean of (p_-d - p_c)/dx and (p_c - p_+d)/dx
  emag[(size_t)b * CELLS + t] = sqrt(fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]))) * (0.5 * ih);
}

// Eq. 5 right-hand side on leaf cells
__global__ void __launch_bounds__(512) k_charge(const int32_t *__restrict__ leaf, const double *__restrict__ ne,
                                                const double *__restrict__ ni, const double *__restrict__ rho,
                                                double q, double inv_eps, int use_rho, double *__restrict__ rhs) {
  size_t x = (size_t)leaf[blockIdx.x] * CELLS + threadIdx.x;
  rhs[x] = use_rho ? -rho[x] * inv_eps : -q * (ni[x] - ne[x]) * inv_eps;
}

// per-cell time-step quantities at table index x of the cell's |E|:
// sum_d mu |E_d|/dx with E_d = (p_{-d} - p_{+d})/(2 dx) (the mean of the two
// face fields), that plus 6 D/dx^2, and mu n_e
__device__ __forceinline__ void dt_terms(const double *__restrict__ phi, const double *__restrict__ gh,
                                         const int32_t *__restrict__ nbr6, const Bc &bc, int b, int t, double ih2,
                                         double x, double ne, const Table &tb, double &adv, double &ad,
                                         double &drt) {
  int c[3] = {t & 7, (t >> 3) & 7, t >> 6};
  const double *p = phi + (size_t)b * CELLS;
  double pc = p[t];
  const int stride[3] = {1, NC, FACE};
  double mu, dc;
  lookup2x(tb.mu, tb.dmu, tb.diff, tb.ddiff, tb.n, tb.xmax, x, mu, dc);
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double pm = c[a] > 0 ? p[t - stride[a]] : pot_ghost(phi, nbr6, gh, b, 2 * a, c[0], c[1], c[2], pc, bc, 0);
    double pp = c[a] < NC - 1 ? p[t + stride[a]]
                              : pot_ghost(phi, nbr6, gh, b, 2 * a + 1, c[0], c[1], c[2], pc, bc, 0);
    d[a] = dabs(pm - pp);
  }
  adv = (mu * ((d[0] + d[1]) + d[2])) * (0.5 * ih2);
  ad = fma(6.0 * ih2, dc, adv);
  drt = mu * ne;
}

// block maxima of three non-negative quantities (negative values count as
// 0) into slots[0..2], compared as bit patterns on the integer pipe; red:
// 3 * (blockDim.x / 32) words of shared memory
__device__ __forceinline__ void block_max3_to(unsigned long long *slots, double a, double b, double c,
                                              long long *red) {
  long long v[3] = {max(dbits(a), 0ll), max(dbits(b), 0ll), max(dbits(c), 0ll)};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = max(v[i], __shfl_xor_sync(0xffffffffu, v[i], o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 3; ++i) red[3 * wid + i] = v[i];
  __syncthreads();
  if (threadIdx.x < 3) {
    long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[3 * w + threadIdx.x]);
    atomicMax(slots + threadIdx.x, (unsigned long long)m);
  }
}

__global__ void __launch_bounds__(512) k_dt(const int32_t *__restrict__ leaf, const int32_t *__restrict__ level,
                                            const double *__restrict__ phi, const double *__restrict__ gh,
                                            const double *__restrict__ emag, const double *__restrict__ ne,
                                            const int32_t *__restrict__ nbr6, Bc bc, LevelH lh, Table tb,
                                            unsigned long long *slots) {
  __shared__ long long red[48];
  int b = leaf[blockIdx.x];
  int t = threadIdx.x;
  size_t x = (size_t)b * CELLS + t;
  double adv, ad, drt;
  dt_terms(phi, gh, nbr6, bc, b, t, lh.inv_h2[level[b]], emag[x] * tb.inv_de, ne[x], tb, adv, ad, drt);
  block_max3_to(slots + SC_ADV, adv, ad, drt, red);
}

// Fine-side fluxes through the refinement faces of leaf boxes (64 threads
// per box, one per face cell, over the list of leaves that have such a
// face); read by the box itself and averaged by its coarse neighbour, so
// both sides use the same numbers.
__global__ void __launch_bounds__(64) k_cf_flux(const int32_t *__restrict__ leaf, const int32_t *__restrict__ level,
                                                const double *__restrict__ n, const double *__restrict__ phi,
                                                const double *__restrict__ gh, const double *__restrict__ emag,
                                                const int32_t *__restrict__ nbr6,
                                                const int32_t *__restrict__ parent,
                                                const int32_t *__restrict__ ijk, LevelH lh, Table tb,
                                                double *__restrict__ cflux, unsigned long long *err) {
  int b = leaf[blockIdx.x];
  int u = threadIdx.x & 7, w = threadIdx.x >> 3;
  double ih = lh.inv_h[level[b]];
  size_t base = (size_t)b * CELLS;
  for (int f = 0; f < 6; ++f) {
    if (__ldg(nbr6 + 6 * b + f) != -2) continue;
    int c0[3], c1[3];
    face_loc(f, 0, u, w, c0);
    face_loc(f, 1, u, w, c1);
    int a = f >> 1;
    double n0 = n[base + cidx(c0[0], c0[1], c0[2])], n1 = n[base + cidx(c1[0], c1[1], c1[2])];
    double g1 = density_cf_ghost(n, nbr6, parent, ijk, b, f, 1, u, w, err);
    double g2 = density_cf_ghost(n, nbr6, parent, ijk, b, f, 2, u, w, err);
    double p0 = phi[base + cidx(c0[0], c0[1], c0[2])];
    double pg = p0 * (1.0 / 3.0) + (2.0 / 3.0) * gh[(size_t)(6 * b + f) * FACE + fcell(a, c0[0], c0[1], c0[2])];
    double e0 = emag[base + cidx(c0[0], c0[1], c0[2])];
    double eg = emag_cf_ghost(emag, nbr6, parent, ijk, b, f, u, w);
    const double x = (e0 + eg) * tb.hinv_de;
    double F;
    if (f & 1) F = face_flux_h(n1, n0, g1, g2, p0, pg, x, tb);
    else F = face_flux_h(g2, g1, n0, n1, pg, p0, x, tb);
    cflux[(size_t)(6 * b + f) * FACE + u + NC * w] = F * ih;
  }
}

// Smem layout of one box for the update kernel
struct UpdSmem {
  double n[12 * 12 * 12];   // density with 2 ghost layers on faces
  double p[10 * 10 * 10];   // potential with 1 ghost layer
  double x[10 * 10 * 10];   // half table index |E| (n-1)/(2 e_max), 1 ghost layer
  double F[3 * 9 * 64];     // face fluxes times dx [a][m][w][u]
  long long red[48];
};
__device__ __forceinline__ int I12(int i, int j, int k) { return (i + 2) + 12 * ((j + 2) + 12 * (k + 2)); }
__device__ __forceinline__ int I10(int i, int j, int k) { return (i + 1) + 10 * ((j + 1) + 10 * (k + 1)); }

// index in a staged box of pitch P (O ghost layers) of the cell with
// coordinate ca along axis a and u, w along axes (a+1)%3, (a+2)%3 (no
// arrays indexed at run time: those would live in local memory)
template <int P, int O>
__device__ __forceinline__ int lin_axis(int a, int ca, int u, int w) {
  const int x = a == 0 ? ca : (a == 1 ? w : u);
  const int y = a == 0 ? u : (a == 1 ? ca : w);
  const int z = a == 0 ? w : (a == 1 ? u : ca);
  return (x + O) + P * ((y + O) + P * (z + O));
}

// One forward-Euler stage on a leaf box: dst = src + dt F(src), with
// F = -div(flux) + alpha mu |E| n_e for electrons and the same source for
// ions.  heun != 0: dst = (n0 + src + dt F(src))/2.  Also writes the Eq. 5
// right-hand side from dst, and with want_dt the time-step maxima of src.
__global__ void __launch_bounds__(512, 3) k_update(
    const int32_t *__restrict__ leaf, const int32_t *__restrict__ level, const double *__restrict__ ne_src,
    const double *__restrict__ ni_src, const double *__restrict__ ne0, const double *__restrict__ ni0,
    double *__restrict__ ne_dst, double *__restrict__ ni_dst, const double *__restrict__ phi,
    const double *__restrict__ gh, const double *__restrict__ emag, const double *__restrict__ cflux,
    const int32_t *__restrict__ nbr6, const int32_t *__restrict__ child, const int32_t *__restrict__ parent,
    const int32_t *__restrict__ ijk, Bc bc, LevelH lh, Table tb, double dt, int heun, double q, double inv_eps,
    double *__restrict__ rhs, int want_dt, unsigned long long *slots) {
  extern __shared__ double smraw[];
  UpdSmem &S = *reinterpret_cast<UpdSmem *>(smraw);
  int b = leaf[blockIdx.x];
  int t = threadIdx.x;
  int l = level[b];
  const double h = lh.h[l], ih2 = lh.inv_h2[l];
  size_t base = (size_t)b * CELLS;
  int ci = t & 7, cj = (t >> 3) & 7, ck = t >> 6;
  const double e = emag[base + t];
  const double xh = e * tb.hinv_de;  // the cell's table index is 2 xh, exactly e (n-1)/e_max
  S.n[I12(ci, cj, ck)] = ne_src[base + t];
  S.p[I10(ci, cj, ck)] = phi[base + t];
  S.x[I10(ci, cj, ck)] = xh;
  __syncthreads();
  // face halos: thread -> (face, face cell)
  if (t < 6 * FACE) {
    const int f = t >> 6, fc = t & 63;
    const int u = fc & 7, w = fc >> 3, a = f >> 1, hi = f & 1;
    const int nb = nbr6[6 * b + f];
    // depths 0, 1 inside the face and the ghosts -1, -2 along axis a
    const int d0 = hi ? NC - 1 : 0, d1 = hi ? NC - 2 : 1, dg1 = hi ? NC : -1, dg2 = hi ? NC + 1 : -2;
    const int r0 = lin_axis<10, 1>(a, d0, u, w);
    double n0 = S.n[lin_axis<12, 2>(a, d0, u, w)], n1 = S.n[lin_axis<12, 2>(a, d1, u, w)];
    double p0 = S.p[r0], x0 = S.x[r0];
    double vg1, vg2, pg, xg;
    if (nb >= 0) {
      // the neighbour's cells at depths 0 and 1 of its opposite face
      const int m0 = lin_axis<8, 0>(a, hi ? 0 : NC - 1, u, w), m1 = lin_axis<8, 0>(a, hi ? 1 : NC - 2, u, w);
      size_t nbase = (size_t)nb * CELLS;
      vg1 = ne_src[nbase + m0];
      vg2 = ne_src[nbase + m1];
      pg = phi[nbase + m0];
      xg = child[8 * nb] < 0 ? emag[nbase + m0] * tb.hinv_de : 0.0;
    } else if (nb == -1) {
      vg1 = n0;
      vg2 = n1;
      pg = bc.type[f] ? 2.0 * bc.val[f] - p0 : p0;
      xg = x0;
    } else {
      vg1 = density_cf_ghost(ne_src, nbr6, parent, ijk, b, f, 1, u, w, slots + SC_ERR);
      vg2 = density_cf_ghost(ne_src, nbr6, parent, ijk, b, f, 2, u, w, slots + SC_ERR);
      pg = p0 * (1.0 / 3.0) + (2.0 / 3.0) * gh[(size_t)(6 * b + f) * FACE + u + NC * w];
      xg = emag_cf_ghost(emag, nbr6, parent, ijk, b, f, u, w) * tb.hinv_de;
    }
    S.n[lin_axis<12, 2>(a, dg1, u, w)] = vg1;
    S.n[lin_axis<12, 2>(a, dg2, u, w)] = vg2;
    const int rg = lin_axis<10, 1>(a, dg1, u, w);
    S.p[rg] = pg;
    S.x[rg] = xg;
  }
  __syncthreads();
  // fluxes: 3 axes x 9 faces x 64
  for (int x = t; x < 3 * 9 * FACE; x += blockDim.x) {
    int a = x / (9 * FACE), rem = x % (9 * FACE);
    int m = rem >> 6, u = rem & 7, w = (rem >> 3) & 7;
    double F;
    bool done = false;
    if (m == 0 || m == NC) {
      int f = 2 * a + (m == NC);
      int nb = nbr6[6 * b + f];
      if (nb == -2) {
        F = cflux[(size_t)(6 * b + f) * FACE + u + NC * w] * h;
        done = true;
      } else if (nb >= 0 && child[8 * nb] >= 0) {
        // coarse side of a refinement face: mean of the 4 fine fluxes
        int ch = child[8 * nb + lin_axis<2, 0>(a, (f & 1) ? 0 : 1, u >> 2, w >> 2)];
        const double *cf = cflux + (size_t)(6 * ch + (f ^ 1)) * FACE;
        int uf = 2 * (u & 3), wf = 2 * (w & 3);
        double s = 0.0;
        s += cf[uf + NC * wf];
        s += cf[uf + 1 + NC * wf];
        s += cf[uf + NC * (wf + 1)];
        s += cf[uf + 1 + NC * (wf + 1)];
        F = (s * 0.25) * h;
        done = true;
      }
    }
    if (!done) {
      // cells m-2 .. m+1 along axis a
      const int q = lin_axis<12, 2>(a, m - 2, u, w), sq = a == 0 ? 1 : (a == 1 ? 12 : 144);
      const int r = lin_axis<10, 1>(a, m - 1, u, w), sr = a == 0 ? 1 : (a == 1 ? 10 : 100);
      F = face_flux_h(S.n[q], S.n[q + sq], S.n[q + 2 * sq], S.n[q + 3 * sq], S.p[r], S.p[r + sr],
                      S.x[r] + S.x[r + sr], tb);
    }
    S.F[(a * 9 + m) * FACE + u + NC * w] = F;
  }
  __syncthreads();
  // update: div = sum over axes of the flux differences (times dx) / dx^2
  const double *Fx = S.F + (0 * 9 + ci) * FACE + cj + NC * ck;
  const double *Fy = S.F + (1 * 9 + cj) * FACE + ck + NC * ci;
  const double *Fz = S.F + (2 * 9 + ck) * FACE + ci + NC * cj;
  const double div = ((Fx[FACE] - Fx[0]) + (Fy[FACE] - Fy[0]) + (Fz[FACE] - Fz[0])) * ih2;
  double nes = S.n[I12(ci, cj, ck)];
  const double x = twice(xh);  // e (n-1)/e_max
  double alpha, mu;
  lookup2x(tb.alpha, tb.dalpha, tb.mu, tb.dmu, tb.n, tb.xmax, x, alpha, mu);
  double src = alpha * mu * e * nes;
  double ne_new = fma(dt, src - div, nes);
  double ni_new = fma(dt, src, ni_src[base + t]);
  if (heun) {
    ne_new = 0.5 * (ne0[base + t] + ne_new);
    ni_new = 0.5 * (ni0[base + t] + ni_new);
  }
  ne_dst[base + t] = ne_new;
  ni_dst[base + t] = ni_new;
  rhs[base + t] = (ni_new - ne_new) * (-q * inv_eps);
  if (want_dt) {
    double adv, ad, drt;
    dt_terms(phi, gh, nbr6, bc, b, t, ih2, x, nes, tb, adv, ad, drt);
    block_max3_to(slots + SC_ADV, adv, ad, drt, S.red);
  }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
static Table table_of(const sm_ctx *ctx) {
  Table tb;
  tb.mu = ctx->tab;
  tb.diff = ctx->tab + 4096;
  tb.alpha = ctx->tab + 8192;
  tb.dmu = ctx->tab + 3 * 4096;
  tb.ddiff = ctx->tab + 4 * 4096;
  tb.dalpha = ctx->tab + 5 * 4096;
  tb.n = ctx->tab_n;
  tb.inv_de = (ctx->tab_n - 1) / ctx->tab_emax;
  tb.hinv_de = 0.5 * tb.inv_de;
  const double top = (double)(ctx->tab_n - 1);
  memcpy(&tb.xmax, &top, sizeof top);
  return tb;
}

static int ready(sm_ctx *ctx) {
  if (!ctx) return SM_EINVAL;
  if (!ctx->arena || ctx->n_levels == 0) return sm_fail(ctx, SM_ESTATE, "octree not built");
  return SM_OK;
}

extern "C" int sm_compute_field(sm_ctx *ctx) {
  SM_RANGE();
  int st = ready(ctx);
  if (st) return st;
  if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
  k_field<<<ctx->n_leaves, 512, 0, ctx->stream>>>(ctx->leaf, ctx->level, ctx->phi, ctx->gh, ctx->nbr6, ctx->bc,
                                                  ctx->lh, ctx->emag);
  ++ctx->n_launch;
  SM_CKL("field");
  return SM_OK;
}

extern "C" int sm_charge_rhs(sm_ctx *ctx, double q, double eps, int use_rho) {
  int st = ready(ctx);
  if (st) return st;
  if (!(eps != 0.0)) return SM_EINVAL;
  k_charge<<<ctx->n_leaves, 512, 0, ctx->stream>>>(ctx->leaf, ctx->nbuf[ctx->ncur], ctx->ibuf[ctx->ncur], ctx->rho,
                                                   q, 1.0 / eps, use_rho, ctx->rhs);
  ++ctx->n_launch;
  SM_CKL("charge");
  return SM_OK;
}

extern "C" int sm_restrict_densities(sm_ctx *ctx) {
  int st = ready(ctx);
  if (st) return st;
  return sm_restrict_pair(ctx, ctx->nbuf[ctx->ncur], ctx->ibuf[ctx->ncur]);
}

// dt from time-step maxima already copied to host scalars hs (SC_N words)
static int dt_of(sm_ctx *ctx, const double *hs, double q, double eps, double *dt) {
  unsigned long long e;
  memcpy(&e, &hs[SC_ERR], sizeof e);
  if (e) return sm_fail(ctx, SM_ESTATE, "device consistency check failed (flags 0x%llx)", e);
  double m_adv = hs[SC_ADV], m_ad = hs[SC_AD], m_drt = hs[SC_DRT];
  double d = 1e300;
  if (m_adv > 0.0 && 0.5 / m_adv < d) d = 0.5 / m_adv;
  if (m_ad > 0.0 && 1.0 / m_ad < d) d = 1.0 / m_ad;
  if (m_drt > 0.0 && eps / (q * m_drt) < d) d = eps / (q * m_drt);
  *dt = 0.9 * d;
  return SM_OK;
}

static int dt_from_slots(sm_ctx *ctx, double q, double eps, double *dt) {
  SM_CK(cudaMemcpyAsync(ctx->hscal, ctx->dscal, sizeof(double) * SC_N, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  return dt_of(ctx, ctx->hscal, q, eps, dt);
}

extern "C" int sm_dt_limit(sm_ctx *ctx, double q, double eps, double *dt) {
  SM_RANGE();
  int st = ready(ctx);
  if (st) return st;
  if (!dt || ctx->tab_n < 2) return sm_fail(ctx, SM_ESTATE, "no coefficient table");
  if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_ADV, 0, 3 * sizeof(unsigned long long), ctx->stream));
  k_dt<<<ctx->n_leaves, 512, 0, ctx->stream>>>(ctx->leaf, ctx->level, ctx->phi, ctx->gh, ctx->emag,
                                               ctx->nbuf[ctx->ncur], ctx->nbr6, ctx->bc, ctx->lh, table_of(ctx),
                                               ctx->dscal);
  ++ctx->n_launch;
  SM_CKL("dt");
  return dt_from_slots(ctx, q, eps, dt);
}

// one stage from buffer s into buffer d (heun: averaged with buffer h0)
static int stage(sm_ctx *ctx, int s, int d, int h0, double dt, double q, double eps, int want_dt) {
  int st;
  Table tb = table_of(ctx);
  if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
  if (ctx->n_cf_leaves > 0) {
    k_cf_flux<<<ctx->n_cf_leaves, 64, 0, ctx->stream>>>(ctx->cf_leaf, ctx->level, ctx->nbuf[s], ctx->phi,
                                                         ctx->gh, ctx->emag, ctx->nbr6, ctx->parent, ctx->ijk,
                                                         ctx->lh, tb, ctx->cflux, ctx->dscal + SC_ERR);
    ++ctx->n_launch;
    SM_CKL("cf_flux");
  }
  size_t smem = sizeof(UpdSmem);
  k_update<<<ctx->n_leaves, 512, smem, ctx->stream>>>(
      ctx->leaf, ctx->level, ctx->nbuf[s], ctx->ibuf[s], h0 >= 0 ? ctx->nbuf[h0] : nullptr,
      h0 >= 0 ? ctx->ibuf[h0] : nullptr, ctx->nbuf[d], ctx->ibuf[d], ctx->phi, ctx->gh, ctx->emag, ctx->cflux,
      ctx->nbr6, ctx->child, ctx->parent, ctx->ijk, ctx->bc, ctx->lh, tb, dt, h0 >= 0, q, 1.0 / eps, ctx->rhs,
      want_dt, ctx->dscal);
  ++ctx->n_launch;
  SM_CKL("update");
  return sm_restrict_pair(ctx, ctx->nbuf[d], ctx->ibuf[d]);
}

extern "C" int sm_fluid_stage(sm_ctx *ctx, double dt) {
  SM_RANGE();
  int st = ready(ctx);
  if (st) return st;
  if (ctx->tab_n < 2) return sm_fail(ctx, SM_ESTATE, "no coefficient table");
  int a = ctx->ncur, b = (a + 1) % 3;
  if ((st = sm_restrict_pair(ctx, ctx->nbuf[a], ctx->ibuf[a]))) return st;
  // q/eps only feed the right-hand side written alongside; a stage alone
  // uses SI values
  if ((st = stage(ctx, a, b, -1, dt, 1.602176634e-19, 8.8541878128e-12, 0))) return st;
  ctx->ncur = b;
  return SM_OK;
}

extern "C" int sm_advance_fluid_coeffs(sm_ctx *ctx, double dt, const sm_fluid_coeffs *c, double *dt_next,
                                       int *cycles) {
  if (!c) return SM_EINVAL;
  return sm_advance_fluid(ctx, dt, c->q, c->eps, c->tol, c->max_cycles, dt_next, cycles);
}

extern "C" int sm_advance_fluid(sm_ctx *ctx, double dt, double q, double eps, double tol, int max_cycles,
                                double *dt_next, int *cycles) {
  SM_RANGE();
  int st = ready(ctx);
  if (st) return st;
  if (ctx->tab_n < 2) return sm_fail(ctx, SM_ESTATE, "no coefficient table");
  if (!(eps != 0.0) || max_cycles < 1) return SM_EINVAL;
  int A = ctx->ncur, B = (A + 1) % 3, C = (A + 2) % 3;
  if ((st = sm_restrict_pair(ctx, ctx->nbuf[A], ctx->ibuf[A]))) return st;
  // stage 1: n1 = n0 + dt F(n0); new field
  if ((st = stage(ctx, A, B, -1, dt, q, eps, 0))) return st;
  int c1 = 0, c2 = 0, st1, st2;
  if (ctx->pre_solve && (st = ctx->pre_solve(ctx->hook_obj, ctx))) return st;
  st1 = sm_mg_solve(ctx, tol, max_cycles, &c1, nullptr);
  if (st1 && st1 != SM_ENOCONV) return st1;
  if (ctx->post_solve && (st = ctx->post_solve(ctx->hook_obj, ctx))) return st;
  if ((st = sm_compute_field(ctx))) return st;
  // stage 2: n = (n0 + n1 + dt F(n1))/2 with the time-step limits at n1
  SM_CK(cudaMemsetAsync(ctx->dscal + SC_ADV, 0, 3 * sizeof(unsigned long long), ctx->stream));
  if ((st = stage(ctx, B, C, A, dt, q, eps, 1))) return st;
  ctx->ncur = C;
  // the maxima go to the staged host copy without a wait: the solve below
  // synchronises before they are read
  double *staged = ctx->hscal + SC_N;
  SM_CK(cudaMemcpyAsync(staged, ctx->dscal, sizeof(double) * SC_N, cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->pre_solve && (st = ctx->pre_solve(ctx->hook_obj, ctx))) return st;
  st2 = sm_mg_solve(ctx, tol, max_cycles, &c2, nullptr);
  if (st2 && st2 != SM_ENOCONV) return st2;
  if (ctx->post_solve && (st = ctx->post_solve(ctx->hook_obj, ctx))) return st;
  if ((st = sm_compute_field(ctx))) return st;
  SM_CK(cudaStreamSynchronize(ctx->stream));
  double dtn = 0.0;
  if ((st = dt_of(ctx, staged, q, eps, &dtn))) return st;
  if (dt_next) *dt_next = dtn;
  if (cycles) {
    cycles[0] = c1;
    cycles[1] = c2;
  }
  if (st1 || st2) return sm_fail(ctx, SM_ENOCONV, "a Poisson solve did not reach tol %.3e", tol);
  return SM_OK;
}
