// mgfix.cuh -- the FP64 solve's multigrid cycle in exact 64-bit fixed point
// (Sec. 2.1.2: FAS V-cycle, red-black Gauss-Seidel, restriction,
// prolongation and coarse-to-fine ghosts; included by multigrid.cu after
// its per-box helpers).
//
// During an FP64 solve the potential of every box is held as an integer
// multiple of one quantum q = 2^(E - 1080).  E is chosen per solve from the
// largest exponent field among the potential, the Dirichlet ghost
// constants 2g and every h_l^2 f, plus a margin of FX_MARGIN: every input
// is then below 2^53 quanta and stored values must stay below 2^55
// (FX_LIM), which keeps every intermediate sum inside 63 bits.  Sums of
// neighbours are exact; each operation of the cycle rounds once, to the
// nearest quantum with ties away from zero:
//   smoother        phi = (sum of 6 neighbours + 6 G) / 6,
//                   G = -h^2 f / 6 in quanta (rounded once per rhs),
//   restriction     phi_c = (sum of 8 children) / 8,
//   FAS rhs         G_c = (sum over children of (6 G + T) - 2 T_c) / 12,
//                   T = h^2 L phi in quanta = sum of 6 neighbours - 6 phi,
//   prolongation    (c + c_x + c_y + c_z) / 4,
//   coarse-fine     ghost = (2 inner + Ghat) / 6, Ghat = 2c + c_t1 + c_t2.
// The level-0 solve and the residual norm stay in FP64.  A value that
// would leave the range sets error bit FX_ERR_OVF; the solve is then run
// again from its unchanged FP64 inputs with a margin larger by 8.
//
// The fixed-point arrays of a box are stored colour by colour: the 256
// red cells ((i+j+k) even, level-global) first, then the 256 black ones,
// each half ordered (i/2) + 4j + 32k.  A colour pass of the red-black
// smoother then reads only the other colour, the G of its own colour and
// (at walls and refinement faces) its own face cells, and writes its own
// colour in place: 12 bytes per cell and pass, with every load and store
// of the box coalesced.
#pragma once

namespace fx {

constexpr long long FX_LIM = 1ll << 55;     // |stored value| < FX_LIM quanta
constexpr int FX_MARGIN = 5;                // E = exponent bound + margin
constexpr int FX_EMIN = 64;                 // keeps q and q/h^2 normal
constexpr unsigned long long FX_ERR_OVF = 8ull;

__device__ __forceinline__ bool fx_bad(long long x) {
  return (unsigned long long)(x + FX_LIM) >= (unsigned long long)(2 * FX_LIM);
}

// t / D rounded to the nearest integer, ties away from zero (D constant)
template <unsigned D>
__device__ __forceinline__ long long fx_rdiv(long long t) {
  const unsigned long long u = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  const unsigned long long r = (u + (D >> 1)) / D;
  return t < 0 ? -(long long)r : (long long)r;
}

// t / 6 rounded to the nearest integer, ties towards +infinity, for
// |t| < 1.5 * 2^62: a bias that is a multiple of 6 makes the dividend
// non-negative, so the division is an unsigned one by a constant
__device__ __forceinline__ long long fx_div6(long long t) {
  return (long long)(((unsigned long long)t + (6ull << 60) + 3ull) / 6ull) - (1ll << 60);
}

// colour-split position of cell (i,j,k) of a box, and of natural cell
// index c = i + 8j + 64k; natural cell of split position p
__device__ __forceinline__ int xpos(int i, int j, int k) {
  return (((i + j + k) & 1) << 8) | (i >> 1) | (j << 2) | (k << 5);
}
__device__ __forceinline__ int xsplit(int c) { return xpos(c & 7, (c >> 3) & 7, c >> 6); }
__device__ __forceinline__ int xcell(int p) {
  const int k = (p >> 5) & 7, j = (p >> 2) & 7;
  return 2 * (p & 3) + ((j + k + (p >> 8)) & 1) + 8 * j + 64 * k;
}

// quantum q = 2^(E - 1080) as a double
__device__ __forceinline__ double fx_q(int E) { return __longlong_as_double((long long)(E - 57) << 52); }

// nearest multiple of the quantum, in quanta; `bad` set when the value is
// not below 2^55 quanta (exponent field above E - 3, infinities, NaNs)
__device__ __forceinline__ long long fx_of(double d, int E, bool &bad) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
  bad |= (int)((bits >> 52) & 0x7ffu) > E - 3;
  return fix_of_bits(bits, E);
}

__device__ __forceinline__ int fx_E(const unsigned long long *sc) { return (int)sc[SC_FXE]; }
__device__ __forceinline__ long long fx_2g(const unsigned long long *sc, int f) {
  return (long long)sc[SC_FX2G + f];
}

// one flag per warp; every lane of the warp must call it
__device__ __forceinline__ void fx_flag(bool bad, unsigned long long *sc) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(sc + SC_ERR, FX_ERR_OVF);
}

// Stage box b of the fixed-point potential v and its six face halos in
// s[1000] (10^3, one ghost layer): same-level neighbour cells, Dirichlet
// 2g - inner, Neumann inner, refinement faces (2 inner + Ghat)/6.
__device__ __forceinline__ void fx_stage(const Grp &g, long long *s, const long long *v, const Nb &nbv,
                                         const long long *ghx, int b, const Bc &bc, const unsigned long long *sc) {
  const long long *p = v + (size_t)b * CELLS;
  long long x[CPT];
#pragma unroll
  for (int h = 0; h < CPT; ++h) x[h] = p[g.t + h * GT];
  const int slice = g.t >> 6, u = g.t & 7, w = (g.t >> 3) & 7;
  long long hv[FPS];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (f % NSL != slice) continue;
    const int r = f / NSL;
    const int nb = nbv.v[r];
    if (nb >= 0) hv[r] = v[(size_t)nb * CELLS + xsplit(face_cell(f ^ 1, u, w))];
    else if (nb == -2) hv[r] = ghx[(size_t)(6 * b + f) * FACE + u + NC * w];
    else hv[r] = bc.type[f] ? fx_2g(sc, f) : 0;
  }
  g.sync();  // earlier users of s are done
#pragma unroll
  for (int h = 0; h < CPT; ++h) s[s10(xcell(g.t + h * GT))] = x[h];
  g.sync();
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (f % NSL != slice) continue;
    const int r = f / NSL, a = f >> 1;
    const int q = s10(face_cell(f, u, w));
    const int stride = a == 0 ? 1 : (a == 1 ? 10 : 100);
    const long long inner = s[q];
    long long gv;
    if (nbv.v[r] >= 0) gv = hv[r];
    else if (nbv.v[r] == -1) gv = bc.type[f] ? hv[r] - inner : inner;
    else gv = fx_div6(2 * inner + hv[r]);
    s[q + ((f & 1) ? stride : -stride)] = gv;
  }
  g.sync();
}

// h^2 L phi in quanta at staged position q: sum of 6 neighbours - 6 phi
__device__ __forceinline__ long long fx_T(const long long *s, int q) {
  return s[q - 1] + s[q + 1] + s[q - 10] + s[q + 10] + s[q - 100] + s[q + 100] - 6 * s[q];
}

// ---------------------------------------------------------------------------
// red-black Gauss-Seidel, one colour per pass
// ---------------------------------------------------------------------------

// One colour of a red-black sweep on box b (Sec. 2.1.2): the cells with
// (i+j+k) % 2 == color get (sum of 6 neighbours + 6 G)/6 from the other
// colour's values; the ghosts across walls and refinement faces are
// evaluated from the updated cell's own current value.  True when a result
// leaves the fixed-point range.
__device__ __forceinline__ bool fx_color_box(const Grp &g, long long *s, int b, int color, long long *phx,
                                             const long long *__restrict__ gx, const long long *__restrict__ ghx,
                                             const Nb &nbv, const Bc &bc, const unsigned long long *sc) {
  const size_t base = (size_t)b * CELLS;
  const int oc = color ^ 1;
  long long G[RPT], x[RPT];
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    G[h] = gx[base + (color << 8) + g.t + h * GT];
    x[h] = phx[base + (oc << 8) + g.t + h * GT];
  }
  // halo cells next to this colour's face cells: the neighbour's face cell,
  // or the ghost of the face cell itself
  const int slice = g.t >> 6, u = g.t & 7, w = (g.t >> 3) & 7;
  const int cw = (u + w) & 1;
  long long hv[FPS], inn[FPS];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (f % NSL != slice) continue;
    const int r = f / NSL;
    hv[r] = 0;
    inn[r] = 0;
    if (((cw + ((f & 1) ? 1 : 0)) & 1) != color) continue;  // the face cell has the other colour
    const int nb = nbv.v[r];
    if (nb >= 0) {
      hv[r] = phx[(size_t)nb * CELLS + xsplit(face_cell(f ^ 1, u, w))];
    } else {
      inn[r] = phx[base + xsplit(face_cell(f, u, w))];
      hv[r] = nb == -2 ? ghx[(size_t)(6 * b + f) * FACE + u + NC * w] : (bc.type[f] ? fx_2g(sc, f) : 0);
    }
  }
  g.sync();  // earlier users of s are done
#pragma unroll
  for (int h = 0; h < RPT; ++h) s[s10(xcell((oc << 8) + g.t + h * GT))] = x[h];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (f % NSL != slice) continue;
    if (((cw + ((f & 1) ? 1 : 0)) & 1) != color) continue;
    const int r = f / NSL, a = f >> 1;
    const int q = s10(face_cell(f, u, w));
    const int stride = a == 0 ? 1 : (a == 1 ? 10 : 100);
    const int nb = nbv.v[r];
    long long gv;
    if (nb >= 0) gv = hv[r];
    else if (nb == -1) gv = bc.type[f] ? hv[r] - inn[r] : inn[r];
    else gv = fx_div6(2 * inn[r] + hv[r]);
    s[q + ((f & 1) ? stride : -stride)] = gv;
  }
  g.sync();
  bool bad = false;
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    const int pp = (color << 8) + g.t + h * GT;
    const int q = s10(xcell(pp));
    const long long v =
        fx_div6(s[q - 1] + s[q + 1] + s[q - 10] + s[q + 10] + s[q - 100] + s[q + 100] + 6 * G[h]);
    bad |= fx_bad(v);
    phx[base + pp] = v;
  }
  return bad;
}

// ---------------------------------------------------------------------------
// residual, restriction, FAS right-hand side, prolongation, ghosts
// ---------------------------------------------------------------------------

// Residual and restriction of box b (level l): the 64 cells of the parent
// region get the mean of their 8 children (potential) and the undivided
// sum over the children of 6 G + T (completed by fx_fas_box).
__device__ __forceinline__ void fx_resid_restrict_box(const Grp &g, long long *s, long long *sr, int b,
                                                      long long *phx, long long *gx, const long long *ghx,
                                                      const Nb &nb, const Place &pl, const Bc &bc,
                                                      const unsigned long long *sc, long long *oldx = nullptr) {
  const size_t base = (size_t)b * CELLS;
  long long G[CPT];
#pragma unroll
  for (int h = 0; h < CPT; ++h) G[h] = gx[base + g.t + h * GT];
  fx_stage(g, s, phx, nb, ghx, b, bc, sc);
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const int c = xcell(g.t + h * GT);
    sr[c] = 6 * G[h] + fx_T(s, s10(c));
  }
  g.sync();
  if (g.t >= 64) return;
  const int ci = g.t & 3, cj = (g.t >> 2) & 3, ck = g.t >> 4;
  long long ap = 0, ar = 0;
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
  const size_t cc = (size_t)pl.P * CELLS + xpos(4 * pl.ox + ci, 4 * pl.oy + cj, 4 * pl.oz + ck);
  const long long v = fx_rdiv<8>(ap);
  phx[cc] = v;
  if (oldx) oldx[cc] = v;
  gx[cc] = ar;
}

// After restriction into box b (level l-1): keep a copy of the potential,
// and on a refined box complete the FAS right-hand side
// G = (sum of children's 6 G + T - 2 T_c) / 12.  True on overflow.
__device__ __forceinline__ bool fx_fas_box(const Grp &g, long long *s, int b, const long long *phx, long long *oldx,
                                           long long *gx, const long long *ghx, const Nb &nb, bool refined,
                                           const Bc &bc, const unsigned long long *sc) {
  const size_t base = (size_t)b * CELLS;
  if (!refined) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      reinterpret_cast<longlong2 *>(oldx + base)[g.t + GT * h] =
          reinterpret_cast<const longlong2 *>(phx + base)[g.t + GT * h];
    return false;
  }
  long long P[CPT];
#pragma unroll
  for (int h = 0; h < CPT; ++h) P[h] = gx[base + g.t + h * GT];
  fx_stage(g, s, phx, nb, ghx, b, bc, sc);
  bool bad = false;
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const int pp = g.t + h * GT, q = s10(xcell(pp));
    oldx[base + pp] = s[q];
    const long long G = fx_rdiv<12>(P[h] - 2 * fx_T(s, q));
    bad |= fx_bad(G);
    gx[base + pp] = G;
  }
  return bad;
}

// Ghat = 2c + c_t1 + c_t2 of ghost cell (u,w) of refinement face F of box
// b (level l) from the level l-1 potential (Dirichlet walls 2g - c)
template <int F>
__device__ __forceinline__ void fx_cf_value(const long long *phx, long long *ghx, const int32_t *__restrict__ nbr6,
                                            const int32_t *__restrict__ parent, const int32_t *__restrict__ ijk,
                                            const Bc &bc, const unsigned long long *sc, int b, int u, int w,
                                            unsigned long long *err) {
  auto val = [&](int Q, int c) { return phx[(size_t)Q * CELLS + xsplit(c)]; };
  auto wall = [&](int f, long long ctr) { return bc.type[f] ? fx_2g(sc, f) - ctr : ctr; };
  long long c, c1, c2;
  if (!cf_coarse3<F, long long>(val, wall, nbr6, parent, ijk, b, u, w, err, c, c1, c2)) return;
  ghx[(size_t)(6 * b + F) * FACE + u + NC * w] = 2 * c + c1 + c2;
}

__device__ __forceinline__ void fx_cf_faces_box(int e, int nthreads, const long long *phx, long long *ghx,
                                                const int32_t *__restrict__ nbr6, const int32_t *__restrict__ parent,
                                                const int32_t *__restrict__ ijk, const Bc &bc,
                                                const unsigned long long *sc, int b, unsigned long long *err) {
  const int u = e & 7, w = (e >> 3) & 7, first = e >> 6, step = nthreads >> 6;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (f < first || (f - first) % step) continue;
    if (__ldg(nbr6 + 6 * b + f) != -2) continue;
    switch (f) {
      case 0: fx_cf_value<0>(phx, ghx, nbr6, parent, ijk, bc, sc, b, u, w, err); break;
      case 1: fx_cf_value<1>(phx, ghx, nbr6, parent, ijk, bc, sc, b, u, w, err); break;
      case 2: fx_cf_value<2>(phx, ghx, nbr6, parent, ijk, bc, sc, b, u, w, err); break;
      case 3: fx_cf_value<3>(phx, ghx, nbr6, parent, ijk, bc, sc, b, u, w, err); break;
      case 4: fx_cf_value<4>(phx, ghx, nbr6, parent, ijk, bc, sc, b, u, w, err); break;
      default: fx_cf_value<5>(phx, ghx, nbr6, parent, ijk, bc, sc, b, u, w, err); break;
    }
  }
}

// Prolongation into box b (level l) and the Ghat values of its refinement
// faces: mode 0 adds the correction (phi - old of level l-1, homogeneous
// wall ghosts), mode 1 overwrites with the prolonged solution (FMG).  The
// coarse values of the 4^3 parent cells under b and their face neighbours
// are staged once in sp[216].  True on overflow.
__device__ __forceinline__ bool fx_prolong_box(const Grp &g, long long *sp, int b, int mode, long long *phx,
                                               const long long *oldx, long long *ghx,
                                               const int32_t *__restrict__ nbr6, const int32_t *__restrict__ parent,
                                               const int32_t *__restrict__ ijk, const Bc &bc,
                                               const unsigned long long *sc, unsigned long long *err) {
  const int P = __ldg(parent + b);
  const int o[3] = {__ldg(ijk + 3 * b) & 1, __ldg(ijk + 3 * b + 1) & 1, __ldg(ijk + 3 * b + 2) & 1};
  auto val = [&](int Q, int c) {
    const size_t x = (size_t)Q * CELLS + xsplit(c);
    return mode ? phx[x] : phx[x] - oldx[x];
  };
  auto reg = [](int x, int y, int z) { return x + 6 * y + 36 * z; };
  g.sync();  // earlier users of sp are done
  if (g.t < 64) {
    const int x = g.t & 3, y = (g.t >> 2) & 3, z = g.t >> 4;
    sp[reg(x + 1, y + 1, z + 1)] = val(P, cidx(4 * o[0] + x, 4 * o[1] + y, 4 * o[2] + z));
  }
#pragma unroll
  for (int F = 0; F < 6; ++F) {
    const int slot = F < 4 ? 64 + 16 * F : 16 * (F - 4);
    if (g.t < slot || g.t >= slot + 16) continue;
    const int E = F >> 1, S = (F & 1) ? 1 : -1;
    const int u = (g.t - slot) & 3, w = (g.t - slot) >> 2;
    int rc[3], lc[3];
    rc[E] = S > 0 ? 5 : 0;
    rc[(E + 1) % 3] = u + 1;
    rc[(E + 2) % 3] = w + 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) lc[d] = 4 * o[d] - 1 + rc[d];
    long long v;
    if (lc[E] >= 0 && lc[E] < NC) {
      v = val(P, cidx(lc[0], lc[1], lc[2]));
    } else {
      const int Qn = __ldg(nbr6 + 6 * P + F);
      if (Qn >= 0) {
        lc[E] = S > 0 ? 0 : NC - 1;
        v = val(Qn, cidx(lc[0], lc[1], lc[2]));
      } else {
        lc[E] -= S;
        const long long ctr = val(P, cidx(lc[0], lc[1], lc[2]));
        if (Qn == -1) {
          v = bc.type[F] ? (mode ? fx_2g(sc, F) : 0) - ctr : ctr;
        } else {
          atomicOr(err, 1ull);
          v = ctr;
        }
      }
    }
    sp[reg(rc[0], rc[1], rc[2])] = v;
  }
  g.sync();
  bool bad = false;
  {
    const int cc = g.t >> 1, dx = g.t & 1;
    const int ci = cc & 3, cj = (cc >> 2) & 3, ck = cc >> 4;
    const int q = reg(ci + 1, cj + 1, ck + 1);
    const long long A = sp[q] + sp[q + (dx ? 1 : -1)];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const long long B = A + sp[q + (dy ? 6 : -6)];
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        const long long v = fx_rdiv<4>(B + sp[q + (dz ? 36 : -36)]);
        const size_t x = (size_t)b * CELLS + xpos(2 * ci + dx, 2 * cj + dy, 2 * ck + dz);
        const long long nv = mode ? v : phx[x] + v;
        bad |= fx_bad(nv);
        phx[x] = nv;
      }
    }
  }
  fx_cf_faces_box(g.t, GT, phx, ghx, nbr6, parent, ijk, bc, sc, b, err);
  return bad;
}

// max over a box group of a non-negative double given by its bit pattern
// (NaN patterns order above every finite value and infinity), pushed to
// *slot by thread 0 (red: GT/32 words of shared memory of the group)
__device__ __forceinline__ void group_umax_to(const Grp &g, unsigned long long *slot, unsigned long long v,
                                              unsigned long long *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, v, o);
    v = x > v ? x : v;
  }
  if ((g.t & 31) == 0) red[g.t >> 5] = v;
  g.sync();
  if (g.t == 0) {
    unsigned long long x = red[0];
#pragma unroll
    for (int i = 1; i < GT / 32; ++i) x = red[i] > x ? red[i] : x;
    atomicMax(slot, x);
  }
  g.sync();
}

// max over the cells of leaf box b of |f - L phi| (FP64 f, fixed-point
// phi), as the bit pattern of the non-negative double
__device__ __forceinline__ unsigned long long fx_resid_max_box(const Grp &g, long long *s, int b, const long long *phx,
                                                               const double *rhs, const long long *ghx,
                                                               const Nb &nb, const Bc &bc,
                                                               const unsigned long long *sc, double nqih2) {
  const size_t base = (size_t)b * CELLS;
  double f[CPT];
#pragma unroll
  for (int h = 0; h < CPT; ++h) f[h] = rhs[base + g.t + h * GT];
  fx_stage(g, s, phx, nb, ghx, b, bc, sc);
  unsigned long long m = 0;
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const double r = fma(__ll2double_rn(fx_T(s, s10(g.t + h * GT))), nqih2, f[h]);
    const unsigned long long a = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;
    m = a > m ? a : m;
  }
  return m;
}

// ---------------------------------------------------------------------------
// red-black Gauss-Seidel by rows: one thread per x row of the colour
// ---------------------------------------------------------------------------
//
// In the colour-split layout the 4 cells of colour c in the x row (j, k)
// of a box are contiguous (4j + 32k of the colour's half), and so are the
// other colour's 4 cells of that row.  A cell i = 2q + p of the row
// (p = (c + j + k) & 1) has its y and z neighbours at the same q in the
// other colour's rows (j+-1, k) and (j, k+-1), and its x neighbours at
// q - 1 + p and q + p in the other colour's own row; only one cell of the
// row (q = 0 when p = 0, q = 3 when p = 1) reaches across an x face.  A
// thread updates the 4 cells of its row: the other colour's rows of the
// box are staged once in shared memory (32 bytes per row), the rows
// across the box's y and z faces and the x-face value are read by the
// threads that need them, and ghosts at walls and refinement faces are
// formed from the row's own current values as in fx_color_box.  The sums
// are the same exact integer sums, so the results are bit-identical.
constexpr int RBOX = 1;  // boxes per block, 64 threads each

// the 4 values at p (16-byte aligned)
__device__ __forceinline__ void row_ld(const long long *p, long long (&v)[4]) {
  const longlong2 a = reinterpret_cast<const longlong2 *>(p)[0], b = reinterpret_cast<const longlong2 *>(p)[1];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// ghosts of face f for the 4 cells i = 2q + p of a face row (own: the
// cells' current values; gi: ghx index of the face cell of q = 0, stride
// gs per q) when the face is a wall or a refinement face
__device__ __forceinline__ void row_ghost(int nb, int f, const long long (&own)[4], const long long *ghx,
                                          size_t gi, int gs, const Bc &bc, const unsigned long long *sc,
                                          long long (&g)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (nb == -1) g[q] = bc.type[f] ? fx_2g(sc, f) - own[q] : own[q];
    else g[q] = fx_div6(2 * own[q] + ghx[gi + (size_t)gs * q]);
  }
}

__global__ void __launch_bounds__(64 * RBOX, 16 / RBOX) k_fcolor_rows(int lo, int n, int color, long long *__restrict__ phx,
                                                           const long long *__restrict__ gx,
                                                           const long long *__restrict__ ghx,
                                                           const int32_t *__restrict__ nbr6, Bc bc,
                                                           unsigned long long *sc) {
  // the other colour's rows of each box, first and second halves apart
  // (lanes on consecutive rows read consecutive 16-byte words)
  __shared__ longlong2 srow[RBOX][2][64];
  const int sub = threadIdx.x >> 6, r = threadIdx.x & 63;
  const int bi = blockIdx.x * RBOX + sub;
  const bool live = bi < n;
  const int b = lo + (live ? bi : n - 1);
  const int j = r & 7, k = r >> 3, p = (color + j + k) & 1, oc = color ^ 1;
  const int fxf = p;  // x face reached by this row: 0 (-x) when p = 0, 1 (+x) when p = 1
  const int fyf = j == 0 ? 2 : (j == NC - 1 ? 3 : -1), fzf = k == 0 ? 4 : (k == NC - 1 ? 5 : -1);
  const int nbx = __ldg(nbr6 + 6 * b + fxf);
  const int nby = fyf >= 0 ? __ldg(nbr6 + 6 * b + fyf) : 0;
  const int nbz = fzf >= 0 ? __ldg(nbr6 + 6 * b + fzf) : 0;
  pdl_wait();
  const size_t base = (size_t)b * CELLS;
  const int ro = 4 * j + 32 * k;
  // every global load first: G, the other colour's row, the row's own
  // values (for ghosts at walls and refinement faces), the rows across a y
  // or z face and the value across the x face
  long long G[4], R[4];
  row_ld(gx + base + (color << 8) + ro, G);
  row_ld(phx + base + (oc << 8) + ro, R);
  long long own[4] = {0, 0, 0, 0};
  if (nbx < 0 || nby < 0 || nbz < 0) row_ld(phx + base + (color << 8) + ro, own);
  long long ym[4], yp[4], zm[4], zp[4];
  if (j == 0) {
    if (nby >= 0) row_ld(phx + (size_t)nby * CELLS + (oc << 8) + 4 * (NC - 1) + 32 * k, ym);
    else row_ghost(nby, 2, own, ghx, (size_t)(6 * b + 2) * FACE + k + NC * p, 2 * NC, bc, sc, ym);
  } else if (j == NC - 1) {
    if (nby >= 0) row_ld(phx + (size_t)nby * CELLS + (oc << 8) + 32 * k, yp);
    else row_ghost(nby, 3, own, ghx, (size_t)(6 * b + 3) * FACE + k + NC * p, 2 * NC, bc, sc, yp);
  }
  if (k == 0) {
    if (nbz >= 0) row_ld(phx + (size_t)nbz * CELLS + (oc << 8) + 4 * j + 32 * (NC - 1), zm);
    else row_ghost(nbz, 4, own, ghx, (size_t)(6 * b + 4) * FACE + p + NC * j, 2, bc, sc, zm);
  } else if (k == NC - 1) {
    if (nbz >= 0) row_ld(phx + (size_t)nbz * CELLS + (oc << 8) + 4 * j, zp);
    else row_ghost(nbz, 5, own, ghx, (size_t)(6 * b + 5) * FACE + p + NC * j, 2, bc, sc, zp);
  }
  long long xg;
  {
    const long long oe = p ? own[3] : own[0];  // the row's cell at the face
    if (nbx >= 0) xg = phx[(size_t)nbx * CELLS + (oc << 8) + ro + (p ? 0 : 3)];
    else if (nbx == -1) xg = bc.type[fxf] ? fx_2g(sc, fxf) - oe : oe;
    else xg = fx_div6(2 * oe + ghx[(size_t)(6 * b + fxf) * FACE + j + NC * k]);
  }
  srow[sub][0][r] = make_longlong2(R[0], R[1]);
  srow[sub][1][r] = make_longlong2(R[2], R[3]);
  __syncthreads();
  auto srow_ld = [&](int rr, long long (&v)[4]) {
    const longlong2 a = srow[sub][0][rr], c2 = srow[sub][1][rr];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = c2.x;
    v[3] = c2.y;
  };
  if (j > 0) srow_ld(r - 1, ym);
  if (j < NC - 1) srow_ld(r + 1, yp);
  if (k > 0) srow_ld(r - 8, zm);
  if (k < NC - 1) srow_ld(r + 8, zp);
  bool bad = false;
  long long v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long xm = p ? R[q] : (q == 0 ? xg : R[q - 1]);
    const long long xp = p ? (q == 3 ? xg : R[q + 1]) : R[q];
    v[q] = fx_div6(xm + xp + ym[q] + yp[q] + zm[q] + zp[q] + 6 * G[q]);
    bad |= fx_bad(v[q]);
  }
  if (live) {
    longlong2 *dst = reinterpret_cast<longlong2 *>(phx + base + (color << 8) + ro);
    dst[0] = make_longlong2(v[0], v[1]);
    dst[1] = make_longlong2(v[2], v[3]);
  }
  fx_flag(bad && live, sc);
}

// The same colour pass with two threads per x row (128 per box): thread
// (r, h) updates the cells q = 2h, 2h + 1 of row r, with 16-byte loads and
// stores of its half rows; the other colour's own row is staged by the two
// halves and the value across the middle of the row read back from shared
// memory.  Half the work per thread of k_fcolor_rows and the warp count of
// the box kernel, for levels that are one partial wave of blocks.
__device__ __forceinline__ void half_ld(const long long *p, long long (&v)[2]) {
  const longlong2 a = *reinterpret_cast<const longlong2 *>(p);
  v[0] = a.x;
  v[1] = a.y;
}

__global__ void __launch_bounds__(128) k_fcolor_half(int lo, int color, long long *__restrict__ phx,
                                                     const long long *__restrict__ gx,
                                                     const long long *__restrict__ ghx,
                                                     const int32_t *__restrict__ nbr6, Bc bc,
                                                     unsigned long long *sc) {
  __shared__ longlong2 srow[64][2];  // the other colour's rows: half h of row r at [r][h]
  const int t = threadIdx.x, r = t >> 1, h = t & 1;
  const int b = lo + blockIdx.x;
  const int j = r & 7, k = r >> 3, p = (color + j + k) & 1, oc = color ^ 1;
  // this half holds the row's x-face cell when p == h (q = 0 for p = 0, q = 3 for p = 1)
  const bool xface = p == h;
  const int fyf = j == 0 ? 2 : (j == NC - 1 ? 3 : -1), fzf = k == 0 ? 4 : (k == NC - 1 ? 5 : -1);
  const int nbx = xface ? __ldg(nbr6 + 6 * b + p) : 0;
  const int nby = fyf >= 0 ? __ldg(nbr6 + 6 * b + fyf) : 0;
  const int nbz = fzf >= 0 ? __ldg(nbr6 + 6 * b + fzf) : 0;
  pdl_wait();
  const size_t base = (size_t)b * CELLS;
  const int ro = 4 * j + 32 * k + 2 * h;  // first of this half's two entries
  long long G[2], R[2];
  half_ld(gx + base + (color << 8) + ro, G);
  half_ld(phx + base + (oc << 8) + ro, R);
  long long own[2] = {0, 0};
  if (nbx < 0 || nby < 0 || nbz < 0) half_ld(phx + base + (color << 8) + ro, own);
  long long ym[2], yp[2], zm[2], zp[2];
  auto ghost2 = [&](int nb, int f, size_t gi, int gs, long long (&g)[2]) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (nb == -1) g[e] = bc.type[f] ? fx_2g(sc, f) - own[e] : own[e];
      else g[e] = fx_div6(2 * own[e] + ghx[gi + (size_t)gs * e]);
    }
  };
  // face cell indices of q = 2h: y faces k + 8 i, z faces i + 8 j, i = 2q + p
  const int i0 = 4 * h + p;
  if (j == 0) {
    if (nby >= 0) half_ld(phx + (size_t)nby * CELLS + (oc << 8) + 4 * (NC - 1) + 32 * k + 2 * h, ym);
    else ghost2(nby, 2, (size_t)(6 * b + 2) * FACE + k + NC * i0, 2 * NC, ym);
  } else if (j == NC - 1) {
    if (nby >= 0) half_ld(phx + (size_t)nby * CELLS + (oc << 8) + 32 * k + 2 * h, yp);
    else ghost2(nby, 3, (size_t)(6 * b + 3) * FACE + k + NC * i0, 2 * NC, yp);
  }
  if (k == 0) {
    if (nbz >= 0) half_ld(phx + (size_t)nbz * CELLS + (oc << 8) + 4 * j + 32 * (NC - 1) + 2 * h, zm);
    else ghost2(nbz, 4, (size_t)(6 * b + 4) * FACE + i0 + NC * j, 2, zm);
  } else if (k == NC - 1) {
    if (nbz >= 0) half_ld(phx + (size_t)nbz * CELLS + (oc << 8) + 4 * j + 2 * h, zp);
    else ghost2(nbz, 5, (size_t)(6 * b + 5) * FACE + i0 + NC * j, 2, zp);
  }
  long long xg = 0;
  if (xface) {
    const long long oe = p ? own[1] : own[0];
    if (nbx >= 0) xg = phx[(size_t)nbx * CELLS + (oc << 8) + 4 * j + 32 * k + (p ? 0 : 3)];
    else if (nbx == -1) xg = bc.type[p] ? fx_2g(sc, p) - oe : oe;
    else xg = fx_div6(2 * oe + ghx[(size_t)(6 * b + p) * FACE + j + NC * k]);
  }
  srow[r][h] = make_longlong2(R[0], R[1]);
  __syncthreads();
  if (j > 0) half_ld(reinterpret_cast<const long long *>(&srow[r - 1][h]), ym);
  if (j < NC - 1) half_ld(reinterpret_cast<const long long *>(&srow[r + 1][h]), yp);
  if (k > 0) half_ld(reinterpret_cast<const long long *>(&srow[r - 8][h]), zm);
  if (k < NC - 1) half_ld(reinterpret_cast<const long long *>(&srow[r + 8][h]), zp);
  // x neighbours of q = 2h + e: p = 0 -> R[q - 1], R[q]; p = 1 -> R[q], R[q + 1];
  // the entry beyond this half is the other half's nearest one (or the face value)
  const longlong2 other = srow[r][h ^ 1];
  const long long left = h ? other.y : xg;    // entry q = 2h - 1 (p = 0 uses it)
  const long long right = h ? xg : other.x;   // entry q = 2h + 2 (p = 1 uses it)
  bool bad = false;
  long long v[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const long long xm = p ? R[e] : (e == 0 ? left : R[0]);
    const long long xp = p ? (e == 1 ? right : R[1]) : R[e];
    v[e] = fx_div6(xm + xp + ym[e] + yp[e] + zm[e] + zp[e] + 6 * G[e]);
    bad |= fx_bad(v[e]);
  }
  *reinterpret_cast<longlong2 *>(phx + base + (color << 8) + ro) = make_longlong2(v[0], v[1]);
  fx_flag(bad, sc);
}

// ---------------------------------------------------------------------------
// residual and restriction by rows: one thread per x row of 8 cells
// ---------------------------------------------------------------------------

// the 8 values of x row (j, k) of a box in natural order i = 0..7 from the
// two colour quads of the row (colour c holds the cells i = 2q + p_c,
// p_c = (c + j + k) & 1)
__device__ __forceinline__ void row8_from(const long long (&q0)[4], const long long (&q1)[4], int j, int k,
                                          long long (&v)[8]) {
  const int p0 = (j + k) & 1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[2 * q] = p0 ? q1[q] : q0[q];
    v[2 * q + 1] = p0 ? q0[q] : q1[q];
  }
}

__device__ __forceinline__ void row8_ld(const long long *box, int j, int k, long long (&v)[8]) {
  long long a[4], c[4];
  row_ld(box + 4 * j + 32 * k, a);
  row_ld(box + 256 + 4 * j + 32 * k, c);
  row8_from(a, c, j, k, v);
}

// ghosts of face f for the 8 cells of a face row from the row's own values
// (wall or refinement face; gi, gs: ghx index of the face cell of i = 0
// and its stride per i)
__device__ __forceinline__ void row8_ghost(int nb, int f, const long long (&v)[8], const long long *ghx, size_t gi,
                                           int gs, const Bc &bc, const unsigned long long *sc, long long (&g)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (nb == -1) g[i] = bc.type[f] ? fx_2g(sc, f) - v[i] : v[i];
    else g[i] = fx_div6(2 * v[i] + ghx[gi + (size_t)gs * i]);
  }
}

// Residual and restriction of box b (as fx_resid_restrict_box) with one
// thread per x row: the row's 8 values of 6 G + T (T = h^2 L phi in quanta)
// and of phi are summed in x pairs, then over the 2 x 2 rows of a coarse
// row with lane shuffles (rows j ^ 1 and k ^ 1 are lanes ^ 1 and ^ 8); the
// lanes of even j and k write the 4 coarse cells.  Exact integer sums: the
// same bits as the box kernel.
__global__ void __launch_bounds__(64, 12) k_fresid_restrict_rows(int lo, long long *__restrict__ phx,
                                                                 long long *__restrict__ gx,
                                                                 const long long *__restrict__ ghx,
                                                                 const int32_t *__restrict__ nbr6,
                                                                 const int32_t *__restrict__ parent,
                                                                 const int32_t *__restrict__ ijk, Bc bc,
                                                                 const unsigned long long *sc) {
  __shared__ longlong2 srow[4][64];  // the rows of the box, four 16-byte chunks apart
  const int r = threadIdx.x, j = r & 7, k = r >> 3;
  const int b = lo + blockIdx.x;
  const int fyf = j == 0 ? 2 : (j == NC - 1 ? 3 : -1), fzf = k == 0 ? 4 : (k == NC - 1 ? 5 : -1);
  const int nx0 = __ldg(nbr6 + 6 * b), nx1 = __ldg(nbr6 + 6 * b + 1);
  const int nby = fyf >= 0 ? __ldg(nbr6 + 6 * b + fyf) : 0;
  const int nbz = fzf >= 0 ? __ldg(nbr6 + 6 * b + fzf) : 0;
  const Place pl = load_place(parent, ijk, b);
  pdl_wait();
  const size_t base = (size_t)b * CELLS;
  // global loads first: the row (both colours), its G, the rows across y
  // and z faces and the values across both x faces
  long long q0[4], q1[4], v[8], acc[8];
  row_ld(phx + base + 4 * j + 32 * k, q0);
  row_ld(phx + base + 256 + 4 * j + 32 * k, q1);
  row8_from(q0, q1, j, k, v);
  row8_ld(gx + base, j, k, acc);
  long long xm, xp;
  if (nx0 >= 0) xm = phx[(size_t)nx0 * CELLS + xpos(NC - 1, j, k)];
  else if (nx0 == -1) xm = bc.type[0] ? fx_2g(sc, 0) - v[0] : v[0];
  else xm = fx_div6(2 * v[0] + ghx[(size_t)(6 * b) * FACE + j + NC * k]);
  if (nx1 >= 0) xp = phx[(size_t)nx1 * CELLS + xpos(0, j, k)];
  else if (nx1 == -1) xp = bc.type[1] ? fx_2g(sc, 1) - v[NC - 1] : v[NC - 1];
  else xp = fx_div6(2 * v[NC - 1] + ghx[(size_t)(6 * b + 1) * FACE + j + NC * k]);
  // 6 G + T = 6 G - 6 phi + the six neighbours, the rows added as they come
#pragma unroll
  for (int i = 0; i < 8; ++i)
    acc[i] = 6 * acc[i] - 6 * v[i] + (i > 0 ? v[i - 1] : xm) + (i < NC - 1 ? v[i + 1] : xp);
  auto add8 = [&](const long long (&w)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] += w[i];
  };
  {
    long long w[8];
    if (j == 0) {
      if (nby >= 0) row8_ld(phx + (size_t)nby * CELLS, NC - 1, k, w);
      else row8_ghost(nby, 2, v, ghx, (size_t)(6 * b + 2) * FACE + k, NC, bc, sc, w);
      add8(w);
    } else if (j == NC - 1) {
      if (nby >= 0) row8_ld(phx + (size_t)nby * CELLS, 0, k, w);
      else row8_ghost(nby, 3, v, ghx, (size_t)(6 * b + 3) * FACE + k, NC, bc, sc, w);
      add8(w);
    }
    if (k == 0) {
      if (nbz >= 0) row8_ld(phx + (size_t)nbz * CELLS, j, NC - 1, w);
      else row8_ghost(nbz, 4, v, ghx, (size_t)(6 * b + 4) * FACE + NC * j, 1, bc, sc, w);
      add8(w);
    } else if (k == NC - 1) {
      if (nbz >= 0) row8_ld(phx + (size_t)nbz * CELLS, j, 0, w);
      else row8_ghost(nbz, 5, v, ghx, (size_t)(6 * b + 5) * FACE + NC * j, 1, bc, sc, w);
      add8(w);
    }
  }
  srow[0][r] = make_longlong2(q0[0], q0[1]);
  srow[1][r] = make_longlong2(q0[2], q0[3]);
  srow[2][r] = make_longlong2(q1[0], q1[1]);
  srow[3][r] = make_longlong2(q1[2], q1[3]);
  __syncthreads();
  auto srow8 = [&](int rr, int jj, int kk) {
    long long a4[4], c4[4], w[8];
    const longlong2 t0 = srow[0][rr], t1 = srow[1][rr], t2 = srow[2][rr], t3 = srow[3][rr];
    a4[0] = t0.x; a4[1] = t0.y; a4[2] = t1.x; a4[3] = t1.y;
    c4[0] = t2.x; c4[1] = t2.y; c4[2] = t3.x; c4[3] = t3.y;
    row8_from(a4, c4, jj, kk, w);
    add8(w);
  };
  if (j > 0) srow8(r - 1, j - 1, k);
  if (j < NC - 1) srow8(r + 1, j + 1, k);
  if (k > 0) srow8(r - 8, j, k - 1);
  if (k < NC - 1) srow8(r + 8, j, k + 1);
  long long sp[4], sa[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    sp[c] = v[2 * c] + v[2 * c + 1];
    sa[c] = acc[2 * c] + acc[2 * c + 1];
    sp[c] += __shfl_xor_sync(0xffffffffu, sp[c], 1);
    sa[c] += __shfl_xor_sync(0xffffffffu, sa[c], 1);
    sp[c] += __shfl_xor_sync(0xffffffffu, sp[c], 8);
    sa[c] += __shfl_xor_sync(0xffffffffu, sa[c], 8);
  }
  if (((j | k) & 1) == 0) {
    const size_t pb = (size_t)pl.P * CELLS;
    const int cy = 4 * pl.oy + (j >> 1), cz = 4 * pl.oz + (k >> 1);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const size_t cc = pb + xpos(4 * pl.ox + c, cy, cz);
      phx[cc] = fx_rdiv<8>(sp[c]);
      gx[cc] = sa[c];
    }
  }
}

// Blocks [0, n) take the boxes lo.. of level l.  With oldx != nullptr the
// restricted values also go to oldx (the FAS copy of the level below), and
// blocks [n, n + nl) copy the leaf boxes leaf[0, nl) of the level below
// into oldx, so that k_ffas_color0 finds the whole level's values as they
// are before its colour pass in oldx.
__global__ void __launch_bounds__(GT) k_fresid_restrict(int lo, int n, long long *__restrict__ phx,
                                                        long long *__restrict__ gx,
                                                        const long long *__restrict__ ghx,
                                                        const int32_t *__restrict__ nbr6,
                                                        const int32_t *__restrict__ parent,
                                                        const int32_t *__restrict__ ijk, Bc bc,
                                                        const unsigned long long *sc, long long *__restrict__ oldx,
                                                        const int32_t *__restrict__ leaf) {
  __shared__ long long s[1000], sr[CELLS];
  const Grp g = block_grp();
  if ((int)blockIdx.x >= n) {
    const int b = __ldg(leaf + blockIdx.x - n);
    pdl_wait();
    const size_t base = (size_t)b * CELLS;
#pragma unroll
    for (int h = 0; h < CPT; ++h) oldx[base + g.t + h * GT] = phx[base + g.t + h * GT];
    return;
  }
  const int b = lo + blockIdx.x;
  const Nb nb = load_nb(g, nbr6, b);
  const Place pl = load_place(parent, ijk, b);
  pdl_wait();
  fx_resid_restrict_box(g, s, sr, b, phx, gx, ghx, nb, pl, bc, sc, oldx);
}

__global__ void __launch_bounds__(GT) k_ffas(int lo, const long long *__restrict__ phx, long long *__restrict__ oldx,
                                             long long *__restrict__ gx, const long long *__restrict__ ghx,
                                             const int32_t *__restrict__ nbr6, const int32_t *__restrict__ child,
                                             Bc bc, unsigned long long *sc) {
  __shared__ long long s[1000];
  const Grp g = block_grp();
  const int b = lo + blockIdx.x;
  const Nb nb = load_nb(g, nbr6, b);
  const bool refined = __ldg(child + 8 * b) >= 0;
  pdl_wait();
  const bool bad = fx_fas_box(g, s, b, phx, oldx, gx, ghx, nb, refined, bc, sc);
  fx_flag(bad, sc);
}

// k_ffas fused with the first colour pass (colour 0) of the smoothing that
// follows it on the same level, for levels of one partial wave of blocks.
// The FAS term of a box reads its neighbours' face cells, whose colour-0
// values the neighbours' own blocks of this launch overwrite; so every value
// is staged from oldx, which the restriction launch before (k_fresid_restrict
// with oldx) filled with the whole level as it is now and which nothing in
// this launch writes.  The box staged once serves the FAS right-hand side
// and the colour-0 update (which reads colour-1 cells and halo values only).
// The same integer operations as k_ffas followed by a colour-0 pass: the
// same bits.  Colour 0 is the first half of the split layout: positions
// g.t + h GT with h < RPT.
__global__ void __launch_bounds__(GT) k_ffas_color0(int lo, long long *__restrict__ phx,
                                                    const long long *__restrict__ oldx, long long *__restrict__ gx,
                                                    const long long *__restrict__ ghx,
                                                    const int32_t *__restrict__ nbr6,
                                                    const int32_t *__restrict__ child, Bc bc,
                                                    unsigned long long *sc) {
  __shared__ long long s[1000];
  const Grp g = block_grp();
  const int b = lo + blockIdx.x;
  const Nb nb = load_nb(g, nbr6, b);
  const bool refined = __ldg(child + 8 * b) >= 0;
  pdl_wait();
  const size_t base = (size_t)b * CELLS;
  long long P[CPT];  // children's sums of 6 G + T (refined box) or G (leaf box)
#pragma unroll
  for (int h = 0; h < CPT; ++h) P[h] = gx[base + g.t + h * GT];
  fx_stage(g, s, oldx, nb, ghx, b, bc, sc);
  bool bad = false;
  long long G0[RPT];
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const int pp = g.t + h * GT, q = s10(xcell(pp));
    long long G = P[h];
    if (refined) {
      G = fx_rdiv<12>(P[h] - 2 * fx_T(s, q));
      bad |= fx_bad(G);
      gx[base + pp] = G;
    }
    if (h < RPT) G0[h] = G;
  }
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    const int pp = g.t + h * GT, q = s10(xcell(pp));
    const long long v =
        fx_div6(s[q - 1] + s[q + 1] + s[q - 10] + s[q + 10] + s[q - 100] + s[q + 100] + 6 * G0[h]);
    bad |= fx_bad(v);
    phx[base + pp] = v;
  }
  fx_flag(bad, sc);
}

// leaf boxes of one level whose residual norm a prolongation launch
// computes in extra blocks (n = 0: none)
struct FxNorm {
  const int32_t *leaf;
  int n;
  const double *rhs;
  double inv_h2;
  unsigned long long *slot;
};

// Prolongation by rows (large levels): blocks of 128 threads take two boxes
// of level l, one thread per fine x row of a box.  The 6^3 coarse values
// (the 4^3 parent cells under the box and their face neighbours, as in
// fx_prolong_box) are staged per box; each thread forms its row's 8 fine
// values (c + c_x + c_y + c_z)/4 and adds them to (mode 0) or writes them
// over (mode 1) its row with 16-byte loads and stores, then the box's Ghat
// values.  Blocks beyond the prolongation add the residual max of the leaf
// boxes of level l-1 (final once level l is prolonged into) to nm.slot.
// The same integer sums as fx_prolong_box (the persistent kernel's): the
// same bits.
__global__ void __launch_bounds__(128) k_fprolong_rows(int lo, int n, int mode, long long *__restrict__ phx,
                                                       const long long *__restrict__ oldx,
                                                       long long *__restrict__ ghx,
                                                       const int32_t *__restrict__ nbr6,
                                                       const int32_t *__restrict__ parent,
                                                       const int32_t *__restrict__ ijk, Bc bc,
                                                       unsigned long long *sc, FxNorm nm) {
  __shared__ long long sm[1000];  // two 216-value coarse regions, or a norm block's staged box
  __shared__ unsigned long long red[GT / 32];
  const int nblk = (n + 1) >> 1;
  if ((int)blockIdx.x >= nblk) {
    const Grp g = block_grp();
    const int b = __ldg(nm.leaf + blockIdx.x - nblk);
    const Nb nb = load_nb(g, nbr6, b);
    pdl_wait();
    const double nq = -fx_q(fx_E(sc)) * nm.inv_h2;
    const unsigned long long m = fx_resid_max_box(g, sm, b, phx, nm.rhs, ghx, nb, bc, sc, nq);
    group_umax_to(g, nm.slot, m, red);
    return;
  }
  const int sub = threadIdx.x >> 6, r = threadIdx.x & 63;
  const int bi = 2 * blockIdx.x + sub;
  const bool live = bi < n;
  const int b = lo + (live ? bi : n - 1);
  const int P = __ldg(parent + b);
  const int ox = __ldg(ijk + 3 * b) & 1, oy = __ldg(ijk + 3 * b + 1) & 1, oz = __ldg(ijk + 3 * b + 2) & 1;
  long long *sp = sm + 216 * sub;
  auto val = [&](int Q, int c) {
    const size_t x = (size_t)Q * CELLS + xsplit(c);
    return mode ? phx[x] : phx[x] - oldx[x];
  };
  auto reg = [](int x, int y, int z) { return x + 6 * y + 36 * z; };
  pdl_wait();
  {
    const int x = r & 3, y = (r >> 2) & 3, z = r >> 4;
    sp[reg(x + 1, y + 1, z + 1)] = val(P, cidx(4 * ox + x, 4 * oy + y, 4 * oz + z));
  }
  // face neighbours of the parent region: region coordinate 0 or 5 along
  // the face axis E, u + 1 and w + 1 along (E+1)%3 and (E+2)%3
  for (int e = r; e < 96; e += 64) {
    const int F = e >> 4, E = F >> 1, S = (F & 1) ? 1 : -1;
    const int u = e & 3, w = (e >> 2) & 3, ce = S > 0 ? 5 : 0;
    const int rx = E == 0 ? ce : (E == 1 ? w + 1 : u + 1);
    const int ry = E == 0 ? u + 1 : (E == 1 ? ce : w + 1);
    const int rz = E == 0 ? w + 1 : (E == 1 ? u + 1 : ce);
    int lx = 4 * ox - 1 + rx, ly = 4 * oy - 1 + ry, lz = 4 * oz - 1 + rz;
    const int le = E == 0 ? lx : (E == 1 ? ly : lz);
    long long v;
    if (le >= 0 && le < NC) {
      v = val(P, cidx(lx, ly, lz));
    } else {
      const int Qn = __ldg(nbr6 + 6 * P + F);
      if (Qn >= 0) {
        const int wrap = S > 0 ? 0 : NC - 1;
        v = val(Qn, cidx(E == 0 ? wrap : lx, E == 1 ? wrap : ly, E == 2 ? wrap : lz));
      } else {
        const long long ctr =
            val(P, cidx(lx - (E == 0 ? S : 0), ly - (E == 1 ? S : 0), lz - (E == 2 ? S : 0)));
        if (Qn == -1) {
          v = bc.type[F] ? (mode ? fx_2g(sc, F) : 0) - ctr : ctr;
        } else {
          atomicOr(sc + SC_ERR, 1ull);
          v = ctr;
        }
      }
    }
    sp[reg(rx, ry, rz)] = v;
  }
  const int j = r & 7, k = r >> 3;
  const size_t base = (size_t)b * CELLS;
  long long q0[4], q1[4], f[8];
  row_ld(phx + base + 4 * j + 32 * k, q0);
  row_ld(phx + base + 256 + 4 * j + 32 * k, q1);
  row8_from(q0, q1, j, k, f);
  __syncthreads();
  bool bad = false;
  {
    const int y = (j >> 1) + 1, z = (k >> 1) + 1, sy = (j & 1) ? 6 : -6, sz = (k & 1) ? 36 : -36;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = reg((i >> 1) + 1, y, z);
      const long long v = fx_rdiv<4>(sp[q] + sp[q + ((i & 1) ? 1 : -1)] + sp[q + sy] + sp[q + sz]);
      f[i] = mode ? v : f[i] + v;
      bad |= fx_bad(f[i]);
    }
  }
  if (live) {
    const int p0 = (j + k) & 1;
    long long a[4], c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = p0 ? f[2 * q + 1] : f[2 * q];
      c[q] = p0 ? f[2 * q] : f[2 * q + 1];
    }
    longlong2 *d0 = reinterpret_cast<longlong2 *>(phx + base + 4 * j + 32 * k);
    longlong2 *d1 = reinterpret_cast<longlong2 *>(phx + base + 256 + 4 * j + 32 * k);
    d0[0] = make_longlong2(a[0], a[1]);
    d0[1] = make_longlong2(a[2], a[3]);
    d1[0] = make_longlong2(c[0], c[1]);
    d1[1] = make_longlong2(c[2], c[3]);
    fx_cf_faces_box(r, 64, phx, ghx, nbr6, parent, ijk, bc, sc, b, sc + SC_ERR);
  }
  fx_flag(bad && live, sc);
}

// Prolongation with two threads per fine x row (128 per box, small
// levels): thread (r, h) forms the 4 fine cells i = 4h .. 4h + 3 of row r
// and updates them with one 16-byte load and store per colour.  Staging,
// Ghat values and the leaf-residual blocks as in k_fprolong_rows; the same
// bits.
__global__ void __launch_bounds__(GT) k_fprolong_half(int lo, int n, int mode, long long *__restrict__ phx,
                                                      const long long *__restrict__ oldx,
                                                      long long *__restrict__ ghx,
                                                      const int32_t *__restrict__ nbr6,
                                                      const int32_t *__restrict__ parent,
                                                      const int32_t *__restrict__ ijk, Bc bc,
                                                      unsigned long long *sc, FxNorm nm) {
  __shared__ long long sm[1000];  // the 216-value coarse region, or a norm block's staged box
  __shared__ unsigned long long red[GT / 32];
  const Grp g = block_grp();
  if ((int)blockIdx.x >= n) {
    const int b = __ldg(nm.leaf + blockIdx.x - n);
    const Nb nb = load_nb(g, nbr6, b);
    pdl_wait();
    const double nq = -fx_q(fx_E(sc)) * nm.inv_h2;
    const unsigned long long m = fx_resid_max_box(g, sm, b, phx, nm.rhs, ghx, nb, bc, sc, nq);
    group_umax_to(g, nm.slot, m, red);
    return;
  }
  const int t = threadIdx.x, b = lo + blockIdx.x;
  const int P = __ldg(parent + b);
  const int ox = __ldg(ijk + 3 * b) & 1, oy = __ldg(ijk + 3 * b + 1) & 1, oz = __ldg(ijk + 3 * b + 2) & 1;
  long long *sp = sm;
  auto val = [&](int Q, int c) {
    const size_t x = (size_t)Q * CELLS + xsplit(c);
    return mode ? phx[x] : phx[x] - oldx[x];
  };
  auto reg = [](int x, int y, int z) { return x + 6 * y + 36 * z; };
  pdl_wait();
  if (t < 64) {
    const int x = t & 3, y = (t >> 2) & 3, z = t >> 4;
    sp[reg(x + 1, y + 1, z + 1)] = val(P, cidx(4 * ox + x, 4 * oy + y, 4 * oz + z));
  }
  // face neighbours of the parent region (96 items: threads 64-127, then 0-31)
  const int e = t >= 64 ? t - 64 : t + 64;
  if (e < 96) {
    const int F = e >> 4, E = F >> 1, S = (F & 1) ? 1 : -1;
    const int u = e & 3, w = (e >> 2) & 3, ce = S > 0 ? 5 : 0;
    const int rx = E == 0 ? ce : (E == 1 ? w + 1 : u + 1);
    const int ry = E == 0 ? u + 1 : (E == 1 ? ce : w + 1);
    const int rz = E == 0 ? w + 1 : (E == 1 ? u + 1 : ce);
    const int lx = 4 * ox - 1 + rx, ly = 4 * oy - 1 + ry, lz = 4 * oz - 1 + rz;
    const int le = E == 0 ? lx : (E == 1 ? ly : lz);
    long long v;
    if (le >= 0 && le < NC) {
      v = val(P, cidx(lx, ly, lz));
    } else {
      const int Qn = __ldg(nbr6 + 6 * P + F);
      if (Qn >= 0) {
        const int wrap = S > 0 ? 0 : NC - 1;
        v = val(Qn, cidx(E == 0 ? wrap : lx, E == 1 ? wrap : ly, E == 2 ? wrap : lz));
      } else {
        const long long ctr =
            val(P, cidx(lx - (E == 0 ? S : 0), ly - (E == 1 ? S : 0), lz - (E == 2 ? S : 0)));
        if (Qn == -1) {
          v = bc.type[F] ? (mode ? fx_2g(sc, F) : 0) - ctr : ctr;
        } else {
          atomicOr(sc + SC_ERR, 1ull);
          v = ctr;
        }
      }
    }
    sp[reg(rx, ry, rz)] = v;
  }
  const int r = t >> 1, h = t & 1, j = r & 7, k = r >> 3, p0 = (j + k) & 1;
  const size_t base = (size_t)b * CELLS;
  const int ro = 4 * j + 32 * k + 2 * h;
  long long a[2], c[2];
  half_ld(phx + base + ro, a);        // colour 0, entries q = 2h, 2h + 1
  half_ld(phx + base + 256 + ro, c);  // colour 1
  g.sync();
  bool bad = false;
  {
    const int y = (j >> 1) + 1, z = (k >> 1) + 1, sy = (j & 1) ? 6 : -6, sz = (k & 1) ? 36 : -36;
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4) {
      const int i = 4 * h + e4;
      const int q = reg((i >> 1) + 1, y, z);
      const long long v = fx_rdiv<4>(sp[q] + sp[q + ((i & 1) ? 1 : -1)] + sp[q + sy] + sp[q + sz]);
      // cell i is entry e4 >> 1 of colour 0 when (i + j + k) is even, else of colour 1
      long long &cell = ((e4 + p0) & 1) ? c[e4 >> 1] : a[e4 >> 1];
      cell = mode ? v : cell + v;
      bad |= fx_bad(cell);
    }
  }
  *reinterpret_cast<longlong2 *>(phx + base + ro) = make_longlong2(a[0], a[1]);
  *reinterpret_cast<longlong2 *>(phx + base + 256 + ro) = make_longlong2(c[0], c[1]);
  fx_cf_faces_box(t, GT, phx, ghx, nbr6, parent, ijk, bc, sc, b, sc + SC_ERR);
  fx_flag(bad, sc);
}

// Ghat values of the refinement faces of boxes [lo, lo + grid), 64 threads
// per box
__global__ void __launch_bounds__(64) k_ffill_cf(int lo, const long long *__restrict__ phx, long long *__restrict__ ghx,
                                                 const int32_t *__restrict__ nbr6, const int32_t *__restrict__ parent,
                                                 const int32_t *__restrict__ ijk, Bc bc, unsigned long long *sc) {
  pdl_wait();
  fx_cf_faces_box((int)threadIdx.x, 64, phx, ghx, nbr6, parent, ijk, bc, sc, lo + blockIdx.x, sc + SC_ERR);
}

// max over leaf cells of |f - L phi| into *slot (bit pattern of a double)
__global__ void __launch_bounds__(GT) k_fresnorm(const int32_t *__restrict__ leaf, const int32_t *__restrict__ level,
                                                 const long long *__restrict__ phx, const double *__restrict__ rhs,
                                                 const long long *__restrict__ ghx, const int32_t *__restrict__ nbr6,
                                                 Bc bc, LevelH lh, unsigned long long *sc, unsigned long long *slot) {
  __shared__ long long s[1000];
  __shared__ unsigned long long red[GT / 32];
  const Grp g = block_grp();
  const int b = __ldg(leaf + blockIdx.x);
  const Nb nb = load_nb(g, nbr6, b);
  const int l = __ldg(level + b);
  pdl_wait();
  const double nq = -fx_q(fx_E(sc)) * lh.inv_h2[l];
  group_umax_to(g, slot, fx_resid_max_box(g, s, b, phx, rhs, ghx, nb, bc, sc, nq), red);
}

// Level-0 exact solve: the FAS right-hand side of level 0 from its G
// (f = -6 G q / h^2), the FP64 eigenbasis solve of the double path
// (coarse_box_io) with the Dirichlet values folded in, the result rounded
// to quanta.  It is split over a cluster of 8 blocks of 64 threads (eight
// SMs' FP64 pipes instead of one).  The transforms keep the order of
// coarse_box_io (x, y, z forward; x, y, z backward) and each coefficient is
// the same 8-term sum in the same order, so the result has the bits of the
// one-block solve (which the persistent kernel runs).
// Block r first holds the z-plane r (rhs, x and y forward), then the y-slab
// r (z forward from the 8 planes in the other blocks' shared memory, the
// eigenvalue scaling, x backward), then the x-slab r (y backward from the 8
// y-slabs, z backward, store).
// With fas != 0 it first completes the FAS right-hand side of the level-0
// box (the work of k_ffas on it: every face is a wall), each block for its
// plane from the whole box staged with its wall ghosts; the box's potential
// is only written after the last cluster barrier, when every block has
// read it.
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(64)
    k_fcoarse8(long long *__restrict__ phx, long long *__restrict__ gx, long long *__restrict__ oldx,
               const double *__restrict__ basis, Bc bc, double h2, double inv_h2, int fas,
               unsigned long long *sc) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double pa[64], pb[64], sd[64], se[64], V[192], lam[24];
  __shared__ long long sx[1000];
  const int r = (int)cl.block_rank(), t = threadIdx.x, lo = t & 7, hi = t >> 3;
  for (int i = t; i < 216; i += 64) {
    if (i < 192) V[i] = __ldg(basis + i);
    else lam[i - 192] = __ldg(basis + i);
  }
  pdl_wait();
  const int E = fx_E(sc);
  const double cf = -6.0 * fx_q(E) * inv_h2;
  bool bad = false;
  const int pp = xsplit(cidx(lo, hi, r));
  long long G;
  if (fas) {
    for (int i = t; i < CELLS; i += 64) sx[s10(i)] = phx[xsplit(i)];
    __syncthreads();
    for (int i = t; i < 6 * FACE; i += 64) {
      const int f = i >> 6, u = i & 7, w = (i >> 3) & 7, a = f >> 1;
      const int q = s10(face_cell(f, u, w)), stride = a == 0 ? 1 : (a == 1 ? 10 : 100);
      const long long inner = sx[q];
      sx[q + ((f & 1) ? stride : -stride)] = bc.type[f] ? fx_2g(sc, f) - inner : inner;
    }
    __syncthreads();
    const int q = s10(cidx(lo, hi, r));
    oldx[pp] = sx[q];
    G = fx_rdiv<12>(gx[pp] - 2 * fx_T(sx, q));
    bad |= fx_bad(G);
    gx[pp] = G;
  } else {
    G = gx[pp];
  }
  {  // plane c2 = r, cell (lo, hi, r)
    const int c[3] = {lo, hi, r};
    double v = __ll2double_rn(G) * cf;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int q = c[f >> 1] + ((f & 1) ? 1 : -1);
      if ((q < 0 || q >= NC) && bc.type[f]) v -= 2.0 * bc.val[f] * inv_h2;
    }
    pa[t] = v;
  }
  __syncthreads();
  {
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[0 * 64 + m * 8 + lo] * pa[m + 8 * hi];
    pb[t] = acc;
  }
  __syncthreads();
  {
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[1 * 64 + m * 8 + hi] * pb[lo + 8 * m];
    pa[t] = acc;  // read by the other blocks after the cluster barrier
  }
  cl.sync();
  {  // y-slab c1 = r, cell (lo, r, hi)
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) {
      const double *pm = cl.map_shared_rank(pa, m);
      acc += V[2 * 64 + m * 8 + hi] * pm[lo + 8 * r];
    }
    pb[t] = acc * h2 / (lam[lo] + lam[8 + r] + lam[16 + hi]);
  }
  __syncthreads();
  {
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[0 * 64 + lo * 8 + m] * pb[m + 8 * hi];
    sd[t] = acc;  // read by the other blocks after the cluster barrier
  }
  cl.sync();
  {  // x-slab c0 = r, cell (r, lo, hi)
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) {
      const double *pm = cl.map_shared_rank(sd, m);
      acc += V[1 * 64 + lo * 8 + m] * pm[r + 8 * hi];
    }
    se[t] = acc;
  }
  cl.sync();  // the other blocks' reads of sd are done; se is complete
  {
    double acc = 0.0;
    for (int m = 0; m < NC; ++m) acc += V[2 * 64 + hi * 8 + m] * se[lo + 8 * m];
    phx[xsplit(cidx(r, lo, hi))] = fx_of(acc, E, bad);
  }
  fx_flag(bad, sc);
}

// per-level constants of the scale computation: exponent bound of h_l^2
// (|h^2 f| < 2^(expo(f) - 1022 + eh)) and -h_l^2 / 6
struct FxLev {
  int eh[MAXL];
  double mh6[MAXL];
};

// largest exponent field of the potential and of h^2 f over all cells
// (grid-stride over boxes) into sc[SC_FXI]
__global__ void __launch_bounds__(256) k_fx_expo(int n_boxes, const int32_t *__restrict__ level,
                                                 const double *__restrict__ phi, const double *__restrict__ rhs,
                                                 FxLev fl, unsigned long long *sc) {
  pdl_wait();
  int m = 0;
  const size_t total = (size_t)n_boxes * CELLS;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int l = __ldg(level + i / CELLS);
    const int ep = (int)expo_of(phi[i]);
    const int ef = (int)expo_of(rhs[i]);
    m = max(m, max(ep, ef ? ef + fl.eh[l] : 0));
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(sc + SC_FXI, (unsigned long long)m);
}

// E = max(bound, expo(2g), FX_EMIN) + margin; the Dirichlet constants 2g
// in quanta (one thread)
__global__ void k_fx_scale(Bc bc, unsigned long long *sc) {
  pdl_wait();
  int m = (int)sc[SC_FXI];
  for (int f = 0; f < 6; ++f)
    if (bc.type[f]) m = max(m, (int)expo_of(bc.g2[f]));
  const int E = max(m, FX_EMIN) + (int)sc[SC_FXM];
  sc[SC_FXE] = (unsigned long long)E;
  bool bad = false;
  for (int f = 0; f < 6; ++f) sc[SC_FX2G + f] = (unsigned long long)(bc.type[f] ? fx_of(bc.g2[f], E, bad) : 0ll);
  if (bad) sc[SC_ERR] |= FX_ERR_OVF;
}

// phx = phi and gx = -h^2 f / 6 in quanta, for every box (CELLS / GT pairs
// per thread); with den, on leaf boxes also max |f - L 0| into *den, the
// residual of the zero potential that relative residuals divide by: its
// ghosts are 2g at Dirichlet walls and 0 everywhere else (same-level and
// refinement faces, Neumann walls), so L 0 is the sum of the wall
// constants of the cell's Dirichlet faces (added in face order) / h^2
__global__ void __launch_bounds__(GT) k_fx_init(const int32_t *__restrict__ level, const int32_t *__restrict__ child,
                                                const int32_t *__restrict__ nbr6, const double *__restrict__ phi,
                                                const double *__restrict__ rhs, long long *__restrict__ phx,
                                                long long *__restrict__ gx, FxLev fl, Bc bc, LevelH lh,
                                                unsigned long long *sc, unsigned long long *den) {
  __shared__ double red[GT / 32];
  const int b = blockIdx.x;
  const int l = __ldg(level + b);
  const bool leaf = den && __ldg(child + 8 * b) < 0;
  int wall = 0;  // bit f: face f is a Dirichlet wall
#pragma unroll
  for (int f = 0; f < 6; ++f)
    if (bc.type[f] && __ldg(nbr6 + 6 * b + f) == -1) wall |= 1 << f;
  pdl_wait();
  const int E = fx_E(sc);
  const double mh6 = fl.mh6[l], ih2 = lh.inv_h2[l];
  bool bad = false;
  double m = 0.0;
  const size_t base = (size_t)b * CELLS;
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const int c = threadIdx.x + h * GT;
    const size_t x = base + c, y = base + xsplit(c);
    const double f = rhs[x];
    phx[y] = fx_of(phi[x], E, bad);
    gx[y] = fx_of(f * mh6, E, bad);
    if (leaf) {
      const int i = c & 7, j = (c >> 3) & 7, k = c >> 6;
      double sum = 0.0;
      if ((wall & 1) && i == 0) sum += bc.g2[0];
      if ((wall & 2) && i == NC - 1) sum += bc.g2[1];
      if ((wall & 4) && j == 0) sum += bc.g2[2];
      if ((wall & 8) && j == NC - 1) sum += bc.g2[3];
      if ((wall & 16) && k == 0) sum += bc.g2[4];
      if ((wall & 32) && k == NC - 1) sum += bc.g2[5];
      m = fmax(m, fabs(fma(-sum, ih2, f)));
    }
  }
  fx_flag(bad, sc);
  if (leaf) group_max_to(block_grp(), den, m, red);
}

// phi = phx q for every box, unless the solve left the fixed-point range
// (its FP64 inputs then stay as they were for the next attempt)
__global__ void __launch_bounds__(GT) k_fx_final(const long long *__restrict__ phx, double *__restrict__ phi,
                                                 const unsigned long long *__restrict__ sc) {
  pdl_wait();
  if (sc[SC_ERR] & FX_ERR_OVF) return;
  const double q = fx_q(fx_E(sc));
  const size_t base = (size_t)blockIdx.x * CELLS;
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    const int c = threadIdx.x + h * GT;
    phi[base + c] = __ll2double_rn(phx[base + xsplit(c)]) * q;
  }
}

}  // namespace fx
