// batch.cu -- many independent Poisson solves (Eq. 1 with constant
// permittivity, the 7-point operator of the octree solve) on uniform grids
// of uneven sizes, advanced together: the batched form.
//
// Every solve s has levels k = 0 (finest, N_s cells per side) .. K_s, with
// N halved while it is even and larger than 8; the coarsest grid (at most
// 16 per side) is solved exactly in FP64 by separable eigenbases.  The work
// of all solves at one level index is one work list, processed by one
// grid-stride ("persistent") launch per level and phase: z-marching columns
// for the smoother (a whole red-black sweep per launch), the prolongation
// and the FP64 outer residual, small 3-D tiles for the restriction.  The
// cycle is a correction-scheme V(nu1,nu2) in FP32 on the error equation
// inside a per-solve FP64 defect-correction loop (residual and
// accumulation in FP64); converged solves are masked out.  A whole batched solve is one
// CUDA graph with a device-side loop; tile shape and grid size are chosen
// by timing candidate configurations (sm_batch_tune).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "sm_internal.cuh"
#include "sm_nvtx.h"

using namespace sm;

namespace {

constexpr int BMAXL = 8;          // levels per solve
constexpr int BMAXC = 16;         // coarsest grid side limit
constexpr int TILE_CELLS = 512;   // threads per tile
constexpr int NSHAPES = 5;  // four 3-D tile shapes, then the column-marching restriction
constexpr int SHAPE_COLS = 4;
// candidate tile shapes (x, y, z), x fastest in memory; the column schedule
// uses 8x8x8 tiles on the levels with less than a wave of columns
constexpr int SHAPES[NSHAPES][3] = {{8, 8, 8}, {16, 8, 4}, {32, 4, 4}, {32, 8, 2}, {8, 8, 8}};
// blocks per SM tried by the autotuner; past the resident count the hardware
// hands out the remaining columns as blocks finish, which evens out columns
// of uneven length (256-solve batch: 38.6 ms at 8, 37.7 ms at 32)
constexpr int GRID_MULTS[5] = {2, 4, 8, 16, 32};

struct BSolve {
  int nlev;                // levels 0..nlev-1, nlev-1 the coarsest
  int N[BMAXL];
  long long off[BMAXL];    // offset of level k in the FP32 pool
  float h2f[BMAXL];        // h^2 per level
  double h2, inv_h2;       // finest h^2 and 1/h^2 (FP64 outer residual)
  long long off64;         // offset of the finest grid in the FP64 arrays
};

struct TileShape {
  int tx, ty, tz;
};

__device__ __forceinline__ long long gidx(int N, int x, int y, int z) {
  return (long long)x + (long long)N * (y + (long long)N * z);
}

// physical-boundary ghost of `in` across face f (homogeneous for errors)
template <typename T>
__device__ __forceinline__ T wall(const Bc &bc, int f, T in, int homog) {
  if (bc.type[f]) return (homog ? T(0) : bc_g2<T>(bc, f)) - in;
  return in;
}

template <typename T>
__device__ __forceinline__ T sum6(const T *__restrict__ v, int N, int x, int y, int z, T c, const Bc &bc,
                                  int homog) {
  long long i = gidx(N, x, y, z);
  long long sy = N, sz = (long long)N * N;
  T s = x > 0 ? v[i - 1] : wall(bc, 0, c, homog);
  s += x < N - 1 ? v[i + 1] : wall(bc, 1, c, homog);
  s += y > 0 ? v[i - sy] : wall(bc, 2, c, homog);
  s += y < N - 1 ? v[i + sy] : wall(bc, 3, c, homog);
  s += z > 0 ? v[i - sz] : wall(bc, 4, c, homog);
  s += z < N - 1 ? v[i + sz] : wall(bc, 5, c, homog);
  return s;
}

// tile t of a list: (solve, tile x, tile y, tile z)
__device__ __forceinline__ bool tile_cell(const int4 &T, TileShape sh, int N, int &x, int &y, int &z) {
  int t = threadIdx.x;
  x = T.y * sh.tx + t % sh.tx;
  y = T.z * sh.ty + (t / sh.tx) % sh.ty;
  z = T.w * sh.tz + t / (sh.tx * sh.ty);
  return x < N && y < N && z < N;
}

// ---- z-marching columns -------------------------------------------------
//
// The smoother and the outer residual walk columns of CX x CY cells in x, y
// through the whole grid in z: one block of CT threads per column, thread t
// owning x = x0 + t % 32 and the two rows y = y0 + 2 (t / 32) + {0, 1}.
// Planes of the column, with an x/y halo, are staged in a ring of RING
// shared-memory slots by asynchronous copies (cp.async) issued several
// planes ahead.  Staged rows start 16 bytes before x0 so that rows of grids
// with N % 4 == 0 (FP32) or N even (FP64) are copied in aligned 16-byte
// chunks; other grids are copied element by element.  Halo cells outside
// the grid are zero-filled by the copy (source size 0), so in-plane
// neighbour sums need no tests; the wall ghosts enter through one
// coefficient per cell: the homogeneous ghost is +c (Neumann) or -c
// (Dirichlet), the inhomogeneous one c or 2g - c.

constexpr int CX = 32, CY = 16, CT = 256;
constexpr int RW = CX + 8;                    // FP32 staged row: x0-4 .. x0+35
constexpr int ER = CY + 4, FR = CY + 2;       // staged rows: error halo 2, rhs halo 1
constexpr int EPL = RW * ER, FPL = RW * FR;   // floats per staged plane
constexpr int RWD = CX + 4;                   // FP64 staged row: x0-2 .. x0+33
constexpr int DPL = RWD * FR;                 // doubles per staged potential plane
constexpr int RING = 8;                       // staged planes per block (power of 2)
constexpr int NRING = 2 * (CX + 2) + 2 * CY;  // cells of the one-cell ring around a column
constexpr size_t SWEEP_SMEM = sizeof(float) * RING * (EPL + FPL);
constexpr size_t SWEEP_SMEM_PHI = SWEEP_SMEM + sizeof(double) * RING * CX * CY;
constexpr size_t OUTER_SMEM = sizeof(double) * RING * DPL;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// asynchronous copy of B bytes global -> shared; zero fill when !valid
template <int B>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool valid) {
  if (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(B),
                 "r"(valid ? B : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// coefficient of c in the sum of the homogeneous wall ghosts of cell
// coordinate v along axis a (faces 2a, 2a+1)
__device__ __forceinline__ float wall_w(const Bc &bc, int a, int v, int N) {
  float w = 0.f;
  if (v == 0) w += bc.type[2 * a] ? -1.f : 1.f;
  if (v == N - 1) w += bc.type[2 * a + 1] ? -1.f : 1.f;
  return w;
}

// One full red-black Gauss-Seidel sweep (colour 0, then colour 1) of level
// k on the error, column by column, from e_in into e_out (two buffers, so
// that every column reads the sweep's starting values: a column's halo is
// never a value another column has already swept).  Step p updates colour 0
// on plane p over the column and the one-cell ring around it (the ring
// repeats what the neighbouring columns compute, from the same values),
// then colour 1 on plane p-1 over the column, which by then has all its
// colour-0 neighbours, and stores plane p-1.  The updates use the values of
// two separate colour passes over the level.  With zero_in the sweep starts
// from e = 0 (the first sweep of a level in a V-cycle): e_in is not read,
// the staged error planes are zero-filled.  With phi != nullptr (level 0,
// last sweep of a cycle) the swept error is not stored but added to the
// FP64 potential, phi += (double)e, and emax of the solve is raised to the
// largest exponent field of the new values.
// Ring use at step p: planes p-2 .. p+1 are read, p+2 .. p+4 are in flight,
// and plane p+5 is issued into the slot of plane p-3 (last read at step p-1).
// The slots of planes -1 and N are zero-filled, so every update adds six
// staged neighbours (the wall ghosts come in through the coefficient w).
__global__ void __launch_bounds__(CT) k_bt_sweep(const int4 *__restrict__ cols, int ncols, int k,
                                                 const BSolve *__restrict__ tab,
                                                 const unsigned char *__restrict__ active,
                                                 const float *__restrict__ e_in, float *__restrict__ e_out,
                                                 const float *__restrict__ f, Bc bc, double *__restrict__ phi,
                                                 unsigned *__restrict__ emax, int zero_in) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float(*se)[EPL] = reinterpret_cast<float(*)[EPL]>(smem_raw);
  float(*sf)[FPL] = reinterpret_cast<float(*)[FPL]>(smem_raw + sizeof(float) * RING * EPL);
  double(*sph)[CX * CY] = reinterpret_cast<double(*)[CX * CY]>(smem_raw + SWEEP_SMEM);
  const int t = threadIdx.x, tx = t % CX, ty2 = 2 * (t / CX);
  constexpr int NCH = (ER + FR) * (RW / 4);  // 16-byte chunks of one staged plane pair (e, f)
  for (int it = blockIdx.x; it < ncols; it += gridDim.x) {
    const int4 C = cols[it];
    if (!active[C.x]) continue;  // uniform per block
    const int N = tab[C.x].N[k];
    const long long off = tab[C.x].off[k], NN = (long long)N * N;
    const float h2 = tab[C.x].h2f[k];
    const int x0 = C.y * CX, y0 = C.z * CY;
    const float *ev = e_in + off, *fv = f + off;
    float *eo = e_out + off;
    double *pv = phi ? phi + tab[C.x].off64 : nullptr;
    const bool vec = (N & 3) == 0;
    // this thread's 16-byte chunks (at most two): shared address in slot 0,
    // source plane (e or f), in-plane element offset, inside the grid
    unsigned cdst[2] = {0u, 0u};
    int coff[2] = {0, 0};
    bool cise[2] = {false, false}, cok[2] = {false, false}, chas[2] = {false, false};
    if (vec) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = t + u * CT;
        if (i >= NCH) continue;
        const bool ise = i < ER * (RW / 4);
        const int j = ise ? i : i - ER * (RW / 4);
        const int r = j / (RW / 4), c4 = 4 * (j % (RW / 4));
        const int y = y0 - (ise ? 2 : 1) + r, x = x0 - 4 + c4;
        chas[u] = true;
        cise[u] = ise;
        cok[u] = y >= 0 && y < N && x >= 0 && x < N && !(ise && zero_in);
        coff[u] = cok[u] ? y * N + x : 0;
        cdst[u] = ise ? smem_u32(&se[0][r * RW + c4]) : smem_u32(&sf[0][r * RW + c4]);
      }
    }
    // error-plane copies into slot sl that only zero-fill it (planes -1 and
    // N, the z neighbours beyond the grid, whose terms are then exact zeros)
    auto zero_slot = [&](int sl) {
      if (vec) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (chas[u] && cise[u])
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, 0;\n" ::"r"(cdst[u] + (unsigned)sl * (EPL * 4u)),
                         "l"(ev)
                         : "memory");
      } else {
        for (int i = t; i < EPL; i += CT) cp_async<4>(&se[sl][i], ev, false);
      }
    };
    // this thread's chunk sources in plane z, advanced one plane per issue
    const float *csrc[2] = {(cise[0] ? ev : fv) + coff[0], (cise[1] ? ev : fv) + coff[1]};
    const unsigned cstr[2] = {cise[0] ? EPL * 4u : FPL * 4u, cise[1] ? EPL * 4u : FPL * 4u};
    // copies of plane z (if it exists) into slot sl = z mod RING as one
    // commit group; called for z = 0, 1, 2, ... in order
    auto issue = [&](int z, int sl) {
      if (z == N) zero_slot(sl);
      if (z < N) {
        const float *ez = ev + z * NN, *fz = fv + z * NN;
        if (vec) {
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (chas[u]) {
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(cdst[u] + (unsigned)sl * cstr[u]),
                           "l"(csrc[u]), "r"(cok[u] ? 16 : 0)
                           : "memory");
              csrc[u] += NN;
            }
        } else {
          for (int i = t; i < (ER + FR) * RW; i += CT) {
            const bool ise = i < ER * RW;
            const int j = ise ? i : i - ER * RW;
            const int r = j / RW, c = j % RW;
            const int y = y0 - (ise ? 2 : 1) + r, x = x0 - 4 + c;
            const bool ok = y >= 0 && y < N && x >= 0 && x < N && !(ise && zero_in);
            const float *src = ise ? ez : fz;
            float *dst = ise ? &se[sl][j] : &sf[sl][j];
            cp_async<4>(dst, ok ? src + y * N + x : src, ok);
          }
        }
        if (pv) {  // level 0: N even, rows of the column in 16-byte pairs
          const int r = t / (CX / 2), x = x0 + 2 * (t % (CX / 2)), y = y0 + r;
          const bool ok = x < N && y < N;
          cp_async<16>(&sph[sl][r * CX + 2 * (t % (CX / 2))], ok ? pv + z * NN + y * N + x : pv, ok);
        }
      }
      cp_commit();
    };
    // Gauss-Seidel update of the staged cell at e-plane index q (rhs index
    // qf) of the plane held in pz, with the planes below / above it in pm /
    // pp (zero planes beyond the grid) and its rhs plane in fz; w is the
    // cell's wall coefficient
    auto update = [&](float *pz, const float *pm, const float *pp, const float *fz, int q, int qf, float w) {
      const float c = pz[q];
      float s = pz[q - 1] + pz[q + 1];
      s += pz[q - RW];
      s += pz[q + RW];
      s += pm[q];
      s += pp[q];
      s = fmaf(w, c, s);
      pz[q] = (s - h2 * fz[qf]) * (1.0f / 6.0f);
    };
    // this thread's two column cells (rows ya, ya+1) and its ring cell
    const int x = x0 + tx, ya = y0 + ty2;
    const bool in = x < N && ya < N;  // N even, ya even: both rows or neither
    const int q0 = (ty2 + 2) * RW + tx + 4, qf0 = (ty2 + 1) * RW + tx + 4;
    const float wx = wall_w(bc, 0, x, N);
    const float w0 = wx + wall_w(bc, 1, ya, N), w1 = wx + wall_w(bc, 1, ya + 1, N);
    int rx = -1, ry = -1;
    if (t < NRING) {
      if (t < CX + 2) rx = x0 - 1 + t, ry = y0 - 1;
      else if (t < 2 * (CX + 2)) rx = x0 - 1 + t - (CX + 2), ry = y0 + CY;
      else if (t < 2 * (CX + 2) + CY) rx = x0 - 1, ry = y0 + t - 2 * (CX + 2);
      else rx = x0 + CX, ry = y0 + t - 2 * (CX + 2) - CY;
    }
    const bool rin = rx >= 0 && rx < N && ry >= 0 && ry < N;
    const int rq = (ry - y0 + 2) * RW + (rx - x0 + 4), rqf = (ry - y0 + 1) * RW + (rx - x0 + 4);
    const float rw = rin ? wall_w(bc, 0, rx, N) + wall_w(bc, 1, ry, N) : 0.f;
    const long long row0 = (long long)ya * N + x;
    float *eo_z = eo + row0;                         // this thread's cells of the plane stored next
    double *pv_z = pv ? pv + row0 : nullptr;
    const int par = (x + ya) & 1, rpar = (rx + ry) & 1;  // colour parities at plane 0
    unsigned em = 0;  // with phi: largest exponent field written
    __syncthreads();  // the previous column's planes are no longer read
    zero_slot((-1) & (RING - 1));  // plane -1, landing with plane 0's group
#pragma unroll
    for (int z = 0; z < RING - 3; ++z) issue(z, z);  // planes 0 .. RING-4
    // steps p = pb + i, unrolled by the ring size so that every slot index
    // and colour parity is a constant (pb is a multiple of RING)
    for (int pb = 0; pb <= N; pb += RING) {
#pragma unroll
      for (int i = 0; i < RING; ++i) {
        const int p = pb + i;
        if (p > N) break;
        cp_wait<RING - 5>();  // this thread's copies of planes <= p+1 have landed
        __syncthreads();      // everyone's have; step p-1's reads of plane p-3 are done
        issue(p + RING - 3, (i + RING - 3) & (RING - 1));
        float *Pm2 = se[(i - 2) & (RING - 1)], *Pm1 = se[(i - 1) & (RING - 1)], *P0 = se[i & (RING - 1)],
              *Pp1 = se[(i + 1) & (RING - 1)];
        const int o = par ^ (i & 1);  // row offset of the colour-0 cell of plane p and the colour-1 cell of p-1
        if (p < N) {                  // colour 0 on plane p: one column cell per thread, and the ring
          const float wz = wall_w(bc, 2, p, N);
          const float *F0 = sf[i & (RING - 1)];
          if (in) update(P0, Pm1, Pp1, F0, q0 + o * RW, qf0 + o * RW, (o ? w1 : w0) + wz);
          if (rin && rpar == (i & 1)) update(P0, Pm1, Pp1, F0, rq, rqf, rw + wz);
        }
        __syncthreads();
        if (p >= 1 && in) {  // colour 1 on plane p-1, then store both cells
          update(Pm1, Pm2, P0, sf[(i - 1) & (RING - 1)], q0 + o * RW, qf0 + o * RW,
                 (o ? w1 : w0) + wall_w(bc, 2, p - 1, N));
          const float v0 = Pm1[q0], v1 = Pm1[q0 + RW];
          if (pv) {
            const double *ph = sph[(i - 1) & (RING - 1)];
            const double n0 = ph[ty2 * CX + tx] + cvt_f32_f64(v0), n1 = ph[(ty2 + 1) * CX + tx] + cvt_f32_f64(v1);
            pv_z[0] = n0;
            pv_z[N] = n1;
            pv_z += NN;
            em = max(em, max(expo_of(n0), expo_of(n1)));
          } else {
            eo_z[0] = v0;
            eo_z[N] = v1;
            eo_z += NN;
          }
        }
      }
    }
    cp_wait<0>();
    if (pv) {  // uniform per block
      em = __reduce_max_sync(0xffffffffu, em);
      if ((t & 31) == 0 && em) atomicMax(emax + C.x, em);
    }
  }
}

// e_out = e_in on the listed columns of level k (odd sweep counts)
__global__ void __launch_bounds__(CT) k_bt_copy(const int4 *__restrict__ cols, int ncols, int k,
                                                const BSolve *__restrict__ tab,
                                                const unsigned char *__restrict__ active,
                                                const float *__restrict__ e_in, float *__restrict__ e_out) {
  const int t = threadIdx.x, tx = t % CX, ty2 = 2 * (t / CX);
  for (int it = blockIdx.x; it < ncols; it += gridDim.x) {
    const int4 C = cols[it];
    if (!active[C.x]) continue;
    const int N = tab[C.x].N[k];
    const long long off = tab[C.x].off[k];
    const int x = C.y * CX + tx;
    for (int r = 0; r < 2; ++r) {
      const int y = C.z * CY + ty2 + r;
      if (x >= N || y >= N) continue;
      for (int z = 0; z < N; ++z) e_out[off + gidx(N, x, y, z)] = e_in[off + gidx(N, x, y, z)];
    }
  }
}

// coarse rhs of level k+1 = mean of the 8 fine residuals (the coarse
// error starts at zero: the level's first sweep does not read it)
__global__ void __launch_bounds__(TILE_CELLS) k_bt_restrict(const int4 *__restrict__ tiles, int ntiles, int k,
                                                            const BSolve *__restrict__ tab,
                                                            const unsigned char *__restrict__ active,
                                                            const float *__restrict__ e, float *__restrict__ f,
                                                            Bc bc, TileShape sh) {
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    int4 T = tiles[it];
    if (!active[T.x]) continue;
    const BSolve &S = tab[T.x];
    int Nc = S.N[k + 1], Nf = S.N[k];
    int X, Y, Z;
    if (!tile_cell(T, sh, Nc, X, Y, Z)) continue;
    const float *ef = e + S.off[k], *ff = f + S.off[k];
    float inv_h2 = 1.0f / S.h2f[k];
    float acc = 0.0f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
          long long i = gidx(Nf, x, y, z);
          float c = ef[i];
          acc += ff[i] - (sum6(ef, Nf, x, y, z, c, bc, 1) - 6.0f * c) * inv_h2;
        }
    long long ic = gidx(Nc, X, Y, Z);
    f[S.off[k + 1] + ic] = acc * 0.125f;
  }
}

// Restriction of the error equation's residual r = f - A e from level k to
// f of level k+1, on the sweep columns of level k (the solves for which
// level k is not the coarsest), marching the fine planes: each thread's two
// rows (one coarse row) are summed, then x pairs by a lane shuffle, then the
// two fine planes of a coarse plane in a register; the even lanes write 1/8
// of the sum.  The error planes (one-cell halo, zero outside the grid, the
// planes -1 and N zero) are staged in a ring of eight shared-memory slots by
// 16-byte asynchronous copies issued four planes ahead, and each thread's
// two f values are loaded two planes ahead into registers; walls enter
// through the homogeneous ghost coefficient (+1 Neumann, -1 Dirichlet per
// wall face).
constexpr int RRW = CX + 8;     // staged row: x0-4 .. x0+35, whole 16-byte chunks
constexpr int RFR = CY + 2;     // staged rows: y0-1 .. y0+16
constexpr int RPL = RRW * RFR;  // floats per staged plane
__global__ void __launch_bounds__(CT, 6) k_bt_restrict_col(const int4 *__restrict__ cols, int ncols, int k,
                                                        const BSolve *__restrict__ tab,
                                                        const unsigned char *__restrict__ active,
                                                        const float *__restrict__ e, float *__restrict__ f, Bc bc) {
  __shared__ __align__(16) float se[RING][RPL];
  const int t = threadIdx.x, tx = t % CX, ty2 = 2 * (t / CX);
  for (int it = blockIdx.x; it < ncols; it += gridDim.x) {
    const int4 C = cols[it];
    if (!active[C.x]) continue;  // uniform per block
    const BSolve &S = tab[C.x];
    const int N = S.N[k], Nc = S.N[k + 1];  // N = 2 Nc
    const long long NN = (long long)N * N;
    const float *ef = e + S.off[k], *ff = f + S.off[k];
    float *fc = f + S.off[k + 1];
    const float inv_h2 = 1.0f / S.h2f[k];
    const int x0 = C.y * CX, y0 = C.z * CY, x = x0 + tx, ya = y0 + ty2;
    const bool in = x < N && ya < N;  // N even, ya even: both rows or neither
    const bool vec = (N & 3) == 0;
    // this thread's 16-byte chunk of a staged plane (vec grids): slot-0
    // offset, in-plane element offset, inside the grid
    int cdst = -1, coff = 0;
    bool cok = false;
    if (vec && t < RFR * (RRW / 4)) {
      const int r = t / (RRW / 4), c4 = 4 * (t % (RRW / 4)), y = y0 - 1 + r, xx = x0 - 4 + c4;
      cok = y >= 0 && y < N && xx >= 0 && xx < N;
      coff = cok ? y * N + xx : 0;
      cdst = r * RRW + c4;
    }
    // this thread's chunk source in plane z (vec grids), advanced one plane
    // per issue of a plane of the grid
    const float *csrc = ef + coff;
    // copies of plane z into slot sl = z mod RING (zero planes outside the
    // grid); called for z = -1, 0, 1, ... in order
    auto issue = [&](int z, int sl) {
      const bool zin = z >= 0 && z < N;
      if (vec) {
        if (cdst >= 0) cp_async<16>(&se[sl][cdst], zin ? csrc : ef, cok && zin);
        if (zin) csrc += NN;
      } else {
        for (int i = t; i < RPL; i += CT) {
          const int y = y0 - 1 + i / RRW, xx = x0 - 4 + i % RRW;
          const bool ok = zin && y >= 0 && y < N && xx >= 0 && xx < N;
          cp_async<4>(&se[sl][i], ok ? ef + z * NN + y * N + xx : ef, ok);
        }
      }
      cp_commit();
    };
    const int q0 = (ty2 + 1) * RRW + tx + 4;
    const float wx = wall_w(bc, 0, x, N);
    const float w0 = wx + wall_w(bc, 1, ya, N), w1 = wx + wall_w(bc, 1, ya + 1, N);
    // this thread's two f values of planes z (fa) and z+1 (fb), loaded two
    // planes ahead of their use
    const float *frow = ff + (in ? (long long)ya * N + x : 0);
    float fa0 = 0.f, fa1 = 0.f, fb0 = 0.f, fb1 = 0.f;
    if (in) {
      fa0 = __ldg(frow), fa1 = __ldg(frow + N);
      if (N > 1) fb0 = __ldg(frow + NN), fb1 = __ldg(frow + NN + N);
    }
    const float *fnext = frow + 2 * NN;  // f of plane z+2 at step z
    float *fcz = fc + (long long)(ya >> 1) * Nc + (x >> 1);  // this thread's coarse cell, coarse plane z/2
    float acc = 0.f;
    __syncthreads();  // the previous column's planes are no longer read
#pragma unroll
    for (int z = -1; z <= 3; ++z) issue(z, z & (RING - 1));
    // steps z = zb + i, unrolled by the ring size so that every slot index
    // is a constant (zb is a multiple of RING)
    for (int zb = 0; zb < N; zb += RING) {
#pragma unroll
      for (int i = 0; i < RING; ++i) {
        const int z = zb + i;
        if (z >= N) break;
        float fn0 = 0.f, fn1 = 0.f;
        if (in && z + 2 < N) fn0 = __ldg(fnext), fn1 = __ldg(fnext + N);
        fnext += NN;
        cp_wait<2>();     // this thread's copies of planes <= z+1 have landed
        __syncthreads();  // everyone's have; step z-1's reads are done
        issue(z + 4, (i + 4) & (RING - 1));  // into the slot of plane z-4, last read at step z-3
        const float *pm = se[(i - 1) & (RING - 1)], *pz = se[i & (RING - 1)], *pp = se[(i + 1) & (RING - 1)];
        const float wz = wall_w(bc, 2, z, N);
        float rs = 0.f;
        if (in) {
#pragma unroll
          for (int o = 0; o < 2; ++o) {
            const int q = q0 + o * RRW;
            const float c = pz[q];
            float sum = pz[q - 1] + pz[q + 1];
            sum += pz[q - RRW];
            sum += pz[q + RRW];
            sum += pm[q];
            sum += pp[q];
            sum = fmaf((o ? w1 : w0) + wz, c, sum);
            rs += (o ? fa1 : fa0) - (sum - 6.0f * c) * inv_h2;
          }
        }
        fa0 = fb0, fa1 = fb1, fb0 = fn0, fb1 = fn1;
        rs += __shfl_xor_sync(0xffffffffu, rs, 1);
        acc = (i & 1) ? acc + rs : rs;
        if (i & 1) {
          if (in && !(tx & 1)) *fcz = acc * 0.125f;
          fcz += (long long)Nc * Nc;
        }
      }
    }
    cp_wait<0>();
  }
}

// e_k += (c + c_sx + c_sy + c_sz)/4 from level k+1 (homogeneous walls), on
// the sweep columns of level k: one coarse plane Z (fine planes 2Z, 2Z+1)
// per step.  The coarse planes Z-1 .. Z+1 of the column's coarse footprint
// (with a one-cell halo, zero outside the grid) sit in a ring of four
// shared-memory slots, plane Z+2 is loaded into registers during step Z;
// the fine values are loaded two steps ahead.  A coarse neighbour outside
// the grid is the homogeneous wall ghost +c (Neumann) or -c (Dirichlet),
// added through one coefficient per fine cell.
constexpr int PX = CX / 2 + 2, PY = CY / 2 + 2, PPL = PX * PY;  // staged coarse plane
__global__ void __launch_bounds__(CT) k_bt_prolong(const int4 *__restrict__ cols, int ncols, int k,
                                                   const BSolve *__restrict__ tab,
                                                   const unsigned char *__restrict__ active,
                                                   float *__restrict__ e, Bc bc) {
  __shared__ float sc[4][PPL];
  const int t = threadIdx.x, tx = t % CX, ty2 = 2 * (t / CX);
  for (int it = blockIdx.x; it < ncols; it += gridDim.x) {
    const int4 C = cols[it];
    if (!active[C.x]) continue;  // uniform per block
    const BSolve &S = tab[C.x];
    const int N = S.N[k], Nc = S.N[k + 1];  // N = 2 Nc
    const long long NN = (long long)N * N, NNc = (long long)Nc * Nc;
    float *ef = e + S.off[k];
    const float *ec = e + S.off[k + 1];
    const int x0 = C.y * CX, y0 = C.z * CY, X0 = x0 / 2 - 1, Y0 = y0 / 2 - 1;
    const int x = x0 + tx, ya = y0 + ty2;
    const bool in = x < N && ya < N;  // N even, ya even: both rows or neither
    // this thread's coarse cell (both rows share it) and neighbour offsets
    const int Xi = x / 2 - X0, Yi = ya / 2 - Y0, sx = (x & 1) ? 1 : -1;
    const int qc = Yi * PX + Xi;
    // wall coefficients: a neighbour outside the coarse grid on the fine cell's side
    auto ww = [&](int face) { return bc.type[face] ? -1.f : 1.f; };
    float wxy0 = 0.f, wxy1 = 0.f;  // row ya looks to Y-1, row ya+1 to Y+1
    if (sx < 0 && x / 2 == 0) wxy0 += ww(0), wxy1 += ww(0);
    if (sx > 0 && x / 2 == Nc - 1) wxy0 += ww(1), wxy1 += ww(1);
    if (ya / 2 == 0) wxy0 += ww(2);
    if (ya / 2 == Nc - 1) wxy1 += ww(3);
    // coarse plane Z of the footprint (zero outside the grid): one value per thread
    auto load_c = [&](int Z) {
      float v = 0.f;
      if (t < PPL && Z < Nc) {
        const int X = X0 + t % PX, Y = Y0 + t / PX;
        if (X >= 0 && X < Nc && Y >= 0 && Y < Nc) v = ec[Z * NNc + (long long)Y * Nc + X];
      }
      return v;
    };
    const long long row0 = (long long)ya * N + x;
    // fine values (rows ya, ya+1) of planes 2Z, 2Z+1 (f) and 2Z+2, 2Z+3 (g);
    // those of step Z+2 are loaded during step Z
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
    if (in) {
      f0 = ef[row0], f1 = ef[row0 + N], f2 = ef[NN + row0], f3 = ef[NN + row0 + N];
      if (Nc > 1) g0 = ef[2 * NN + row0], g1 = ef[2 * NN + row0 + N], g2 = ef[3 * NN + row0], g3 = ef[3 * NN + row0 + N];
    }
    const float *enext = ef + 4 * NN + row0;  // plane 2Z+4 at step Z
    float *eout = ef + row0;                  // plane 2Z at step Z
    __syncthreads();  // the previous column's coarse planes are no longer read
    if (t < PPL) {
      sc[0][t] = load_c(0);
      sc[1][t] = load_c(1);
    }
    float nxt = load_c(2);
    __syncthreads();
    // steps Z = Zb + i, unrolled by the four slots so that every slot index
    // is a constant (Zb is a multiple of 4)
    for (int Zb = 0; Zb < Nc; Zb += 4) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int Z = Zb + i;
        if (Z >= Nc) break;
        float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f;
        if (in && Z + 2 < Nc) h0 = enext[0], h1 = enext[N], h2 = enext[NN], h3 = enext[NN + N];
        enext += 2 * NN;
        if (in) {
          const float *cz = sc[i & 3];
          const float c = cz[qc], cxn = cz[qc + sx];
          const float c_lo = (Z > 0) ? sc[(i - 1) & 3][qc] : 0.f;  // fine plane 2Z looks to Z-1
          const float c_hi = (Z + 1 < Nc) ? sc[(i + 1) & 3][qc] : 0.f;
          const float wz_lo = (Z == 0) ? ww(4) : 0.f, wz_hi = (Z == Nc - 1) ? ww(5) : 0.f;
          const float cym = cz[qc - PX], cyp = cz[qc + PX];
          // (c + c_x + c_y + c_z) with the wall ghosts, for the four fine cells
          eout[0] = f0 + 0.25f * fmaf(wxy0 + wz_lo, c, ((c + cxn) + cym) + c_lo);
          eout[N] = f1 + 0.25f * fmaf(wxy1 + wz_lo, c, ((c + cxn) + cyp) + c_lo);
          eout[NN] = f2 + 0.25f * fmaf(wxy0 + wz_hi, c, ((c + cxn) + cym) + c_hi);
          eout[NN + N] = f3 + 0.25f * fmaf(wxy1 + wz_hi, c, ((c + cxn) + cyp) + c_hi);
        }
        eout += 2 * NN;
        __syncthreads();  // plane Z-2's slot is free
        if (t < PPL) sc[(i + 2) & 3][t] = nxt;
        nxt = load_c(Z + 3);
        __syncthreads();
        f0 = g0, f1 = g1, f2 = g2, f3 = g3;
        g0 = h0, g1 = h1, g2 = h2, g3 = h3;
      }
    }
  }
}

// exact FP64 solve of the error equation on the coarsest grid of each
// listed solve (one block per solve): separable eigenbases per axis.  When
// the coarsest grid is the finest (k = 0) the correction, rounded to FP32
// like every other correction, is added to the FP64 potential directly (and
// emax of the solve raised to the largest exponent field written).
__global__ void __launch_bounds__(512) k_bt_coarse(const int *__restrict__ solves, int k,
                                                   const BSolve *__restrict__ tab,
                                                   const unsigned char *__restrict__ active,
                                                   float *__restrict__ e, const float *__restrict__ f, Bc bc,
                                                   double *__restrict__ phi, unsigned *__restrict__ emax) {
  extern __shared__ double sm[];
  int s = solves[blockIdx.x];
  if (!active[s]) return;
  const BSolve &S = tab[s];
  int n = S.N[k];
  int n3 = n * n * n;
  double *x = sm, *y = sm + n3, *V = sm + 2 * n3, *lam = V + 3 * BMAXC * BMAXC;
  int t = threadIdx.x;
  if (t < 3 * n) {
    int a = t / n, m = t % n;
    int lo = bc.type[2 * a], hi = bc.type[2 * a + 1];
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
      double u = (i + 0.5) / n, v;
      if (!lo && !hi) v = cospi(m * u);
      else if (lo && hi) v = sinpi((m + 1) * u);
      else if (lo) v = sinpi((m + 0.5) * u);
      else v = sinpi((m + 0.5) * (n - i - 0.5) / n);
      V[(a * BMAXC + i) * BMAXC + m] = v;
      nrm += v * v;
    }
    nrm = rsqrt(nrm);
    for (int i = 0; i < n; ++i) V[(a * BMAXC + i) * BMAXC + m] *= nrm;
    double th = (!lo && !hi) ? m : ((lo && hi) ? m + 1 : m + 0.5);
    double sn = sinpi(th / (2.0 * n));
    lam[a * BMAXC + m] = -4.0 * sn * sn;
  }
  const float *fv = f + S.off[k];
  for (int c = t; c < n3; c += blockDim.x) x[c] = (double)fv[c];
  __syncthreads();
  // forward along x, y, z; divide; backward along x, y, z
  for (int pass = 0; pass < 6; ++pass) {
    int a = pass % 3;
    bool fwd = pass < 3;
    double *src = (pass & 1) ? y : x, *dst = (pass & 1) ? x : y;
    for (int c = t; c < n3; c += blockDim.x) {
      int q[3] = {c % n, (c / n) % n, c / (n * n)};
      int stride = a == 0 ? 1 : (a == 1 ? n : n * n);
      int base = c - q[a] * stride;
      double acc = 0.0;
      for (int m = 0; m < n; ++m) {
        double vv = fwd ? V[(a * BMAXC + m) * BMAXC + q[a]] : V[(a * BMAXC + q[a]) * BMAXC + m];
        acc += vv * src[base + m * stride];
      }
      if (pass == 2) acc *= S.h2 * (double)(1 << (2 * k)) /
                            (lam[q[0]] + lam[BMAXC + q[1]] + lam[2 * BMAXC + q[2]]);
      dst[c] = acc;
    }
    __syncthreads();
  }
  // passes alternate x -> y -> x ...: the sixth ends in x
  if (k == 0) {
    double *pv = phi + S.off64;
    unsigned em = 0;
    for (int c = t; c < n3; c += blockDim.x) {
      const double v = pv[c] + (double)(float)x[c];
      pv[c] = v;
      em = max(em, expo_of(v));
    }
    em = __reduce_max_sync(0xffffffffu, em);
    if ((t & 31) == 0 && em) atomicMax(emax + s, em);
  } else {
    float *ev = e + S.off[k];
    for (int c = t; c < n3; c += blockDim.x) ev[c] = (float)x[c];
  }
}

// Outer residual on the finest grids, column by column: r = f - L phi, its
// max norm per solve and the FP32 copy of r as the error equation's rhs (the
// error itself starts at zero: the first sweep does not read it).
// The stencil sum S = (sum of the six neighbours) - 6 phi is formed exactly
// in 64-bit fixed point on the integer pipe: each staged value is mapped
// once to the nearest multiple of 2^(E - 1080), where E (at least 123)
// bounds the exponent fields of the solve's potential (emax, raised by every
// kernel that writes phi) and of the Dirichlet wall values 2g; the sum of
// the integers then has no rounding at all.  r = f - S 2^(E-1080) h^-2 is
// one FMA after S is rounded to binary64 (the hardware conversion, which
// measured faster here than the same rounding on the integer pipe).  The error of r is at most
// 6.5 2^(E-1080) h^-2 (the twelve mapped values) plus two roundings, below
// that of the plain FP64 sum (five additions and a multiply-add rounding at
// 2^-53 of values up to 2^(E-1022)), and the FP64 pipe does one operation
// per cell instead of seven.  A solve whose potential holds an infinity or
// a NaN gets NaN residuals.
// Planes of phi (one-cell halo) are staged by asynchronous copies and
// converted in place one step ahead: at step p planes p-1 .. p+1 are read,
// plane p+2 is converted, p+3 .. p+4 are in flight and plane p+5 is issued
// into the slot of plane p-3; f is loaded into registers two planes ahead.
// The max norm is taken on the bit patterns of |r|.
__global__ void __launch_bounds__(CT, 5) k_bt_outer(const int4 *__restrict__ cols, int ncols,
                                                 const BSolve *__restrict__ tab,
                                                 const unsigned char *__restrict__ active,
                                                 const double *__restrict__ phi, const double *__restrict__ f64,
                                                 float *__restrict__ f32, Bc bc, const unsigned *__restrict__ emax,
                                                 unsigned long long *__restrict__ num) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long(*sp)[DPL] = reinterpret_cast<long long(*)[DPL]>(smem_raw);
  __shared__ unsigned long long red[CT / 32];
  const int t = threadIdx.x, tx = t % CX, ty2 = 2 * (t / CX);
  int ebc = 0;  // exponent bound of the Dirichlet wall values
#pragma unroll
  for (int f = 0; f < 6; ++f)
    if (bc.type[f]) ebc = max(ebc, (int)expo_of(bc.g2[f]));
  for (int it = blockIdx.x; it < ncols; it += gridDim.x) {
    const int4 C = cols[it];
    if (!active[C.x]) continue;  // uniform per block
    const BSolve &S = tab[C.x];
    const int N = S.N[0];
    const long long o64 = S.off64, o32 = S.off[0], NN = (long long)N * N;
    const int E = max(max((int)emax[C.x], ebc), 123);
    const bool finite = E < 0x7ff;
    // 2^(E-1080) h^-2, exact: a power of two (exponent field E - 57 >= 66)
    // times h^-2
    const double kk = S.inv_h2 * __longlong_as_double((long long)(finite ? E - 57 : 1023) << 52);
    const int x0 = C.y * CX, y0 = C.z * CY;
    const double *pv = phi + o64, *fv = f64 + o64;
    const bool vec = (N & 1) == 0;
    const int x = x0 + tx, ya = y0 + ty2;
    const bool in0 = x < N && ya < N, in1 = x < N && ya + 1 < N;
    // this thread's 16-byte chunks of a staged plane (at most two): slot-0
    // shared offset, in-plane element offset, inside the grid
    int cdst[2] = {-1, -1}, coff[2] = {0, 0};
    bool cok[2] = {false, false};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = t + u * CT;
      if (!vec || i >= FR * (RWD / 2)) continue;
      const int r = i / (RWD / 2), c2 = 2 * (i % (RWD / 2)), y = y0 - 1 + r, xx = x0 - 2 + c2;
      cok[u] = y >= 0 && y < N && xx >= 0 && xx < N;
      coff[u] = cok[u] ? y * N + xx : 0;
      cdst[u] = r * RWD + c2;
    }
    auto issue = [&](int z) {
      if (z < N) {
        const int sl = z & (RING - 1);
        const double *pz = pv + z * NN;
        if (vec) {
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (cdst[u] >= 0) cp_async<16>(&sp[sl][cdst[u]], pz + coff[u], cok[u]);
        } else {
          for (int i = t; i < FR * RWD; i += CT) {
            const int y = y0 - 1 + i / RWD, xx = x0 - 2 + i % RWD;
            const bool ok = y >= 0 && y < N && xx >= 0 && xx < N;
            cp_async<8>(&sp[sl][i], ok ? pz + y * N + xx : pz, ok);
          }
        }
      }
      cp_commit();
    };
    // staged plane z -> fixed point, in place (the columns x0-1 .. x0+32
    // that the stencil reads; cells outside the grid were zero-filled)
    constexpr int NCV = FR * (CX + 2);  // values converted per plane
    int cj[3];                          // this thread's (at most three), -1 for none
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int i = t + u * CT;
      cj[u] = i < NCV ? (i / (CX + 2)) * RWD + 1 + i % (CX + 2) : -1;
    }
    auto convert = [&](int z) {
      if (z < N) {
        long long *pz = sp[z & (RING - 1)];
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (cj[u] >= 0) pz[cj[u]] = fix_of_bits((unsigned long long)pz[cj[u]], E);
      }
    };
    // ghost across wall face f of a cell holding c: c (Neumann) or 2g - c
    auto wallv = [&](int f, long long c) {
      return bc.type[f] ? fix_of_bits((unsigned long long)__double_as_longlong(bc.g2[f]), E) - c : c;
    };
    const long long row0 = (long long)ya * N + x;
    // f of planes p (set A for even p, B for odd p): loaded two steps ahead
    double fa0 = 0.0, fa1 = 0.0, fb0 = 0.0, fb1 = 0.0;
    if (in0) fa0 = fv[row0];
    if (in1) fa1 = fv[row0 + N];
    if (N > 1 && in0) fb0 = fv[NN + row0];
    if (N > 1 && in1) fb1 = fv[NN + row0 + N];
    unsigned long long m = 0;  // bit pattern of max |r|
    __syncthreads();           // the previous column's planes are no longer read
#pragma unroll
    for (int z = 0; z < RING - 3; ++z) issue(z);
    cp_wait<RING - 5>();  // planes 0 and 1 have landed
    __syncthreads();
    convert(0);
    convert(1);
    // NEU: all four in-plane faces are Neumann (a compile-time path: the
    // in-plane ghosts are then selects of c)
    auto step = [&](auto neu_tag, int p, double &f0, double &f1) {
      constexpr bool NEU = decltype(neu_tag)::value;
      cp_wait<RING - 6>();  // this thread's copies of planes <= p+2 have landed
      __syncthreads();      // everyone's have; planes <= p+1 are converted; step p-1's reads are done
      issue(p + RING - 3);
      convert(p + 2);
      const long long *pz = sp[p & (RING - 1)], *pm = sp[(p - 1) & (RING - 1)], *pp = sp[(p + 1) & (RING - 1)];
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        if (!(o ? in1 : in0)) continue;
        const int q = (ty2 + o + 1) * RWD + tx + 2, y = ya + o;
        const long long c = pz[q];
        long long xm, xp, ym, yp;
        if constexpr (NEU) {
          xm = x == 0 ? c : pz[q - 1];
          xp = x == N - 1 ? c : pz[q + 1];
          ym = y == 0 ? c : pz[q - RWD];
          yp = y == N - 1 ? c : pz[q + RWD];
        } else {
          xm = x == 0 ? wallv(0, c) : pz[q - 1];
          xp = x == N - 1 ? wallv(1, c) : pz[q + 1];
          ym = y == 0 ? wallv(2, c) : pz[q - RWD];
          yp = y == N - 1 ? wallv(3, c) : pz[q + RWD];
        }
        const long long zm = p == 0 ? wallv(4, c) : pm[q];
        const long long zp = p == N - 1 ? wallv(5, c) : pp[q];
        const long long sx = ((xm + xp) + (ym + yp)) + (zm + zp) - 6 * c;  // exact
        const double r = fma(-__ll2double_rn(sx), kk, o ? f1 : f0);
        const unsigned long long rb = finite ? (unsigned long long)__double_as_longlong(r) : 0x7ff8000000000000ull;
        f32[o32 + p * NN + row0 + o * N] = cvt_bits_f32_rn(rb);
        const unsigned long long a = rb & 0x7fffffffffffffffull;
        m = a > m ? a : m;
      }
      if (p + 2 < N) {  // this set's next plane
        if (in0) f0 = fv[(p + 2) * NN + row0];
        if (in1) f1 = fv[(p + 2) * NN + row0 + N];
      }
    };
    if (!(bc.type[0] | bc.type[1] | bc.type[2] | bc.type[3])) {
      for (int p = 0; p < N; p += 2) {
        step(std::true_type{}, p, fa0, fa1);
        if (p + 1 < N) step(std::true_type{}, p + 1, fb0, fb1);
      }
    } else {
      for (int p = 0; p < N; p += 2) {
        step(std::false_type{}, p, fa0, fa1);
        if (p + 1 < N) step(std::false_type{}, p + 1, fb0, fb1);
      }
    }
    cp_wait<0>();
    // one max per column and solve
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
      m = v > m ? v : m;
    }
    if ((t & 31) == 0) red[t >> 5] = m;
    __syncthreads();
    if (t == 0) {
      unsigned long long x2 = red[0];
      for (int i = 1; i < CT / 32; ++i) x2 = red[i] > x2 ? red[i] : x2;
      atomicMax(num + C.x, x2);
    }
  }
}

constexpr int OUTER0_BLOCKS = 4;  // resident blocks per SM (64 registers a thread)
// Residual of phi = 0 on the finest grid of every solve flagged in `active`
// (the denominators of the relative residual): r0 = f - L0, where L0 has
// only the Dirichlet ghosts 2g of wall faces.  A cell with no Dirichlet face
// takes f with no FP64 work (-(+0) * h^-2 + f = f bit for bit); the others
// take r = f - S h^-2 with one rounding, S the FP64 sum of their ghosts.
// k_bt_outer gives the same bits for a potential that is all +0 whenever
// each 2g is a multiple of its fixed-point unit and S is exact (so for
// plate values such as 0 and 2g = 2); otherwise the two differ by the
// rounding of S and of the fixed-point map, both valid residuals.  Also flags
// (nz) the solves whose stored potential is not all +0 and raises emax to
// the largest exponent field of the stored potential.
__global__ void __launch_bounds__(CT, OUTER0_BLOCKS) k_bt_outer0(const int4 *__restrict__ cols, int ncols,
                                                  const BSolve *__restrict__ tab,
                                                  const unsigned char *__restrict__ active,
                                                  const double *__restrict__ phi,
                                                  const double *__restrict__ f64, float *__restrict__ f32, Bc bc,
                                                  unsigned long long *__restrict__ num,
                                                  unsigned *__restrict__ nz, unsigned *__restrict__ emax) {
  __shared__ unsigned long long red[CT / 32];
  const int t = threadIdx.x;
  for (int it = blockIdx.x; it < ncols; it += gridDim.x) {
    const int4 C = cols[it];
    if (!active[C.x]) continue;  // uniform per block
    const BSolve &S = tab[C.x];
    const int N = S.N[0];
    const long long o64 = S.off64, o32 = S.off[0], NN = (long long)N * N;
    const double inv_h2 = S.inv_h2;
    // this thread's cells: (x, y) and (x+1, y) of every plane
    const int x = C.y * CX + 2 * (t % (CX / 2)), y = C.z * CY + t / (CX / 2);
    unsigned long long m = 0;
    unsigned nzb = 0, em = 0;
    // in-plane Dirichlet ghosts of the two cells: ((g0 + g1) + (g2 + g3)),
    // the first part of the wall sum, which does not change with the plane
    bool wxy[2];
    double sxy[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const bool w0 = x + u == 0 && bc.type[0], w1 = x + u == N - 1 && bc.type[1];
      const bool w2 = y == 0 && bc.type[2], w3 = y == N - 1 && bc.type[3];
      wxy[u] = w0 | w1 | w2 | w3;
      const double g0 = w0 ? bc.g2[0] - 0.0 : 0.0, g1 = w1 ? bc.g2[1] - 0.0 : 0.0;
      const double g2 = w2 ? bc.g2[2] - 0.0 : 0.0, g3 = w3 ? bc.g2[3] - 0.0 : 0.0;
      sxy[u] = (g0 + g1) + (g2 + g3);
    }
    const bool in = x < N && y < N, vec = (N & 1) == 0;  // N even: both cells or neither, 16-byte aligned
    const double *pz = phi + o64 + (long long)y * N + x, *fz = f64 + o64 + (long long)y * N + x;
    float *rz = f32 + o32 + (long long)y * N + x;
    // r of one cell from f, with the plane's wall terms (w4, w5)
    auto resid = [&](int u, double f, bool w4, bool w5) {
      double r = f;
      if (wxy[u] | w4 | w5) {
        const double g4 = w4 ? bc.g2[4] - 0.0 : 0.0, g5 = w5 ? bc.g2[5] - 0.0 : 0.0;
        const double sw = sxy[u] + (g4 + g5);
        r = fma(-fma(-6.0, 0.0, sw), inv_h2, f);
      }
      return (unsigned long long)__double_as_longlong(r);
    };
    auto take = [&](double v, unsigned long long rb) {
      nzb |= (unsigned)(__double2hiint(v) | __double2loint(v));
      em = max(em, expo_of(v));
      const unsigned long long a = rb & 0x7fffffffffffffffull;
      m = a > m ? a : m;
    };
    if (in) {
      // four planes per step: their loads are in flight together
#pragma unroll 4
      for (int p = 0; p < N; ++p) {
        const bool w4 = p == 0 && bc.type[4], w5 = p == N - 1 && bc.type[5];
        const long long at = p * NN;
        if (vec) {
          const double2 v = *reinterpret_cast<const double2 *>(pz + at);
          const double2 f = *reinterpret_cast<const double2 *>(fz + at);
          const unsigned long long r0 = resid(0, f.x, w4, w5), r1 = resid(1, f.y, w4, w5);
          *reinterpret_cast<float2 *>(rz + at) = make_float2(cvt_bits_f32_rn(r0), cvt_bits_f32_rn(r1));
          take(v.x, r0);
          take(v.y, r1);
        } else {
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (x + u < N) {
              const unsigned long long r = resid(u, fz[at + u], w4, w5);
              rz[at + u] = cvt_bits_f32_rn(r);
              take(pz[at + u], r);
            }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
      m = v > m ? v : m;
    }
    if ((t & 31) == 0) red[t >> 5] = m;
    em = __reduce_max_sync(0xffffffffu, em);
    if ((t & 31) == 0 && em) atomicMax(emax + C.x, em);
    const int any_nz = __syncthreads_or(nzb != 0);
    if (t == 0) {
      unsigned long long x2 = red[0];
      for (int i = 1; i < CT / 32; ++i) x2 = red[i] > x2 ? red[i] : x2;
      atomicMax(num + C.x, x2);
      if (any_nz) atomicOr(nz + C.x, 1u);
    }
    __syncthreads();  // red[] is rewritten by the next column
  }
}

// per-solve bookkeeping (one block): mode 0 -- denominators from the
// residual of phi = 0, all solves active; mode 1 -- relative residuals,
// cycles of the solves that ran, new active set and the loop condition
struct BState {
  unsigned long long *num, *den;
  double *rel;
  int *cycles;
  unsigned char *active;
  int *any;
  const unsigned *nz;  // per solve: stored potential not all +0
  unsigned char *work;  // per solve: the first residual of the current potential is needed
};

__global__ void k_bt_check(cudaGraphConditionalHandle h, int in_graph, int n, BState st, int mode, int counted,
                           const double *__restrict__ tolmax) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  double tol = tolmax[0];
  int maxc = (int)tolmax[1];
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    if (mode == 0) {
      // a potential that is all +0 has the residual just computed (the same
      // bits): its max is the denominator, and the next residual pass skips it
      const unsigned long long d = st.num[s];
      const bool zero = st.nz[s] == 0;
      st.den[s] = d;
      st.num[s] = zero ? d : 0;
      st.work[s] = zero ? 0 : 1;
      st.cycles[s] = 0;
      st.active[s] = 1;
      continue;
    }
    if (!st.active[s]) continue;
    double num = __longlong_as_double((long long)st.num[s]);
    double den = __longlong_as_double((long long)st.den[s]);
    double rel = den > 0.0 ? num / den : num;
    st.rel[s] = rel;
    st.num[s] = 0;
    int c = st.cycles[s] + counted;
    st.cycles[s] = c;
    int go = rel > tol && c < maxc;
    st.active[s] = (unsigned char)go;
    if (go) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && mode != 0) {
    *st.any = any;
    if (in_graph) cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct sm_batch {
  int n = 0;
  double length = 0.0;
  Bc bc;
  cudaStream_t stream = nullptr, cap = nullptr, cap2 = nullptr;
  int nu1 = 2, nu2 = 2;
  std::vector<BSolve> solves;
  int kmax = 0;                     // deepest level index over all solves
  long long pool = 0, cells64 = 0;  // FP32 pool length, finest cells
  long long len64 = 0;              // FP64 array length (grids padded, see GRID_ALIGN)
  size_t max_tiles = 0;             // capacity of the tile area (all lists, tiles and columns)
  // arena
  char *arena = nullptr;
  BSolve *d_tab = nullptr;
  double *phi = nullptr, *f64 = nullptr;
  float *e32 = nullptr, *e32b = nullptr, *f32 = nullptr;  // error (two buffers), error-equation rhs
  int4 *d_tiles = nullptr;
  int *d_coarse = nullptr;
  unsigned long long *d_num = nullptr, *d_den = nullptr;
  double *d_rel = nullptr, *d_tolmax = nullptr;
  int *d_cycles = nullptr, *d_any = nullptr;
  unsigned char *d_active = nullptr;
  unsigned *d_nz = nullptr;          // per solve: potential not all +0
  unsigned *d_emax = nullptr;        // per solve: bound of the potential's exponent fields
  unsigned char *d_work = nullptr;   // per solve: first residual of the current potential needed
  double *h_tolmax = nullptr;
  // current schedule
  int shape = 0, gmult = 4, sms = 148;
  // one side stream per level for the exact coarse solves, forked from and
  // joined back into the cycle's stream by events
  cudaStream_t side[BMAXL] = {};
  cudaEvent_t ev_fork[BMAXL] = {}, ev_join[BMAXL] = {};
  unsigned pending = 0;  // levels whose coarse solve is not joined yet
  int rcol_per_sm = 1;  // resident column-restriction blocks per SM: its one-wave grid
  std::vector<size_t> restr_off, restr_cnt;  // per level index: restriction tiles
  std::vector<size_t> coarse_off, coarse_cnt;
  std::vector<size_t> scol_off, scol_cnt;  // per level index: sweep columns
  size_t fine_off = 0, fine_cnt = 0;       // columns of level 0 of every solve (outer loop)
  cudaGraphExec_t exec = nullptr;
  bool graphs = true;
  long long launches_prefix = 0, launches_body = 0, n_launch = 0;
  std::string err;
};

static int bfail(sm_batch *b, int code, const char *msg) {
  if (b) b->err = msg;
  return code;
}
#define BCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      b->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return SM_ECUDA;                                                     \
    }                                                                      \
  } while (0)

static size_t tiles_of(int N, int s) {
  const int *sh = SHAPES[s];
  return (size_t)((N + sh[0] - 1) / sh[0]) * ((N + sh[1] - 1) / sh[1]) * ((N + sh[2] - 1) / sh[2]);
}

// Every grid starts at a multiple of GRID_ALIGN elements in its pool (FP32
// and FP64), whatever the sizes of the grids before it (coarsest grids can
// have odd sides), so that rows of grids with N % 4 == 0 (FP32) or N even
// (FP64) start on 16-byte boundaries for the 16-byte staging copies.
constexpr long long GRID_ALIGN = 32;
static long long pad_grid(long long n) { return (n + GRID_ALIGN - 1) / GRID_ALIGN * GRID_ALIGN; }

static size_t cols_of(int N) { return (size_t)((N + CX - 1) / CX) * ((N + CY - 1) / CY); }

extern "C" int sm_batch_create(sm_batch **out, int n_solves, const int *cells_per_side, double length,
                               const int *bc_type, const double *bc_val, int nu1, int nu2, void *stream) {
  if (!out || !cells_per_side || !bc_type || !bc_val || n_solves < 1 || !(length > 0.0) || nu1 < 1 || nu2 < 1)
    return SM_EINVAL;
  *out = nullptr;
  bool dir = false;
  for (int f = 0; f < 6; ++f) {
    if (bc_type[f] != 0 && bc_type[f] != 1) return SM_EINVAL;
    dir |= bc_type[f] == 1;
  }
  if (!dir) return SM_EINVAL;
  std::vector<BSolve> S(n_solves);
  long long pool = 0, c64 = 0, len64 = 0;
  int kmax = 0;
  for (int s = 0; s < n_solves; ++s) {
    int N = cells_per_side[s];
    if (N < 2 || N > 4096) return SM_EINVAL;
    BSolve &q = S[s];
    memset(&q, 0, sizeof q);
    int n = N, k = 0;
    while (true) {
      if (k >= BMAXL) return SM_EINVAL;
      q.N[k] = n;
      double h = length / n;
      q.h2f[k] = (float)(h * h);
      ++k;
      if (!(n % 2 == 0 && n > 8)) break;
      n /= 2;
    }
    if (n > BMAXC) return SM_EINVAL;  // coarsest grid too large for the exact solve
    q.nlev = k;
    double h = length / N;
    q.h2 = h * h;
    q.inv_h2 = 1.0 / (h * h);
    q.off64 = len64;
    c64 += (long long)N * N * N;
    len64 += pad_grid((long long)N * N * N);
    kmax = std::max(kmax, k - 1);
  }
  // FP32 pool ordered by level index, then solve
  for (int k = 0; k <= kmax; ++k)
    for (int s = 0; s < n_solves; ++s)
      if (k < S[s].nlev) {
        S[s].off[k] = pool;
        pool += pad_grid((long long)S[s].N[k] * S[s].N[k] * S[s].N[k]);
      }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return SM_ECUDA;
  }
  sm_batch *b = new sm_batch();
  b->n = n_solves;
  b->length = length;
  for (int f = 0; f < 6; ++f) {
    b->bc.type[f] = bc_type[f];
    b->bc.val[f] = bc_val[f];
  }
  bc_finish(b->bc);
  b->nu1 = nu1;
  b->nu2 = nu2;
  b->stream = (cudaStream_t)stream;
  b->solves = S;
  b->kmax = kmax;
  b->pool = pool;
  b->cells64 = c64;
  b->len64 = len64;
  size_t mt = 0;
  for (int sh = 0; sh < NSHAPES; ++sh) {
    size_t t = 0;
    for (auto &q : S)
      for (int k = 0; k < q.nlev; ++k) t += tiles_of(q.N[k], sh);  // restriction
    mt = std::max(mt, t);
  }
  for (auto &q : S)
    for (int k = 0; k < q.nlev; ++k) mt += cols_of(q.N[k]) * (k == 0 ? 2 : 1);  // sweep, outer
  b->max_tiles = mt;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMallocHost((void **)&b->h_tolmax, 2 * sizeof(double)) != cudaSuccess) {
    delete b;
    return SM_ECUDA;
  }
  *out = b;
  return SM_OK;
}

struct BLayout {
  size_t tab, phi, f64, e32, e32b, f32, tiles, coarse, num, den, rel, tolmax, cycles, any, active, nz, work,
      emax, total;
};

static BLayout blayout(const sm_batch *b) {
  BLayout L;
  size_t t = 0;
  auto take = [&](size_t bytes) {
    size_t at = t;
    t = (t + bytes + 255) & ~(size_t)255;
    return at;
  };
  L.tab = take(sizeof(BSolve) * b->n);
  L.phi = take(sizeof(double) * b->len64);
  L.f64 = take(sizeof(double) * b->len64);
  L.e32 = take(sizeof(float) * b->pool);
  L.e32b = take(sizeof(float) * b->pool);
  L.f32 = take(sizeof(float) * b->pool);
  L.tiles = take(sizeof(int4) * (b->max_tiles + 2 * (size_t)(b->kmax + 1)));
  L.coarse = take(sizeof(int) * b->n);
  L.num = take(sizeof(unsigned long long) * b->n);
  L.den = take(sizeof(unsigned long long) * b->n);
  L.rel = take(sizeof(double) * b->n);
  L.tolmax = take(2 * sizeof(double));
  L.cycles = take(sizeof(int) * b->n);
  L.any = take(sizeof(int));
  L.active = take(b->n);
  L.nz = take(sizeof(unsigned) * b->n);
  L.work = take(b->n);
  L.emax = take(sizeof(unsigned) * b->n);
  L.total = t;
  return L;
}

extern "C" int sm_batch_arena_size(const sm_batch *b, size_t *bytes) {
  if (!b || !bytes) return SM_EINVAL;
  *bytes = blayout(b).total;
  return SM_OK;
}

// Work lists.  Tiles of one shape: per level index the restriction target
// list (levels 1..coarsest).  Columns (shape-independent): per level index
// the sweep and prolongation list (solves for which the level is not the
// coarsest) and the finest grids of all solves (outer residual); longest
// columns first, so that the grid-stride loops end together.  The
// coarse-solve list per level index.
static int build_lists(sm_batch *b, int shape) {
  const int *sh = SHAPES[shape];
  std::vector<int4> all;
  b->restr_off.assign(b->kmax + 1, 0);
  b->restr_cnt.assign(b->kmax + 1, 0);
  b->scol_off.assign(b->kmax + 1, 0);
  b->scol_cnt.assign(b->kmax + 1, 0);
  auto push_level = [&](int k) {
    size_t start = all.size();
    for (int s = 0; s < b->n; ++s) {
      const BSolve &q = b->solves[s];
      if (!(k >= 1 && k < q.nlev)) continue;
      int N = q.N[k];
      int nx = (N + sh[0] - 1) / sh[0], ny = (N + sh[1] - 1) / sh[1], nz = (N + sh[2] - 1) / sh[2];
      for (int tz = 0; tz < nz; ++tz)
        for (int ty = 0; ty < ny; ++ty)
          for (int tx = 0; tx < nx; ++tx) all.push_back(make_int4(s, tx, ty, tz));
    }
    return std::make_pair(start, all.size() - start);
  };
  auto push_cols = [&](int k, bool fine) {
    size_t start = all.size();
    std::vector<int> order;
    for (int s = 0; s < b->n; ++s)
      if (fine || k < b->solves[s].nlev - 1) order.push_back(s);
    std::stable_sort(order.begin(), order.end(),
                     [&](int u, int v) { return b->solves[u].N[k] > b->solves[v].N[k]; });
    for (int s : order) {
      int N = b->solves[s].N[k];
      for (int cy = 0; cy < (N + CY - 1) / CY; ++cy)
        for (int cx = 0; cx < (N + CX - 1) / CX; ++cx) all.push_back(make_int4(s, cx, cy, 0));
    }
    return std::make_pair(start, all.size() - start);
  };
  for (int k = 0; k <= b->kmax; ++k) {
    auto r = push_level(k);
    b->restr_off[k] = r.first;
    b->restr_cnt[k] = r.second;
    auto c = push_cols(k, false);
    b->scol_off[k] = c.first;
    b->scol_cnt[k] = c.second;
  }
  auto f = push_cols(0, true);
  b->fine_off = f.first;
  b->fine_cnt = f.second;
  if (all.size() > b->max_tiles) return bfail(b, SM_ESTATE, "tile list capacity");
  std::vector<int> coarse;
  b->coarse_off.assign(b->kmax + 1, 0);
  b->coarse_cnt.assign(b->kmax + 1, 0);
  for (int k = 0; k <= b->kmax; ++k) {
    b->coarse_off[k] = coarse.size();
    for (int s = 0; s < b->n; ++s)
      if (b->solves[s].nlev - 1 == k) coarse.push_back(s);
    std::stable_sort(coarse.begin() + b->coarse_off[k], coarse.end(),
                     [&](int u, int v) { return b->solves[u].N[k] > b->solves[v].N[k]; });
    b->coarse_cnt[k] = coarse.size() - b->coarse_off[k];
  }
  BCK(cudaMemcpyAsync(b->d_tiles, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_coarse, coarse.data(), sizeof(int) * coarse.size(), cudaMemcpyHostToDevice,
                      b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  b->shape = shape;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return SM_OK;
}

extern "C" int sm_batch_bind_arena(sm_batch *b, void *dev_ptr, size_t bytes) {
  if (!b || !dev_ptr) return SM_EINVAL;
  BLayout L = blayout(b);
  if (bytes < L.total) return bfail(b, SM_ENOMEM, "arena too small");
  if (((uintptr_t)dev_ptr & 255) != 0) return bfail(b, SM_EINVAL, "arena not 256-byte aligned");
  char *a = (char *)dev_ptr;
  b->arena = a;
  b->d_tab = (BSolve *)(a + L.tab);
  b->phi = (double *)(a + L.phi);
  b->f64 = (double *)(a + L.f64);
  b->e32 = (float *)(a + L.e32);
  b->e32b = (float *)(a + L.e32b);
  b->f32 = (float *)(a + L.f32);
  b->d_tiles = (int4 *)(a + L.tiles);
  b->d_coarse = (int *)(a + L.coarse);
  b->d_num = (unsigned long long *)(a + L.num);
  b->d_den = (unsigned long long *)(a + L.den);
  b->d_rel = (double *)(a + L.rel);
  b->d_tolmax = (double *)(a + L.tolmax);
  b->d_cycles = (int *)(a + L.cycles);
  b->d_any = (int *)(a + L.any);
  b->d_active = (unsigned char *)(a + L.active);
  b->d_nz = (unsigned *)(a + L.nz);
  b->d_work = (unsigned char *)(a + L.work);
  b->d_emax = (unsigned *)(a + L.emax);
  BCK(cudaMemsetAsync(a, 0, L.total, b->stream));
  BCK(cudaMemcpyAsync(b->d_tab, b->solves.data(), sizeof(BSolve) * b->n, cudaMemcpyHostToDevice, b->stream));
  return build_lists(b, 0);
}

extern "C" int sm_batch_destroy(sm_batch *b) {
  if (!b) return SM_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
  for (int k = 0; k < BMAXL; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->ev_fork[k]) cudaEventDestroy(b->ev_fork[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->h_tolmax) cudaFreeHost(b->h_tolmax);
  delete b;
  return SM_OK;
}

extern "C" int sm_batch_ptrs(const sm_batch *b, double **phi, double **rhs, long long *offsets) {
  if (!b || !b->arena) return SM_EINVAL;
  if (phi) *phi = b->phi;
  if (rhs) *rhs = b->f64;
  if (offsets)
    for (int s = 0; s < b->n; ++s) offsets[s] = b->solves[s].off64;
  return SM_OK;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
static TileShape shape_of(const sm_batch *b) {
  return {SHAPES[b->shape][0], SHAPES[b->shape][1], SHAPES[b->shape][2]};
}

static int grid_for(const sm_batch *b, size_t ntiles) {
  size_t g = (size_t)b->gmult * b->sms;
  return (int)std::max<size_t>(1, std::min(g, ntiles));
}

static BState bstate(sm_batch *b) {
  return {b->d_num, b->d_den, b->d_rel, b->d_cycles, b->d_active, b->d_any, b->d_nz, b->d_work};
}

// residual of the solves flagged in `mask`; zero_phi: of phi = 0, also
// flagging (d_nz) the solves whose stored potential is not all +0 and
// setting their exponent bounds (d_emax, zeroed before)
static int outer(sm_batch *b, int zero_phi, const unsigned char *mask) {
  size_t n0 = b->fine_cnt;
  if (zero_phi)
    k_bt_outer0<<<grid_for(b, n0), CT, 0, b->stream>>>(b->d_tiles + b->fine_off, (int)n0, b->d_tab, mask, b->phi,
                                                       b->f64, b->f32, b->bc, b->d_num, b->d_nz, b->d_emax);
  else
    k_bt_outer<<<grid_for(b, n0), CT, OUTER_SMEM, b->stream>>>(b->d_tiles + b->fine_off, (int)n0, b->d_tab, mask,
                                                      b->phi, b->f64, b->f32, b->bc, b->d_emax, b->d_num);
  ++b->n_launch;
  return cudaGetLastError() == cudaSuccess ? SM_OK : bfail(b, SM_ECUDA, "outer residual launch");
}

// nu sweeps of level k, alternating between the two error buffers; the
// result is left in e32.  With from_zero (pre-smoothing) the first sweep
// starts from e = 0 without reading it; with add_phi (level 0 after the
// V-cycle) the last sweep adds the error to the FP64 potential instead of
// storing it.
static int smooth_level(sm_batch *b, int k, int nu, bool from_zero, bool add_phi) {
  size_t n = b->scol_cnt[k];
  if (!n) return SM_OK;
  const int4 *cols = b->d_tiles + b->scol_off[k];
  for (int s = 0; s < nu; ++s) {
    const float *in = (s & 1) ? b->e32b : b->e32;
    float *out = (s & 1) ? b->e32 : b->e32b;
    double *phi = (add_phi && s == nu - 1) ? b->phi : nullptr;
    k_bt_sweep<<<grid_for(b, n), CT, phi ? SWEEP_SMEM_PHI : SWEEP_SMEM, b->stream>>>(
        cols, (int)n, k, b->d_tab, b->d_active, in, out, b->f32, b->bc, phi, b->d_emax, (from_zero && s == 0) ? 1 : 0);
    ++b->n_launch;
  }
  if ((nu & 1) && !add_phi) {
    k_bt_copy<<<grid_for(b, n), CT, 0, b->stream>>>(cols, (int)n, k, b->d_tab, b->d_active, b->e32b, b->e32);
    ++b->n_launch;
  }
  return SM_OK;
}

constexpr size_t coarse_smem(int n) {
  return sizeof(double) * (2 * (size_t)n * n * n + 3 * BMAXC * BMAXC + 3 * BMAXC);
}
// The exact coarse solve is bound by the FP64 pipe of its SM (a 15^3 grid:
// 3e5 multiply-adds, about 75 us).  Its launches ask for more than half of
// an SM's shared memory, so that one block runs per SM, and list the solves
// largest first: the largest grids then each get an SM of their own.
constexpr size_t COARSE_SMEM_LAUNCH = 116 * 1024;
static_assert(COARSE_SMEM_LAUNCH >= coarse_smem(BMAXC), "coarse solve shared memory");

// dynamic shared memory of the kernels that stage more than 48 KB
static int set_attrs(sm_batch *b) {
  BCK(cudaFuncSetAttribute(k_bt_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)COARSE_SMEM_LAUNCH));
  for (int k = 1; k <= b->kmax && k < BMAXL; ++k) {
    if (!b->side[k]) BCK(cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking));
    if (!b->ev_fork[k]) BCK(cudaEventCreateWithFlags(&b->ev_fork[k], cudaEventDisableTiming));
    if (!b->ev_join[k]) BCK(cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming));
  }
  BCK(cudaFuncSetAttribute(k_bt_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM_PHI));
  BCK(cudaFuncSetAttribute(k_bt_outer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OUTER_SMEM));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->rcol_per_sm, k_bt_restrict_col, CT, 0));
  b->rcol_per_sm = std::max(1, b->rcol_per_sm);
  return SM_OK;
}

// the column restriction runs as one wave of at most RCOL_PER_SM resident
// blocks per SM whatever the grid multiplier: its blocks march whole
// columns, longest first, and a second partial wave leaves SMs idle at the
// end; four per SM (about five columns per block on the 256-solve
// workload) balanced better than six (370 against 405 us)
constexpr int RCOL_PER_SM = 4;
static size_t rcol_wave(const sm_batch *b) { return (size_t)std::min(RCOL_PER_SM, b->rcol_per_sm) * b->sms; }
static int rcol_grid(const sm_batch *b, size_t ncols) {
  return (int)std::max<size_t>(1, std::min(rcol_wave(b), ncols));
}
// the column restriction of level k -> k+1 under the column schedule, on
// levels with a full wave of columns (on the coarser ones one thread per
// coarse cell keeps more SMs busy: 17 against 25 us on the third level of
// the 256-solve workload)
static bool rcol_use(const sm_batch *b, int k) {
  return b->shape == SHAPE_COLS && b->scol_cnt[k] >= rcol_wave(b);
}

// exact solves of the solves whose coarsest grid is level k.  Level 0 runs
// in the cycle's stream (it adds to phi); a deeper level runs on its side
// stream, forked here and joined by coarse_join before the prolongation
// from level k, so that the levels' solves overlap one another and the
// coarser levels' smoothing of the other solves (disjoint grids).
static int coarse_at_level(sm_batch *b, int k) {
  size_t nc = b->coarse_cnt[k];
  if (!nc) return SM_OK;
  cudaStream_t st = b->stream;
  if (k > 0) {
    st = b->side[k];
    BCK(cudaEventRecord(b->ev_fork[k], b->stream));
    BCK(cudaStreamWaitEvent(st, b->ev_fork[k], 0));
  }
  k_bt_coarse<<<(int)nc, 512, COARSE_SMEM_LAUNCH, st>>>(b->d_coarse + b->coarse_off[k], k, b->d_tab, b->d_active,
                                                       b->e32, b->f32, b->bc, b->phi, b->d_emax);
  ++b->n_launch;
  if (k > 0) {
    BCK(cudaEventRecord(b->ev_join[k], st));
    b->pending |= 1u << k;
  }
  return SM_OK;
}

static int coarse_join(sm_batch *b, int k) {
  if (b->pending & (1u << k)) {
    BCK(cudaStreamWaitEvent(b->stream, b->ev_join[k], 0));
    b->pending &= ~(1u << k);
  }
  return SM_OK;
}

// correction-scheme V-cycle on the error equation of every active solve,
// ending with phi += e on the finest grids
static int bvcycle(sm_batch *b) {
  b->pending = 0;
  // solves whose finest grid is already the coarsest (adds to phi)
  if (int st = coarse_at_level(b, 0)) return st;
  for (int k = 0; k < b->kmax; ++k) {
    smooth_level(b, k, b->nu1, true, false);
    if (rcol_use(b, k)) {
      const size_t nc = b->scol_cnt[k];
      if (nc) {
        k_bt_restrict_col<<<rcol_grid(b, nc), CT, 0, b->stream>>>(b->d_tiles + b->scol_off[k], (int)nc, k, b->d_tab,
                                                                 b->d_active, b->e32, b->f32, b->bc);
        ++b->n_launch;
      }
    } else {
      size_t nr = b->restr_cnt[k + 1];
      if (nr) {
        k_bt_restrict<<<grid_for(b, nr), TILE_CELLS, 0, b->stream>>>(b->d_tiles + b->restr_off[k + 1], (int)nr, k,
                                                                     b->d_tab, b->d_active, b->e32, b->f32, b->bc,
                                                                     shape_of(b));
        ++b->n_launch;
      }
    }
    if (int st = coarse_at_level(b, k + 1)) return st;
  }
  for (int k = b->kmax - 1; k >= 0; --k) {
    if (int st = coarse_join(b, k + 1)) return st;  // the prolongation reads level k+1
    size_t n = b->scol_cnt[k];
    if (n) {
      k_bt_prolong<<<grid_for(b, n), CT, 0, b->stream>>>(b->d_tiles + b->scol_off[k], (int)n, k, b->d_tab,
                                                         b->d_active, b->e32, b->bc);
      ++b->n_launch;
    }
    smooth_level(b, k, b->nu2, false, k == 0);
  }
  return cudaGetLastError() == cudaSuccess ? SM_OK : bfail(b, SM_ECUDA, "V-cycle launch");
}

static int end_caps(sm_batch *b, cudaStream_t saved, int st) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t tmp = nullptr;
  if (b->cap2 && cudaStreamIsCapturing(b->cap2, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaStreamEndCapture(b->cap2, &tmp);
    if (tmp) cudaGraphDestroy(tmp);
  }
  tmp = nullptr;
  if (b->cap && cudaStreamIsCapturing(b->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaStreamEndCapture(b->cap, &tmp);
    if (tmp) cudaGraphDestroy(tmp);
  }
  b->stream = saved;
  cudaGetLastError();
  return st;
}

// denominators (residual of phi = 0), all solves active, residual of the
// current phi, first check
static int prefix(sm_batch *b, cudaGraphConditionalHandle h, int in_graph) {
  int st;
  if (cudaMemsetAsync(b->d_num, 0, sizeof(unsigned long long) * b->n, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_nz, 0, sizeof(unsigned) * b->n, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_emax, 0, sizeof(unsigned) * b->n, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_active, 1, b->n, b->stream) != cudaSuccess)
    return bfail(b, SM_ECUDA, "memset");
  if ((st = outer(b, 1, b->d_active))) return st;
  k_bt_check<<<1, 256, 0, b->stream>>>(h, in_graph, b->n, bstate(b), 0, 0, b->d_tolmax);
  ++b->n_launch;
  if ((st = outer(b, 0, b->d_work))) return st;
  k_bt_check<<<1, 256, 0, b->stream>>>(h, in_graph, b->n, bstate(b), 1, 0, b->d_tolmax);
  ++b->n_launch;
  return cudaGetLastError() == cudaSuccess ? SM_OK : bfail(b, SM_ECUDA, "prefix launch");
}

// one correction of every active solve: V-cycle with phi += e, residual, check
static int body_step(sm_batch *b, cudaGraphConditionalHandle h, int in_graph) {
  int st;
  if ((st = bvcycle(b))) return st;
  if ((st = outer(b, 0, b->d_active))) return st;
  k_bt_check<<<1, 256, 0, b->stream>>>(h, in_graph, b->n, bstate(b), 1, 1, b->d_tolmax);
  ++b->n_launch;
  return cudaGetLastError() == cudaSuccess ? SM_OK : bfail(b, SM_ECUDA, "body launch");
}

// graph: denominators (residual of phi = 0), residual of the current phi,
// first check, then WHILE(any solve active){ V-cycle; phi += e; residual;
// check }.  Starts from the potential stored in the arena.
static int capture(sm_batch *b) {
  if (!b->cap) BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  if (!b->cap2) BCK(cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking));
  if (int st = set_attrs(b)) return st;
  cudaStream_t saved = b->stream;
  BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  b->stream = b->cap;
  cudaGraph_t g = nullptr, body = nullptr, whole = nullptr;
  cudaStreamCaptureStatus cs;
  cudaGraphConditionalHandle h;
  if (cudaStreamGetCaptureInfo(b->cap, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&h, g, 0u, cudaGraphCondAssignDefault) != cudaSuccess)
    return end_caps(b, saved, bfail(b, SM_ECUDA, "graph setup"));
  long long n0 = b->n_launch;
  int st;
  if ((st = prefix(b, h, 1))) return end_caps(b, saved, st);
  b->launches_prefix = b->n_launch - n0;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(b->cap, &cs, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess)
    return end_caps(b, saved, bfail(b, SM_ECUDA, "capture deps"));
  alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
  memset(pbuf, 0, sizeof pbuf);
  cudaGraphNodeParams &p = *reinterpret_cast<cudaGraphNodeParams *>(pbuf);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &p) != cudaSuccess)
    return end_caps(b, saved, bfail(b, SM_ECUDA, "while node"));
  body = p.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(b->cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
          cudaSuccess ||
      cudaStreamBeginCaptureToGraph(b->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
          cudaSuccess)
    return end_caps(b, saved, bfail(b, SM_ECUDA, "body capture"));
  b->stream = b->cap2;
  n0 = b->n_launch;
  if ((st = body_step(b, h, 1))) return end_caps(b, saved, st);
  b->launches_body = b->n_launch - n0;
  if (cudaStreamEndCapture(b->cap2, &body) != cudaSuccess)
    return end_caps(b, saved, bfail(b, SM_ECUDA, "end body"));
  b->stream = b->cap;
  if (cudaStreamEndCapture(b->cap, &whole) != cudaSuccess)
    return end_caps(b, saved, bfail(b, SM_ECUDA, "end capture"));
  b->stream = saved;
  cudaError_t e = cudaGraphInstantiate(&b->exec, whole, 0);
  cudaGraphDestroy(whole);
  b->n_launch -= b->launches_prefix + b->launches_body;
  if (e != cudaSuccess) return bfail(b, SM_ECUDA, "instantiate");
  return SM_OK;
}

static int run(sm_batch *b, double tol, int max_cycles, int *iterations) {
  if (!b->graphs) {
    // the same launches driven from the host, one flag read per correction
    if (int st = set_attrs(b)) return st;
    b->h_tolmax[0] = tol;
    b->h_tolmax[1] = (double)max_cycles;
    BCK(cudaMemcpyAsync(b->d_tolmax, b->h_tolmax, 2 * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    int st = prefix(b, 0, 0);
    if (st) return st;
    int it = 0, any = 0;
    BCK(cudaMemcpyAsync(&any, b->d_any, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    while (any) {
      if ((st = body_step(b, 0, 0))) return st;
      ++it;
      BCK(cudaMemcpyAsync(&any, b->d_any, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
      BCK(cudaStreamSynchronize(b->stream));
    }
    // launches were counted as they were issued
    b->n_launch -= b->launches_prefix + b->launches_body * (long long)it;
    if (iterations) *iterations = it;
    return SM_OK;
  }
  if (!b->exec) {
    int st = capture(b);
    if (st) return st;
  }
  b->h_tolmax[0] = tol;
  b->h_tolmax[1] = (double)max_cycles;
  BCK(cudaMemcpyAsync(b->d_tolmax, b->h_tolmax, 2 * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaGraphLaunch(b->exec, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (iterations) {
    std::vector<int> cyc(b->n);
    BCK(cudaMemcpy(cyc.data(), b->d_cycles, sizeof(int) * b->n, cudaMemcpyDeviceToHost));
    *iterations = *std::max_element(cyc.begin(), cyc.end());
  }
  return SM_OK;
}

extern "C" int sm_batch_solve(sm_batch *b, double tol, int max_cycles, int *cycles, double *rel_res) {
  SM_RANGE();
  if (!b || max_cycles < 1) return SM_EINVAL;
  if (!b->arena) return bfail(b, SM_ESTATE, "no arena bound");
  int it = 0;
  int st = run(b, tol, max_cycles, &it);
  if (st) return st;
  b->n_launch += b->launches_prefix + b->launches_body * (long long)it;
  std::vector<int> cyc(b->n);
  std::vector<double> rel(b->n);
  BCK(cudaMemcpy(cyc.data(), b->d_cycles, sizeof(int) * b->n, cudaMemcpyDeviceToHost));
  BCK(cudaMemcpy(rel.data(), b->d_rel, sizeof(double) * b->n, cudaMemcpyDeviceToHost));
  bool ok = true;
  for (int s = 0; s < b->n; ++s) {
    if (cycles) cycles[s] = cyc[s];
    if (rel_res) rel_res[s] = rel[s];
    ok &= rel[s] <= tol;
  }
  return ok ? SM_OK : bfail(b, SM_ENOCONV, "a solve did not reach the tolerance");
}

// Autotuner: for every tile shape and grid multiplier, time a solve of
// `iters` corrections (CUDA events around the graph launch) from phi = 0
// and keep the fastest; phi is left at zero.
extern "C" int sm_batch_tune(sm_batch *b, int iters, int *shape, int *grid_mult, double *best_ms) {
  SM_RANGE();
  if (!b || iters < 1) return SM_EINVAL;
  if (!b->arena) return bfail(b, SM_ESTATE, "no arena bound");
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  double best = 1e30;
  int bs = 0, bg = 4;
  for (int s = 0; s < NSHAPES; ++s)
    for (int gm : GRID_MULTS) {
      int st = build_lists(b, s);
      if (st) return st;
      b->gmult = gm;
      BCK(cudaMemsetAsync(b->phi, 0, sizeof(double) * b->len64, b->stream));
      if ((st = run(b, 0.0, iters, nullptr))) return st;  // capture + warm-up
      BCK(cudaMemsetAsync(b->phi, 0, sizeof(double) * b->len64, b->stream));
      BCK(cudaEventRecord(e0, b->stream));
      if ((st = run(b, 0.0, iters, nullptr))) return st;
      BCK(cudaEventRecord(e1, b->stream));
      BCK(cudaEventSynchronize(e1));
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bs = s;
        bg = gm;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int st = build_lists(b, bs);
  if (st) return st;
  b->gmult = bg;
  BCK(cudaMemsetAsync(b->phi, 0, sizeof(double) * b->len64, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (shape) *shape = bs;
  if (grid_mult) *grid_mult = bg;
  if (best_ms) *best_ms = best;
  return SM_OK;
}

// Time one kernel class over all solves (every solve active), CUDA events
// on the batch stream around `reps` back-to-back launches.  Classes:
// 0 level-0 sweep (e read, f read, e written: 12 B per cell), 1 outer
// residual (phi and f read, FP32 rhs written: 20 B and two FP64-pipe
// operations per cell, the stencil sum in fixed point on the integer pipe; the
// exponent bounds are first taken from the stored potential, untimed),
// 2 level-0 prolongation (fine e read and written, coarse e
// read: 8.5 B per fine cell), 3 level-0 -> 1 restriction (fine e and f
// read, coarse f written: 8.5 B per fine cell).  Leaves the potential and
// the error arrays changed; a following solve starts from whatever phi
// holds.  Algorithmic bytes and FP64 operations count compulsory work
// only (no halo re-reads).
extern "C" int sm_batch_kernel_bench(sm_batch *b, int kclass, int reps, double *us_per_launch,
                                     double *bytes_per_launch, double *fp64_per_launch) {
  if (!b || reps < 1 || kclass < 0 || kclass > 3) return SM_EINVAL;
  if (!b->arena) return bfail(b, SM_ESTATE, "no arena bound");
  if (int st = set_attrs(b)) return st;
  long long fine = 0;  // level-0 cells of solves whose level 0 is smoothed
  for (auto &q : b->solves)
    if (q.nlev > 1) fine += (long long)q.N[0] * q.N[0] * q.N[0];
  const size_t nsw = b->scol_cnt.empty() ? 0 : b->scol_cnt[0];
  const bool rcol = b->kmax >= 1 && rcol_use(b, 0);
  const size_t nr = b->kmax >= 1 ? (rcol ? nsw : b->restr_cnt[1]) : 0;
  if ((kclass != 1 && fine == 0) || (kclass == 3 && nr == 0)) return bfail(b, SM_ESTATE, "no level below 0");
  BCK(cudaMemsetAsync(b->d_active, 1, b->n, b->stream));
  if (kclass == 1) {
    BCK(cudaMemsetAsync(b->d_emax, 0, sizeof(unsigned) * b->n, b->stream));
    BCK(cudaMemsetAsync(b->d_nz, 0, sizeof(unsigned) * b->n, b->stream));
    if (int st = outer(b, 1, b->d_active)) return st;
  }
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  auto launch = [&]() {
    switch (kclass) {
      case 0:
        k_bt_sweep<<<grid_for(b, nsw), CT, SWEEP_SMEM, b->stream>>>(b->d_tiles + b->scol_off[0], (int)nsw, 0,
                                                                     b->d_tab, b->d_active, b->e32, b->e32b,
                                                                     b->f32, b->bc, nullptr, nullptr, 0);
        break;
      case 1:
        k_bt_outer<<<grid_for(b, b->fine_cnt), CT, OUTER_SMEM, b->stream>>>(
            b->d_tiles + b->fine_off, (int)b->fine_cnt, b->d_tab, b->d_active, b->phi, b->f64, b->f32, b->bc,
            b->d_emax, b->d_num);
        break;
      case 2:
        k_bt_prolong<<<grid_for(b, nsw), CT, 0, b->stream>>>(b->d_tiles + b->scol_off[0], (int)nsw, 0, b->d_tab,
                                                             b->d_active, b->e32, b->bc);
        break;
      default:
        if (rcol)
          k_bt_restrict_col<<<rcol_grid(b, nr), CT, 0, b->stream>>>(b->d_tiles + b->scol_off[0], (int)nr, 0, b->d_tab,
                                                                   b->d_active, b->e32, b->f32, b->bc);
        else
          k_bt_restrict<<<grid_for(b, nr), TILE_CELLS, 0, b->stream>>>(b->d_tiles + b->restr_off[1], (int)nr, 0,
                                                                       b->d_tab, b->d_active, b->e32, b->f32, b->bc,
                                                                       shape_of(b));
    }
  };
  launch();  // warm-up
  BCK(cudaEventRecord(e0, b->stream));
  for (int r = 0; r < reps; ++r) launch();
  BCK(cudaEventRecord(e1, b->stream));
  BCK(cudaEventSynchronize(e1));
  float ms = 0.f;
  BCK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double cells = kclass == 1 ? (double)b->cells64 : (double)fine;
  const double per_cell[4] = {12.0, 20.0, 8.5, 8.5};
  if (us_per_launch) *us_per_launch = 1e3 * ms / reps;
  if (bytes_per_launch) *bytes_per_launch = per_cell[kclass] * cells;
  if (fp64_per_launch) *fp64_per_launch = kclass == 1 ? 2.0 * cells : 0.0;  // the FMA and the int64 conversion
  b->n_launch += reps + 1;
  return cudaGetLastError() == cudaSuccess ? SM_OK : bfail(b, SM_ECUDA, "kernel bench launch");
}

extern "C" int sm_batch_set_schedule(sm_batch *b, int shape, int grid_mult) {
  if (!b || shape < 0 || shape >= NSHAPES || grid_mult < 1 || grid_mult > 64) return SM_EINVAL;
  if (!b->arena) return bfail(b, SM_ESTATE, "no arena bound");
  b->gmult = grid_mult;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return build_lists(b, shape);
}

extern "C" int sm_batch_set_graphs(sm_batch *b, int enable) {
  if (!b) return SM_EINVAL;
  b->graphs = enable != 0;
  return SM_OK;
}

extern "C" int sm_batch_info(const sm_batch *b, long long *cells, int *levels_max, long long *launches) {
  if (!b) return SM_EINVAL;
  if (cells) *cells = b->cells64;
  if (levels_max) *levels_max = b->kmax + 1;
  if (launches) *launches = b->n_launch;
  return SM_OK;
}

extern "C" const char *sm_batch_last_error(const sm_batch *b) { return b ? b->err.c_str() : "null batch"; }
