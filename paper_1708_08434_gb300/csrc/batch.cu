// batch.cu -- many independent Poisson solves (Eq. 1 with constant
// permittivity, the 7-point operator of the octree solve) on uniform grids
// of uneven sizes, advanced together: the batched form.
//
// Every solve s has levels k = 0 (finest, N_s cells per side) .. K_s, with
// N halved while it is even and larger than 8; the coarsest grid (at most
// 16 per side) is solved exactly in FP64 by separable eigenbases.  All
// solves' tiles of one level index are one work list, processed by one
// grid-stride ("persistent") launch per level and phase.  The cycle is a
// correction-scheme V(nu1,nu2) in FP32 on the error equation inside a
// per-solve FP64 defect-correction loop (residual and accumulation in
// FP64); converged solves are masked out.  A whole batched solve is one
// CUDA graph with a device-side loop; tile shape and grid size are chosen
// by timing candidate configurations (sm_batch_tune).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sm_internal.cuh"

using namespace sm;

namespace {

constexpr int BMAXL = 8;          // levels per solve
constexpr int BMAXC = 16;         // coarsest grid side limit
constexpr int TILE_CELLS = 512;   // threads per tile
constexpr int NSHAPES = 4;
// candidate tile shapes (x, y, z), x fastest in memory
constexpr int SHAPES[NSHAPES][3] = {{8, 8, 8}, {16, 8, 4}, {32, 4, 4}, {32, 8, 2}};
constexpr int GRID_MULTS[3] = {2, 4, 8};

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
  if (bc.type[f]) return (homog ? T(0) : T(2.0 * bc.val[f])) - in;
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

// red-black Gauss-Seidel colour pass of level k on the error e
__global__ void __launch_bounds__(TILE_CELLS) k_bt_smooth(const int4 *__restrict__ tiles, int ntiles, int k,
                                                          int color, const BSolve *__restrict__ tab,
                                                          const unsigned char *__restrict__ active,
                                                          float *__restrict__ e, const float *__restrict__ f,
                                                          Bc bc, TileShape sh) {
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    int4 T = tiles[it];
    if (!active[T.x]) continue;
    int N = tab[T.x].N[k];
    int x, y, z;
    if (!tile_cell(T, sh, N, x, y, z) || ((x + y + z) & 1) != color) continue;
    float *ev = e + tab[T.x].off[k];
    long long i = gidx(N, x, y, z);
    float c = ev[i];
    float s = sum6(ev, N, x, y, z, c, bc, 1);
    ev[i] = (s - tab[T.x].h2f[k] * f[tab[T.x].off[k] + i]) * (1.0f / 6.0f);
  }
}

// coarse rhs of level k+1 = mean of the 8 fine residuals; coarse error = 0
__global__ void __launch_bounds__(TILE_CELLS) k_bt_restrict(const int4 *__restrict__ tiles, int ntiles, int k,
                                                            const BSolve *__restrict__ tab,
                                                            const unsigned char *__restrict__ active,
                                                            float *__restrict__ e, float *__restrict__ f, Bc bc,
                                                            TileShape sh) {
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
    e[S.off[k + 1] + ic] = 0.0f;
  }
}

// e_k += (c + c_sx + c_sy + c_sz)/4 from level k+1 (homogeneous walls)
__global__ void __launch_bounds__(TILE_CELLS) k_bt_prolong(const int4 *__restrict__ tiles, int ntiles, int k,
                                                           const BSolve *__restrict__ tab,
                                                           const unsigned char *__restrict__ active,
                                                           float *__restrict__ e, Bc bc, TileShape sh) {
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    int4 T = tiles[it];
    if (!active[T.x]) continue;
    const BSolve &S = tab[T.x];
    int Nf = S.N[k], Nc = S.N[k + 1];
    int x, y, z;
    if (!tile_cell(T, sh, Nf, x, y, z)) continue;
    const float *ec = e + S.off[k + 1];
    int C[3] = {x >> 1, y >> 1, z >> 1}, g[3] = {x, y, z};
    float c = ec[gidx(Nc, C[0], C[1], C[2])];
    float sum = c;
    for (int a = 0; a < 3; ++a) {
      int s = (g[a] & 1) ? 1 : -1;
      int q[3] = {C[0], C[1], C[2]};
      q[a] += s;
      if (q[a] < 0 || q[a] >= Nc) sum += wall(bc, 2 * a + (s > 0), c, 1);
      else sum += ec[gidx(Nc, q[0], q[1], q[2])];
    }
    e[S.off[k] + gidx(Nf, x, y, z)] += 0.25f * sum;
  }
}

// exact FP64 solve of the error equation on the coarsest grid of each
// listed solve (one block per solve): separable eigenbases per axis
__global__ void __launch_bounds__(512) k_bt_coarse(const int *__restrict__ solves, int k,
                                                   const BSolve *__restrict__ tab,
                                                   const unsigned char *__restrict__ active,
                                                   float *__restrict__ e, const float *__restrict__ f, Bc bc) {
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
  float *ev = e + S.off[k];
  for (int c = t; c < n3; c += blockDim.x) ev[c] = (float)x[c];
}

// FP64 outer residual on the finest grids: r = f - L phi (or of phi = 0
// when zero_phi), its max norm per solve, FP32 copy as the error
// equation's rhs and a zero initial error
__global__ void __launch_bounds__(TILE_CELLS) k_bt_outer(const int4 *__restrict__ tiles, int ntiles,
                                                         const BSolve *__restrict__ tab,
                                                         const unsigned char *__restrict__ active,
                                                         const double *__restrict__ phi,
                                                         const double *__restrict__ f64, float *__restrict__ f32,
                                                         float *__restrict__ e32, Bc bc, TileShape sh,
                                                         int zero_phi, unsigned long long *__restrict__ num) {
  __shared__ double red[16];
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    int4 T = tiles[it];
    if (!active[T.x]) continue;  // uniform per block
    const BSolve &S = tab[T.x];
    int N = S.N[0];
    int x, y, z;
    double r = 0.0;
    if (tile_cell(T, sh, N, x, y, z)) {
      long long i = gidx(N, x, y, z);
      const double *p = phi + S.off64;
      double c = zero_phi ? 0.0 : p[i];
      double s;
      if (zero_phi) {
        s = 0.0;
        int g[3] = {x, y, z};
        for (int fc = 0; fc < 6; ++fc) {
          int q = g[fc >> 1] + ((fc & 1) ? 1 : -1);
          if (q < 0 || q >= N) s += wall(bc, fc, 0.0, 0);
        }
      } else {
        s = sum6(p, N, x, y, z, c, bc, 0);
      }
      r = f64[S.off64 + i] - (s - 6.0 * c) * S.inv_h2;
      f32[S.off[0] + i] = (float)r;
      e32[S.off[0] + i] = 0.0f;
    }
    block_max_to(num + T.x, fabs(r), red);
    __syncthreads();
  }
}

// phi += e on the finest grids (FP64 accumulation of the FP32 correction)
__global__ void __launch_bounds__(TILE_CELLS) k_bt_add(const int4 *__restrict__ tiles, int ntiles,
                                                       const BSolve *__restrict__ tab,
                                                       const unsigned char *__restrict__ active,
                                                       double *__restrict__ phi, const float *__restrict__ e32,
                                                       TileShape sh) {
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    int4 T = tiles[it];
    if (!active[T.x]) continue;
    const BSolve &S = tab[T.x];
    int x, y, z;
    if (!tile_cell(T, sh, S.N[0], x, y, z)) continue;
    long long i = gidx(S.N[0], x, y, z);
    phi[S.off64 + i] += (double)e32[S.off[0] + i];
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
      st.den[s] = st.num[s];
      st.num[s] = 0;
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
  long long pool = 0, cells64 = 0;  // FP32 pool cells, finest cells
  size_t max_tiles = 0;             // capacity of the tile area (all lists)
  // arena
  char *arena = nullptr;
  BSolve *d_tab = nullptr;
  double *phi = nullptr, *f64 = nullptr;
  float *e32 = nullptr, *f32 = nullptr;
  int4 *d_tiles = nullptr;
  int *d_coarse = nullptr;
  unsigned long long *d_num = nullptr, *d_den = nullptr;
  double *d_rel = nullptr, *d_tolmax = nullptr;
  int *d_cycles = nullptr, *d_any = nullptr;
  unsigned char *d_active = nullptr;
  double *h_tolmax = nullptr;
  // current schedule
  int shape = 0, gmult = 4, sms = 148;
  std::vector<size_t> smooth_off, smooth_cnt, restr_off, restr_cnt;  // per level index
  std::vector<size_t> coarse_off, coarse_cnt;
  size_t fine_off = 0, fine_cnt = 0;  // level 0 of every solve (outer loop)
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
  long long pool = 0, c64 = 0;
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
    q.off64 = c64;
    c64 += (long long)N * N * N;
    kmax = std::max(kmax, k - 1);
  }
  // FP32 pool ordered by level index, then solve
  for (int k = 0; k <= kmax; ++k)
    for (int s = 0; s < n_solves; ++s)
      if (k < S[s].nlev) {
        S[s].off[k] = pool;
        pool += (long long)S[s].N[k] * S[s].N[k] * S[s].N[k];
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
  b->nu1 = nu1;
  b->nu2 = nu2;
  b->stream = (cudaStream_t)stream;
  b->solves = S;
  b->kmax = kmax;
  b->pool = pool;
  b->cells64 = c64;
  size_t mt = 0;
  for (int sh = 0; sh < NSHAPES; ++sh) {
    size_t t = 0;
    for (auto &q : S)
      for (int k = 0; k < q.nlev; ++k) t += (k == 0 ? 3 : 2) * tiles_of(q.N[k], sh);  // smooth, restrict, fine
    mt = std::max(mt, t);
  }
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
  size_t tab, phi, f64, e32, f32, tiles, coarse, num, den, rel, tolmax, cycles, any, active, total;
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
  L.phi = take(sizeof(double) * b->cells64);
  L.f64 = take(sizeof(double) * b->cells64);
  L.e32 = take(sizeof(float) * b->pool);
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
  L.total = t;
  return L;
}

extern "C" int sm_batch_arena_size(const sm_batch *b, size_t *bytes) {
  if (!b || !bytes) return SM_EINVAL;
  *bytes = blayout(b).total;
  return SM_OK;
}

// tile lists of one shape: per level index the smoothing/prolongation list
// (solves for which the level is not the coarsest) and the restriction
// target list (levels 1..coarsest); the coarse-solve list per level index
static int build_lists(sm_batch *b, int shape) {
  const int *sh = SHAPES[shape];
  std::vector<int4> all;
  b->smooth_off.assign(b->kmax + 1, 0);
  b->smooth_cnt.assign(b->kmax + 1, 0);
  b->restr_off.assign(b->kmax + 1, 0);
  b->restr_cnt.assign(b->kmax + 1, 0);
  auto push_level = [&](int k, bool restrict_list) {
    size_t start = all.size();
    for (int s = 0; s < b->n; ++s) {
      const BSolve &q = b->solves[s];
      bool take = restrict_list ? (k >= 1 && k < q.nlev) : (k < q.nlev - 1);
      if (!take) continue;
      int N = q.N[k];
      int nx = (N + sh[0] - 1) / sh[0], ny = (N + sh[1] - 1) / sh[1], nz = (N + sh[2] - 1) / sh[2];
      for (int tz = 0; tz < nz; ++tz)
        for (int ty = 0; ty < ny; ++ty)
          for (int tx = 0; tx < nx; ++tx) all.push_back(make_int4(s, tx, ty, tz));
    }
    return std::make_pair(start, all.size() - start);
  };
  for (int k = 0; k <= b->kmax; ++k) {
    auto a = push_level(k, false);
    b->smooth_off[k] = a.first;
    b->smooth_cnt[k] = a.second;
    auto r = push_level(k, true);
    b->restr_off[k] = r.first;
    b->restr_cnt[k] = r.second;
  }
  // finest grids of all solves, including those whose finest is the coarsest
  b->fine_off = all.size();
  for (int s = 0; s < b->n; ++s) {
    int N = b->solves[s].N[0];
    int nx = (N + sh[0] - 1) / sh[0], ny = (N + sh[1] - 1) / sh[1], nz = (N + sh[2] - 1) / sh[2];
    for (int tz = 0; tz < nz; ++tz)
      for (int ty = 0; ty < ny; ++ty)
        for (int tx = 0; tx < nx; ++tx) all.push_back(make_int4(s, tx, ty, tz));
  }
  b->fine_cnt = all.size() - b->fine_off;
  if (all.size() > b->max_tiles) return bfail(b, SM_ESTATE, "tile list capacity");
  std::vector<int> coarse;
  b->coarse_off.assign(b->kmax + 1, 0);
  b->coarse_cnt.assign(b->kmax + 1, 0);
  for (int k = 0; k <= b->kmax; ++k) {
    b->coarse_off[k] = coarse.size();
    for (int s = 0; s < b->n; ++s)
      if (b->solves[s].nlev - 1 == k) coarse.push_back(s);
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
  BCK(cudaMemsetAsync(a, 0, L.total, b->stream));
  BCK(cudaMemcpyAsync(b->d_tab, b->solves.data(), sizeof(BSolve) * b->n, cudaMemcpyHostToDevice, b->stream));
  return build_lists(b, 0);
}

extern "C" int sm_batch_destroy(sm_batch *b) {
  if (!b) return SM_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap2) cudaStreamDestroy(b->cap2);
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
  return {b->d_num, b->d_den, b->d_rel, b->d_cycles, b->d_active, b->d_any};
}

static int outer(sm_batch *b, int zero_phi) {
  size_t n0 = b->fine_cnt;
  k_bt_outer<<<grid_for(b, n0), TILE_CELLS, 0, b->stream>>>(b->d_tiles + b->fine_off, (int)n0, b->d_tab,
                                                            b->d_active, b->phi, b->f64, b->f32, b->e32, b->bc,
                                                            shape_of(b), zero_phi, b->d_num);
  ++b->n_launch;
  return cudaGetLastError() == cudaSuccess ? SM_OK : bfail(b, SM_ECUDA, "outer residual launch");
}

static int smooth_level(sm_batch *b, int k, int nu) {
  size_t n = b->smooth_cnt[k];
  if (!n) return SM_OK;
  for (int s = 0; s < nu; ++s)
    for (int color = 0; color < 2; ++color) {
      k_bt_smooth<<<grid_for(b, n), TILE_CELLS, 0, b->stream>>>(b->d_tiles + b->smooth_off[k], (int)n, k, color,
                                                                b->d_tab, b->d_active, b->e32, b->f32, b->bc,
                                                                shape_of(b));
      ++b->n_launch;
    }
  return SM_OK;
}

static size_t coarse_smem(int n) {
  return sizeof(double) * (2 * (size_t)n * n * n + 3 * BMAXC * BMAXC + 3 * BMAXC);
}

static int coarse_at_level(sm_batch *b, int k) {
  size_t nc = b->coarse_cnt[k];
  if (nc) {
    k_bt_coarse<<<(int)nc, 512, coarse_smem(BMAXC), b->stream>>>(b->d_coarse + b->coarse_off[k], k, b->d_tab,
                                                                b->d_active, b->e32, b->f32, b->bc);
    ++b->n_launch;
  }
  return SM_OK;
}

// correction-scheme V-cycle on the error equation of every active solve
static int bvcycle(sm_batch *b) {
  coarse_at_level(b, 0);  // solves whose finest grid is already the coarsest
  for (int k = 0; k < b->kmax; ++k) {
    smooth_level(b, k, b->nu1);
    size_t nr = b->restr_cnt[k + 1];
    if (nr) {
      k_bt_restrict<<<grid_for(b, nr), TILE_CELLS, 0, b->stream>>>(b->d_tiles + b->restr_off[k + 1], (int)nr, k,
                                                                   b->d_tab, b->d_active, b->e32, b->f32, b->bc,
                                                                   shape_of(b));
      ++b->n_launch;
    }
    coarse_at_level(b, k + 1);
  }
  for (int k = b->kmax - 1; k >= 0; --k) {
    size_t n = b->smooth_cnt[k];
    if (n) {
      k_bt_prolong<<<grid_for(b, n), TILE_CELLS, 0, b->stream>>>(b->d_tiles + b->smooth_off[k], (int)n, k,
                                                                 b->d_tab, b->d_active, b->e32, b->bc,
                                                                 shape_of(b));
      ++b->n_launch;
    }
    smooth_level(b, k, b->nu2);
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
      cudaMemsetAsync(b->d_active, 1, b->n, b->stream) != cudaSuccess)
    return bfail(b, SM_ECUDA, "memset");
  if ((st = outer(b, 1))) return st;
  k_bt_check<<<1, 256, 0, b->stream>>>(h, in_graph, b->n, bstate(b), 0, 0, b->d_tolmax);
  ++b->n_launch;
  if ((st = outer(b, 0))) return st;
  k_bt_check<<<1, 256, 0, b->stream>>>(h, in_graph, b->n, bstate(b), 1, 0, b->d_tolmax);
  ++b->n_launch;
  return cudaGetLastError() == cudaSuccess ? SM_OK : bfail(b, SM_ECUDA, "prefix launch");
}

// one correction of every active solve: V-cycle, phi += e, residual, check
static int body_step(sm_batch *b, cudaGraphConditionalHandle h, int in_graph) {
  int st;
  if ((st = bvcycle(b))) return st;
  size_t n0t = b->fine_cnt;
  k_bt_add<<<grid_for(b, n0t), TILE_CELLS, 0, b->stream>>>(b->d_tiles + b->fine_off, (int)n0t, b->d_tab,
                                                           b->d_active, b->phi, b->e32, shape_of(b));
  ++b->n_launch;
  if ((st = outer(b, 0))) return st;
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
  BCK(cudaFuncSetAttribute(k_bt_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)coarse_smem(BMAXC)));
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
    BCK(cudaFuncSetAttribute(k_bt_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)coarse_smem(BMAXC)));
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
      BCK(cudaMemsetAsync(b->phi, 0, sizeof(double) * b->cells64, b->stream));
      if ((st = run(b, 0.0, iters, nullptr))) return st;  // capture + warm-up
      BCK(cudaMemsetAsync(b->phi, 0, sizeof(double) * b->cells64, b->stream));
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
  BCK(cudaMemsetAsync(b->phi, 0, sizeof(double) * b->cells64, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (shape) *shape = bs;
  if (grid_mult) *grid_mult = bg;
  if (best_ms) *best_ms = best;
  return SM_OK;
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
