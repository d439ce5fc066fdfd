// sm_internal.cuh -- context layout and device helpers shared by the CUDA
// translation units of the library (octree, multigrid, fluid).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <utility>
#include <vector>

#include "sm_streamer.h"

namespace sm {

constexpr int NC = SM_BOX;         // cells per box side (Sec. 2.1.1)
constexpr int CELLS = NC * NC * NC;
constexpr int FACE = NC * NC;
constexpr int MAXL = SM_MAX_LEVELS;

// physical boundary description, passed by value to kernels
struct Bc {
  int type[6];      // 0 Neumann zero, 1 Dirichlet
  double val[6];
  double g2[6];     // 2 val, the Dirichlet ghost's constant part (filled by bc_finish)
  float g2f[6];     // the same rounded to FP32
};

// fill the derived constants of a boundary description (host side)
inline void bc_finish(Bc &bc) {
  for (int f = 0; f < 6; ++f) {
    bc.g2[f] = 2.0 * bc.val[f];
    bc.g2f[f] = (float)bc.g2[f];
  }
}

// 2 g of face f in the arithmetic type of a kernel (no FP64 work in FP32 kernels)
template <typename T>
__host__ __device__ __forceinline__ T bc_g2(const Bc &bc, int f);
template <>
__host__ __device__ __forceinline__ double bc_g2<double>(const Bc &bc, int f) {
  return bc.g2[f];
}
template <>
__host__ __device__ __forceinline__ float bc_g2<float>(const Bc &bc, int f) {
  return bc.g2f[f];
}

// per-level grid spacing tables, passed by value to kernels
struct LevelH {
  double h[MAXL], inv_h[MAXL], h2[MAXL], inv_h2[MAXL];
};

// transport-coefficient lookup table (device arrays)
struct Table {
  const double *mu, *diff, *alpha;
  const double *dmu, *ddiff, *dalpha;  // slopes t[i+1] - t[i]
  int n;
  double inv_de;    // (n-1)/e_max
  double hinv_de;   // (n-1)/(2 e_max): the index of the face value (e_L + e_R)/2 from e_L + e_R
  long long xmax;   // bit pattern of the double n - 1 (upper clamp, compared as an integer)
};

// kernel classes for sm_kernel_bench
enum KClass { K_SMOOTH = 0, K_PERSIST = 1, K_VCYCLE = 2, K_VCYCLE32 = 3, K_NCLASS = 4 };

}  // namespace sm

// an instantiated solve graph and the kernel launches it contains
struct sm_graph {
  cudaGraphExec_t exec = nullptr;
  long long prefix_launches = 0, body_launches = 0;
};

namespace sm {

}  // namespace sm

struct sm_ctx {
  sm_config cfg;
  sm_domain dom;
  int lbase = 0, lmax = 0;       // base level, finest allowed level
  int device = 0;
  cudaStream_t stream = nullptr;
  sm::Bc bc;
  sm::LevelH lh;

  // arena
  char *arena = nullptr;
  size_t arena_bytes = 0;

  // tables (device)
  int32_t *level = nullptr, *ijk = nullptr, *parent = nullptr, *child = nullptr,
          *nbr = nullptr, *nbr6 = nullptr, *leaf = nullptr;
  int32_t *cf_leaf = nullptr;  // leaf boxes with at least one refinement face (nbr6 == -2)
  uint64_t *morton = nullptr;
  int32_t *scan_a = nullptr, *scan_b = nullptr;  // [max_boxes] build scratch
  int32_t *dev_count = nullptr;                   // small device counters
  int8_t *dev_flags = nullptr;

  // fields (device) [max_boxes][512]
  double *phi = nullptr, *rhs = nullptr, *res = nullptr, *old = nullptr,
         *rho = nullptr, *emag = nullptr;
  double *nbuf[3] = {nullptr, nullptr, nullptr};  // electron density buffers
  double *ibuf[3] = {nullptr, nullptr, nullptr};  // ion density buffers
  int ncur = 0;                                   // current density buffer
  double *gh = nullptr;      // [max_boxes][6][64] coarse interpolation values
  // fixed-point potential of the FP64 solve and its rhs term -h^2 f / 6
  // (colour-split order within a box), and the refinement-face sums
  // 2c + c_t1 + c_t2, all in quanta of the solve
  long long *phx = nullptr, *gx = nullptr;                  // [max_boxes][512]
  long long *ghx = nullptr;                                 // [max_boxes][6][64]
  int fx_margin = 5;         // exponent margin of the fixed-point scale
  int rows_min = 2048;       // boxes of a level from which its fixed-point kernels work by rows
  // FP32 error-equation arrays of the mixed-precision solve
  float *e32 = nullptr, *f32 = nullptr, *old32 = nullptr;  // [max_boxes][512]
  float *gh32 = nullptr;                                    // [max_boxes][6][64]
  double *cflux = nullptr;   // [max_boxes][6][64] fine-side refinement fluxes
  double *basis = nullptr;   // level-0 eigenbasis: [3][64] vectors, [3][8] eigenvalues
  double *tab = nullptr;     // [6][4096] coefficient tables and their slopes
  unsigned long long *dscal = nullptr;  // device scalars (max reductions, flags)
  double *hist = nullptr;    // [SM_HIST] relative residual after each cycle of the last solve
  int tab_n = 0;
  double tab_emax = 0.0;

  // host mirrors
  int n_boxes = 0, n_levels = 0, n_leaves = 0, n_cf_leaves = 0;
  int level_off[SM_MAX_LEVELS + 1] = {0};
  int leaf_level_off[SM_MAX_LEVELS + 1] = {0};
  double *hscal = nullptr;   // pinned host scalars [SC_N], then a staged copy [SC_N]
  bool basis_ready = false;
  double den = 0.0;          // residual norm of phi == 0 (current rhs)

  // kernels launched so far (diagnostics)
  long long n_launch = 0;

  // per-solve metrics log (JSON lines), off unless a path was given
  FILE *mlog = nullptr;
  double mlog_peak = 0.0;               // HBM GB/s the line's fraction divides by (0: none)
  long long mlog_seq = 0;
  cudaEvent_t mlog_ev[2] = {nullptr, nullptr};
  std::vector<double> hhist;            // cycle history of the host-loop path

  // optional hooks around the solves of sm_advance_fluid (learned warm start)
  void *hook_obj = nullptr;
  int (*pre_solve)(void *, sm_ctx *) = nullptr;
  int (*post_solve)(void *, sm_ctx *) = nullptr;

  // captured solves (invalidated when the octree changes)
  bool graphs = true;
  bool pdl = true;  // programmatic dependent launch between level kernels
  // the next launch waits for full completion of its predecessor: set after
  // kernels that write the tables, which dependents read before their wait
  bool pdl_fence = false;
  bool persist = false;      // V-cycles as one persistent cooperative launch
  int persist_grid[2] = {0, 0};  // co-resident blocks of the FP64 / FP32 kernel
  cudaStream_t cap = nullptr, cap2 = nullptr;
  sm_graph g_solve, g_fmg, g_solve32, g_fmg32;

  std::string err;
};

// ----------------------------------------------------------------------
// host helpers
// ----------------------------------------------------------------------
int sm_fail(sm_ctx *ctx, int code, const char *fmt, ...);
int sm_cuda_check(sm_ctx *ctx, cudaError_t e, const char *what);
#define SM_CK(call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return sm_cuda_check(ctx, e_, #call);      \
  } while (0)
#define SM_CKL(what)                                                  \
  do {                                                                \
    cudaError_t e_ = cudaGetLastError();                              \
    if (e_ != cudaSuccess) return sm_cuda_check(ctx, e_, what);       \
  } while (0)

// device scalar slots (unsigned long long each)
enum {
  SC_NORM = 0,      // residual max (double bits)
  SC_DEN = 1,       // residual max of phi == 0
  SC_ADV = 2,       // dt: max sum |v|/dx
  SC_AD = 3,        // dt: max adv + 6 D/dx^2
  SC_DRT = 4,       // dt: max mu n_e
  SC_ERR = 5,       // consistency error flag
  SC_CYC = 6,       // V-cycles done by the device-side loop
  SC_REL = 7,       // relative residual after the last cycle (double bits)
  SC_TOL = 8,       // loop tolerance (double bits), set before a launch
  SC_MAXC = 9,      // loop cycle limit, set before a launch
  SC_PN0 = 10,      // residual max of the persistent loop, even passes
  SC_PN1 = 11,      // residual max of the persistent loop, odd passes
  SC_BAR = 12,      // grid barrier arrival counter of the persistent kernel
  SC_FXE = 16,      // fixed-point solve: exponent E of the quantum 2^(E - 1080)
  SC_FXI = 17,      // fixed-point solve: exponent bound of the inputs (reduction)
  SC_FXM = 18,      // fixed-point solve: margin added to the bound, set before a solve
  SC_FX2G = 19,     // fixed-point solve: 2g of the six faces in quanta (19 .. 24)
  SC_N = 32
};

// cycles of a solve whose relative residual the metrics log keeps
constexpr int SM_HIST = 64;

namespace sm {

// ----------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------
__device__ __forceinline__ int cidx(int i, int j, int k) { return i + NC * j + FACE * k; }

// index of a cell within a face of axis a: tangential coordinates
// u along (a+1)%3 and w along (a+2)%3
__device__ __forceinline__ int fcell(int a, int i, int j, int k) {
  return a == 0 ? (j + NC * k) : (a == 1 ? (k + NC * i) : (i + NC * j));
}

// wait for the predecessor grid of a programmatic dependent launch (a
// no-op for a normal launch)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Conversions between IEEE-754 binary64 and binary32 done with integer
// operations on the bit fields.  On this GPU the hardware conversion
// instructions share the narrow FP64 pipe, so FP64 kernels that convert
// every cell lose FP64 throughput to them (and a hardware fallback on a
// rare path is still issued for every cell once the compiler turns the
// branch into a select).  Every class -- normal, subnormal, zero, infinity,
// NaN -- is handled here; the results equal the hardware's bit for bit
// (checked by sm_check_conversions; NaNs compared as NaNs).
//
// binary64 bit pattern -> binary32, round to nearest, ties to even: the
// significand (with its hidden bit) is shifted right to the binary32
// position -- 29 bits for normal results, more for subnormal ones -- and
// rounded on the dropped bits; a carry into the exponent field is the
// correctly rounded result, up to the infinity encoding on overflow.
__device__ __forceinline__ float cvt_bits_f32_rn(unsigned long long b) {
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int fe = e - 1023 + 127;
  if (fe >= 1 && fe <= 254) {  // normal binary32 result
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    unsigned r = ((unsigned)fe << 23) | m;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(r | sign);
  }
  if (e == 0x7ff) {  // infinity or NaN (quiet, top payload bits kept)
    const unsigned long long frac = b & 0x000fffffffffffffull;
    return __uint_as_float(sign | (frac ? 0x7fc00000u | (unsigned)(frac >> 29) : 0x7f800000u));
  }
  if (fe > 254) return __uint_as_float(sign | 0x7f800000u);  // overflow
  if (e == 0) return __uint_as_float(sign);                    // binary64 zero or subnormal
  // subnormal or zero binary32 result: significand 1.f shifted by 29 + (1 - fe)
  const int ts = 30 - fe;
  if (ts > 54) return __uint_as_float(sign);
  const unsigned long long M = (b & 0x000fffffffffffffull) | (1ull << 52);
  const unsigned long long q = M >> ts, rem = M & ((1ull << ts) - 1ull), half = 1ull << (ts - 1);
  const unsigned r = (unsigned)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u);
  return __uint_as_float(sign | r);
}
__device__ __forceinline__ float cvt_f64_f32_rn(double d) {
  return cvt_bits_f32_rn((unsigned long long)__double_as_longlong(d));
}

// binary32 -> binary64 (exact): re-bias the exponent and widen the
// fraction; subnormals are normalised, infinities and NaNs keep their
// class (NaNs quiet)
__device__ __forceinline__ double cvt_f32_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, frac = u & 0x7fffffu;
  unsigned hi, lo;
  if (e != 0u && e != 255u) {
    hi = sign | ((e + 1023u - 127u) << 20) | (frac >> 3);
    lo = u << 29;
  } else if (e == 255u) {
    hi = sign | 0x7ff00000u | (frac ? 0x00080000u : 0u) | (frac >> 3);
    lo = frac << 29;
  } else if (frac == 0u) {
    hi = sign;
    lo = 0u;
  } else {  // subnormal: value frac * 2^-149; normalise the leading one to bit 23
    const int lz = __clz(frac) - 8;  // shifts that bring the leading one to bit 23
    const unsigned m = (frac << lz) & 0x7fffffu;
    hi = sign | ((unsigned)(1023 - 126 - lz) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Exact stencil sums in 64-bit fixed point (integer pipe).  A finite
// binary64 value with biased exponent field e <= E is mapped to the nearest
// multiple of 2^(E - 1080), ties away from zero, as a signed integer: its
// 53-bit significand (hidden bit included; subnormals use e = 1) shifted by
// e - E + 5, so |result| < 2^58 and sums of twelve such values cannot
// overflow.  The rounding error is at most 2^(E - 1081), i.e. 2^-58 of the
// largest value of that exponent.
//
// Branch-free: M = significand * 2^5 (< 2^58), then a right shift by
// rs = E - e >= 0; for rs >= 1 the last dropped bit is kept, incremented
// and shifted out, which rounds half away from zero (shift counts above 63
// give 0, as the result must).
__device__ __forceinline__ long long fix_of_bits(unsigned long long b, int E) {
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned long long M = ((b & 0x000fffffffffffffull) | (e ? (1ull << 52) : 0ull)) << 5;
  const int rs = E - (e ? e : 1);
  const unsigned long long t1 = M >> min(max(rs - 1, 0), 63);
  const unsigned long long u = rs > 0 ? (t1 + 1ull) >> 1 : t1;
  return (long long)((hi >> 31) ? 0ull - u : u);
}

// biased exponent field of a binary64 value (0 for zero and subnormals,
// 0x7ff for infinities and NaNs)
__device__ __forceinline__ unsigned expo_of(double d) {
  return ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;
}

// atomic max of a non-negative double through its bit pattern
__device__ __forceinline__ void atomic_max_pos(unsigned long long *slot, double v) {
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// block-wide max (blockDim.x multiple of 32, <= 1024) pushed to a slot
__device__ __forceinline__ void block_max_to(unsigned long long *slot, double v, double *red) {
  v = warp_max(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    double x = lane < nw ? red[lane] : 0.0;
    x = warp_max(x);
    if (lane == 0) atomic_max_pos(slot, x);
  }
}

// Ghost value of a potential-type variable across face f of box b next to
// interior cell (i,j,k) holding `inner`: same-level neighbour cell, physical
// boundary (Dirichlet 2g - inner or -inner when homogeneous; Neumann
// inner), or refinement boundary inner/3 + 2 phihat/3 with the stored
// coarse interpolation phihat.
template <typename T>
__device__ __forceinline__ T pot_ghost(const T *v, const int32_t *__restrict__ nbr6, const T *gh, int b, int f,
                                       int i, int j, int k, T inner, const Bc &bc, int homog) {
  int nb = __ldg(nbr6 + 6 * b + f);
  int a = f >> 1;
  if (nb >= 0) {
    int c[3] = {i, j, k};
    c[a] = (f & 1) ? 0 : NC - 1;
    return v[(size_t)nb * CELLS + cidx(c[0], c[1], c[2])];
  }
  if (nb == -1) {
    if (bc.type[f]) return (homog ? T(0) : bc_g2<T>(bc, f)) - inner;
    return inner;
  }
  return inner * T(1.0 / 3.0) + T(2.0 / 3.0) * gh[(size_t)(6 * b + f) * FACE + fcell(a, i, j, k)];
}

// sum of the six neighbours of cell (i,j,k) of box b (ghosts as above)
template <typename T>
__device__ __forceinline__ T nb_sum(const T *v, const int32_t *__restrict__ nbr6, const T *gh, int b, int i,
                                    int j, int k, T ctr, const Bc &bc, int homog) {
  const T *p = v + (size_t)b * CELLS;
  int c = cidx(i, j, k);
  T s = (i > 0) ? p[c - 1] : pot_ghost(v, nbr6, gh, b, 0, i, j, k, ctr, bc, homog);
  s += (i < NC - 1) ? p[c + 1] : pot_ghost(v, nbr6, gh, b, 1, i, j, k, ctr, bc, homog);
  s += (j > 0) ? p[c - NC] : pot_ghost(v, nbr6, gh, b, 2, i, j, k, ctr, bc, homog);
  s += (j < NC - 1) ? p[c + NC] : pot_ghost(v, nbr6, gh, b, 3, i, j, k, ctr, bc, homog);
  s += (k > 0) ? p[c - FACE] : pot_ghost(v, nbr6, gh, b, 4, i, j, k, ctr, bc, homog);
  s += (k < NC - 1) ? p[c + FACE] : pot_ghost(v, nbr6, gh, b, 5, i, j, k, ctr, bc, homog);
  return s;
}

}  // namespace sm

// Launch with programmatic dependent launch when enabled: the kernel may
// be scheduled while its predecessor drains; every kernel launched this way
// starts with sm::pdl_wait(), so it still reads nothing before the
// predecessor has finished and its writes are visible.
template <typename... KArgs, typename... Args>
inline cudaError_t sm_launch(sm_ctx *ctx, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (ctx->pdl && !ctx->pdl_fence) ? 1 : 0;
  ctx->pdl_fence = false;
  ++ctx->n_launch;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// entry points implemented in the other translation units
int sm_mg_fill_cf(sm_ctx *ctx, double *var, int level, int homog);
int sm_fill_all_cf(sm_ctx *ctx, double *var);
int sm_exclusive_scan(sm_ctx *ctx, const int32_t *in, int32_t *out, int n);
int sm_restrict_pair(sm_ctx *ctx, double *a, double *b);
void sm_drop_graphs(sm_ctx *ctx);
int sm_rebuild_leaves(sm_ctx *ctx);
int sm_build_neighbours(sm_ctx *ctx, int level);
