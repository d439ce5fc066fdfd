// cnn.cu -- learned warm start for the warm-started Poisson solves of the
// time step (build form, not in the paper): a small per-box 3D
// convolutional network predicts the change of the potential of a box from
// its right-hand side and its previous potential.  It is trained on the GPU
// by the kernels below on pairs the solver itself produces during a run;
// the multigrid residual decides (a prediction is kept only if it
// lowers the relative residual) and iterates to the same tolerance.
//
// Network per 8^3 box (weights BF16, activations rounded to BF16 as the
// next layer's operands, FP32 accumulation, biases FP32):
//   input  X: 2 channels on the 10^3 box-with-ghosts region, the FP64
//          residual h^2 (f - L phi_prev) divided by the box scale s and the
//          normalised right-hand side h^2 f
//   conv 3^3 valid 2->16, ReLU;  conv 3^3 same 16->16, ReLU (5th-generation
//          tensor cores: tcgen05.mma with the accumulator in tensor memory);
//   conv 3^3 same 16->1 -> delta on 8^3;  prediction phi += s * delta.
// Training: mean squared error against (phi_solved - phi_prev)/s (clipped),
// Adam on FP32 master weights, gradients reduced in a fixed order
// (deterministic).  The backward pass of layer 2 (its data and weight
// gradients) runs on the tensor cores too, on dL/dz2 split into three BF16
// terms whose sum is its FP32 value, so the gradient keeps FP32 accuracy.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sm_internal.cuh"
#include "sm_nvtx.h"

using namespace sm;

int sm_rel_residual_now(sm_ctx *ctx, double *rel);

namespace {

constexpr int NW1 = 16 * 2 * 27, NW2 = 16 * 16 * 27, NW3 = 16 * 27;
constexpr int O_W1 = 0, O_B1 = NW1, O_W2 = O_B1 + 16, O_B2 = O_W2 + NW2, O_W3 = O_B2 + 16, O_B3 = O_W3 + NW3;
constexpr int NP = O_B3 + 1;  // 8241 parameters
constexpr int NPOS = 1000;    // 10^3 positions of a box with one ghost layer
constexpr int CT = 256;       // threads per CTA (inference, sample preparation)
constexpr int TT = 512;       // threads per CTA of the training kernel (one CTA per SM)
constexpr int MAX_DEBUG = 16;

typedef __nv_bfloat16 bf16;

// voxel v = x + 8y + 64z of the box -> position in the 10^3 region
__device__ __forceinline__ int Pos(int v) { return ((v & 7) + 1) + 10 * (((v >> 3) & 7) + 1) + 100 * ((v >> 6) + 1); }
// tap t = (dx+1) + 3(dy+1) + 9(dz+1) -> position offset
__device__ __forceinline__ int Off(int t) { return (t % 3 - 1) + 10 * ((t / 3) % 3 - 1) + 100 * (t / 9 - 1); }
__device__ __forceinline__ float bf(bf16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float rbf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// weights as one CTA uses them
struct NetS {
  float w1[NW1];      // [t][co][ci], BF16 values (32 per tap)
  float b1[16];
  bf16 w2[27 * 256];  // per tap four 8x8 core matrices [t][ci/8][co/8][co%8][ci%8] (B operand)
  float b2[16];
  float w3[NW3];      // [t][ci], BF16 values (16 per tap)
  float b3;
};

// Layer-1 activations as a tensor-core operand.  The 10^3 region (one ghost
// layer) is stored row by row, R = y + 10 z in padded coordinates, each row
// as 10 slots of channels 0-7 followed by 10 slots of channels 8-15 (a slot
// is one position, 8 BF16 = 16 bytes): slot x + 10 half + 20 R.  Two rows
// past the region take the reads of the discarded rows of the last tile.
constexpr int A1_ROWS = 102, A1_SLOTS = 20 * A1_ROWS;
__device__ __forceinline__ int A1S(int x, int half, int R) { return x + 10 * half + 20 * R; }
// slot of voxel v (channels 0-7), and the slot offset of tap t
__device__ __forceinline__ int VS(int v) { return A1S((v & 7) + 1, 0, ((v >> 3) & 7) + 1 + 10 * ((v >> 6) + 1)); }
__device__ __forceinline__ int SOff(int t) { return (t % 3 - 1) + 20 * ((t / 3) % 3 - 1) + 200 * (t / 9 - 1); }

struct FwdS {
  bf16 a1[A1_SLOTS * 8];  // zero outside the box interior
  bf16 x[NPOS * 2];       // [pos][ci]
  bf16 a2[1024 * 16];     // a1's layout (100 rows), zero outside the box interior; training
                          // reuses the space for dL/dz1 ([16][512] FP32)
  float out[512];
};

// dL/dz2 of training as a tensor-core operand: every value as the sum of
// three BF16 terms (exact for an FP32 value), stored like a1 with the three
// terms side by side in a row: slot x + 10 half + 20 term + 60 R.
constexpr int D2_ROWS = 102, D2_SLOTS = 60 * D2_ROWS;
__device__ __forceinline__ int D2S(int x, int term, int half, int R) { return x + 10 * half + 20 * term + 60 * R; }


// ---- tcgen05: 5th-generation tensor cores, accumulator in tensor memory ----
//
// Layer 2 (16 -> 16 channels, 3^3 taps) and both of its gradients are
// implicit GEMMs on shifted views of the operands above, with no im2col
// copy.  The shared-memory operands use the no-swizzle canonical layouts: a
// core matrix is 8 rows of 16 contiguous bytes; K-major rows run along M
// (or N) and hold 8 K values, MN-major rows run along K and hold 8 M (or N)
// values; SBO is the byte stride between 8-wide M (N) groups, LBO between
// 8-deep K groups.
//
// forward          D[v][co] = sum_{t,ci} a1[pos(v) + off(t)][ci] W2[co][ci][t].
//   An M = 128 tile is 16 consecutive rows R of 8 voxels along x; rows with
//   y = -1 or 8 (two per z plane) fall inside the tile and are discarded:
//   5 tiles (R = 11 + 16j) cover the 64 rows of the box.  A of tap t: K-major
//   view of a1 from the tile's first row shifted by off(t), SBO 320 (one
//   row), LBO 160 (channels 8-15).  B: W2 of the tap as four 8x8 core
//   matrices (LBO 256: ci 8-15; SBO 128: co 8-15).  27 MMAs (K = 16) per tile
//   into 16 columns.
// backward-data    dA1[q][ci] = sum_{t,co} dZ2[q - off(t)][co] W2[co][ci][t]:
//   the same tiles over dZ2 shifted by -off(t) (SBO 960, LBO 160), one MMA per
//   BF16 term (start + 320 term); B: W2 transposed (w2t).  81 MMAs per tile.
// backward-weight  dW2[co][ci][t] = sum_v dZ2[v][co] a1[pos(v) + off(t)][ci]:
//   voxels are K.  One accumulator per (dy, dz): M = 128 rows (g, c) of an
//   MN-major view of a1 with SBO 16, so group g starts one position further
//   along the row: g = 0-2 are channels 0-7 at dx = -1, 0, 1 and g = 10-12
//   channels 8-15 at dx = -1, 0, 1 (the other ten groups are discarded); K
//   rows are the 8 voxels of an x row, LBO 320 the next row.  B: MN-major
//   view of dZ2, N = 48 = (term, half, co) with SBO 160, LBO 960.  32 MMAs
//   (two x rows each) per box, accumulated over all boxes of the CTA.
// Tensor memory of training: columns 0-79 the forward and backward-data
// tiles, 80 + 48c the backward-weight accumulator of c = (dy+1) + 3(dz+1).
constexpr int TC_TILES = 5, FWD_COLS = 128, TRAIN_COLS = 512, WG_COL0 = 80;
constexpr uint32_t TC_KIND = (1u << 4)    // D: FP32
                             | (1u << 7)  // A: BF16
                             | (1u << 10);  // B: BF16
constexpr uint32_t TC_IDESC = TC_KIND | ((16u >> 3) << 17) | ((128u >> 4) << 24);  // N 16, M 128, K-major
constexpr uint32_t TC_IDESC_WG = TC_KIND | (1u << 15) | (1u << 16)               // A and B MN-major
                                 | ((48u >> 3) << 17) | ((128u >> 4) << 24);      // N 48, M 128
constexpr long long TC_SPIN = 1ll << 22;  // mbarrier polls before giving up (far beyond a box's work)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor without swizzle (descriptor version 1)
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase of an mbarrier; false when the polls ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (long long i = 0; i < TC_SPIN; ++i)
    if (mbar_try(mbar, phase)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Tensor-memory and mbarrier state of a CTA that runs layer 2 on tcgen05:
// warp 0 allocates the columns at the start and frees them at the end.
struct TcState {
  uint32_t taddr;   // tensor-memory address of the allocation (lane 0, first column)
  uint32_t mbar;    // shared address of the MMA-completion mbarrier
  uint32_t phase;   // parity of the next completion
  uint32_t ncols;   // allocated columns (a power of two >= 32)
  unsigned *err;    // device error word: bit 0 = an MMA wait ran out
};

__device__ void tc_begin(TcState &tc, uint64_t *mbar, uint32_t *slot, unsigned *err, uint32_t ncols) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(TC_TILES) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc.taddr = *slot;
  tc.mbar = smem_u32(mbar);
  tc.phase = 0;
  tc.ncols = ncols;
  tc.err = err;
}

__device__ void tc_end(const TcState &tc) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.taddr), "r"(tc.ncols)
                 : "memory");
}

// Bounded wait of every thread for the MMAs of the current phase; false
// (and bit 0 of *tc.err set) when it ran out, after a second bounded wait
// for the MMAs in flight
__device__ bool tc_wait_all(TcState &tc) {
  const bool ok = mbar_wait(tc.mbar, tc.phase);
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) atomicOr(tc.err, 1u);
    mbar_wait(tc.mbar, tc.phase);
    return false;
  }
  tc.phase ^= 1;
  tc_fence_after();
  return true;
}

// position of W2[co][ci][t] in NetS::w2
__device__ __forceinline__ int W2i(int t, int co, int ci) {
  return t * 256 + (ci >> 3) * 128 + (co >> 3) * 64 + (co & 7) * 8 + (ci & 7);
}

__device__ void load_net(NetS &N, const float *__restrict__ w) {
  for (int i = threadIdx.x; i < NW1; i += blockDim.x) N.w1[(i % 27) * 32 + i / 27] = rbf(w[O_W1 + i]);
  for (int i = threadIdx.x; i < NW3; i += blockDim.x) N.w3[(i % 27) * 16 + i / 27] = rbf(w[O_W3 + i]);
  for (int i = threadIdx.x; i < 27 * 256; i += blockDim.x) {
    int t = i / 256, co = (i / 16) % 16, ci = i % 16;
    N.w2[W2i(t, co, ci)] = __float2bfloat16_rn(w[O_W2 + (co * 16 + ci) * 27 + t]);
  }
  if (threadIdx.x < 16) {
    N.b1[threadIdx.x] = w[O_B1 + threadIdx.x];
    N.b2[threadIdx.x] = w[O_B2 + threadIdx.x];
  }
  if (threadIdx.x == 0) N.b3 = w[O_B3];
}

// the 16 channels at slot s of an array in a1's layout, as floats
__device__ __forceinline__ void row16(const bf16 *a, int s, float (&v)[16]) {
  const uint4 u0 = *reinterpret_cast<const uint4 *>(a + 8 * s), u1 = *reinterpret_cast<const uint4 *>(a + 8 * (s + 10));
  const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[i]));
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

// 16 floats (16-byte aligned)
__device__ __forceinline__ void w16(const float *p, float (&v)[16]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 f = reinterpret_cast<const float4 *>(p)[i];
    v[4 * i] = f.x;
    v[4 * i + 1] = f.y;
    v[4 * i + 2] = f.z;
    v[4 * i + 3] = f.w;
  }
}

// sum over the 32 lanes of a warp (butterfly: every lane gets the total)
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ void zero16(void *p, int bytes) {
  uint4 *q = reinterpret_cast<uint4 *>(p);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) q[i] = make_uint4(0u, 0u, 0u, 0u);
}

__device__ void zero_acts(FwdS &F) {
  zero16(F.a1, sizeof(F.a1));
  zero16(F.a2, sizeof(F.a2));
}

// Forward pass of one box whose input is already in F.x.  Debug pointers
// (per box [16][512] / [512], may be null) receive z1, a1, z2, a2.  False
// (and bit 0 of *tc.err set) when the tensor cores' completion wait ran out;
// the caller then stops.
template <int NT>  // threads of the block: 512 / NT voxels per thread
__device__ bool forward_box(const NetS &N, FwdS &F, TcState &tc, float *z1d, float *a1d, float *z2d,
                            float *a2d) {
  constexpr int VPT = 512 / NT;
  const int t = threadIdx.x;
  // layer 1: valid 3^3 conv 2 -> 16 on CUDA cores, voxels t + r NT per
  // thread (the 32 weights of a tap are broadcast 16-byte loads)
  {
    int pv[VPT];
    float acc[VPT][16];
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
      pv[r] = Pos(t + r * NT);
#pragma unroll
      for (int co = 0; co < 16; ++co) acc[r][co] = N.b1[co];
    }
    for (int tp = 0; tp < 27; ++tp) {
      const int off = Off(tp);
      float2 xv[VPT];
#pragma unroll
      for (int r = 0; r < VPT; ++r)
        xv[r] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(F.x + 2 * (pv[r] + off)));
      const float4 *wt = reinterpret_cast<const float4 *>(N.w1 + 32 * tp);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 wv = wt[k];  // W1[2k][0], W1[2k][1], W1[2k+1][0], W1[2k+1][1]
#pragma unroll
        for (int r = 0; r < VPT; ++r) {
          acc[r][2 * k] += wv.x * xv[r].x + wv.y * xv[r].y;
          acc[r][2 * k + 1] += wv.z * xv[r].x + wv.w * xv[r].y;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
      const int v = t + r * NT;
      bf16 *a1v = F.a1 + 8 * A1S((v & 7) + 1, 0, ((v >> 3) & 7) + 1 + 10 * ((v >> 6) + 1));
#pragma unroll
      for (int co = 0; co < 16; ++co) {
        bf16 a = __float2bfloat16_rn(fmaxf(acc[r][co], 0.0f));
        a1v[co < 8 ? co : 80 + (co - 8)] = a;
        if (z1d) {
          z1d[co * 512 + v] = acc[r][co];
          a1d[co * 512 + v] = bf(a);
        }
      }
    }
  }
  // the tensor cores read a1 (and the weights) through the async proxy
  async_proxy_fence();
  tc_fence_before();
  __syncthreads();
  // layer 2 on tcgen05 (the tiling is described above TC_TILES): lane 0 of
  // warp j issues the 27 MMAs of tile j and commits them to the mbarrier
  if ((t & 31) == 0 && (t >> 5) < TC_TILES) {
    tc_fence_after();
    const int j = t >> 5, R0 = 11 + 16 * j;
    const uint32_t a0 = smem_u32(F.a1), b0 = smem_u32(N.w2);
    for (int tp = 0; tp < 27; ++tp) {
      const int dx = tp % 3 - 1, dy = (tp / 3) % 3 - 1, dz = tp / 9 - 1;
      tc_mma(tc.taddr + 16 * j, tc_desc(a0 + 16 * A1S(1 + dx, 0, R0 + dy + 10 * dz), 160, 320),
             tc_desc(b0 + 512 * tp, 256, 128), TC_IDESC, tp > 0);
    }
    tc_commit(tc.mbar);
  }
  if (!tc_wait_all(tc)) return false;
  {
    // warp w reads lanes 32 (w % 4) .. +31 of the tiles j = w / 4 + k (NT / 128)
    const int warp = t >> 5, lane = t & 31, q = warp & 3;
    const int r = 32 * q + lane;  // row of the tile
    for (int j = warp >> 2; j < TC_TILES; j += NT / 128) {
      float acc[16];
      tc_ld16(tc.taddr + ((uint32_t)(32 * q) << 16) + 16 * j, acc);
      const int R = 11 + 16 * j + (r >> 3), x = r & 7, y = R % 10 - 1, z = R / 10 - 1;
      if (y < 0 || y > 7 || z < 0 || z > 7) continue;  // a padding row of the tile
      const int v = x + 8 * y + 64 * z;
      uint32_t pk[8];
#pragma unroll
      for (int co = 0; co < 16; co += 2) {
        float z0 = acc[co] + N.b2[co], z1 = acc[co + 1] + N.b2[co + 1];
        __nv_bfloat162 a2 = __floats2bfloat162_rn(fmaxf(z0, 0.0f), fmaxf(z1, 0.0f));
        pk[co >> 1] = *reinterpret_cast<const uint32_t *>(&a2);
        if (z2d) {
          z2d[co * 512 + v] = z0;
          z2d[(co + 1) * 512 + v] = z1;
          a2d[co * 512 + v] = __low2float(a2);
          a2d[(co + 1) * 512 + v] = __high2float(a2);
        }
      }
      const int s = A1S(x + 1, 0, R);
      *reinterpret_cast<uint4 *>(F.a2 + 8 * s) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      *reinterpret_cast<uint4 *>(F.a2 + 8 * (s + 10)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
  }
  tc_fence_before();
  __syncthreads();
  // layer 3: same 3^3 conv 16 -> 1 on CUDA cores, voxels t + r NT per
  // thread (a2 rows and the 16 weights of a tap as 16-byte loads)
  {
    int sv[VPT];
    float o[VPT];
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
      sv[r] = VS(t + r * NT);
      o[r] = N.b3;
    }
    for (int tp = 0; tp < 27; ++tp) {
      const int so = SOff(tp);
      float wv[16];
      w16(N.w3 + 16 * tp, wv);
#pragma unroll
      for (int r = 0; r < VPT; ++r) {
        float a[16];
        row16(F.a2, sv[r] + so, a);
#pragma unroll
        for (int ci = 0; ci < 16; ++ci) o[r] += wv[ci] * a[ci];
      }
    }
#pragma unroll
    for (int r = 0; r < VPT; ++r) F.out[t + r * NT] = o[r];
  }
  __syncthreads();
  return true;
}

__device__ void load_input(FwdS &F, const bf16 *__restrict__ X) {
  const uint32_t *src = reinterpret_cast<const uint32_t *>(X);
  uint32_t *dst = reinterpret_cast<uint32_t *>(F.x);
  for (int i = threadIdx.x; i < NPOS; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// inference / debug forward over boxes [0, n) of X; out [n][512]
__global__ void __launch_bounds__(CT) k_cnn_forward(const bf16 *__restrict__ X, int n, const float *__restrict__ w,
                                                    float *__restrict__ out, float *__restrict__ dbg,
                                                    unsigned *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  NetS &N = *reinterpret_cast<NetS *>(smraw);
  FwdS &F = *reinterpret_cast<FwdS *>(smraw + ((sizeof(NetS) + 127) & ~(size_t)127));
  TcState tc;
  tc_begin(tc, &mbar, &tslot, err, FWD_COLS);
  load_net(N, w);
  zero_acts(F);
  __syncthreads();
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    load_input(F, X + (size_t)b * NPOS * 2);
    float *d = (dbg && b < MAX_DEBUG) ? dbg + (size_t)b * 4 * 16 * 512 : nullptr;
    if (!forward_box<CT>(N, F, tc, d, d ? d + 8192 : nullptr, d ? d + 16384 : nullptr, d ? d + 24576 : nullptr))
      break;
    for (int v = threadIdx.x; v < 512; v += blockDim.x) out[(size_t)b * 512 + v] = F.out[v];
    __syncthreads();
  }
  tc_end(tc);
}

// ---- training: forward + backward per box, per-CTA partial gradients ----

// gradient entries kept in shared memory, in parameter order without W2
// (whose gradient accumulates in tensor memory)
constexpr int G_W1 = 0, G_B1 = NW1, G_B2 = G_B1 + 16, G_W3 = G_B2 + 16, G_B3 = G_W3 + NW3, NG = G_B3 + 1;
__device__ __forceinline__ int g_to_param(int i) { return i < G_B2 ? i : i + NW2; }

struct TrainS {
  bf16 w2t[27 * 256];     // backward-data B operand: [t][co/8][ci/8][ci%8][co%8]
  bf16 d2[D2_SLOTS * 8];  // dL/dz2 as three BF16 terms, zero outside the box interior
  float g3[512];          // dL/d out
  float grad[NG];
  float part[TT];         // per-thread partial sums of the bias gradients
  float red[TT / 32];
};

static_assert(offsetof(FwdS, a1) % 16 == 0 && offsetof(TrainS, d2) % 16 == 0 && offsetof(TrainS, w2t) % 16 == 0,
              "tensor-core operands start on 16-byte boundaries");
static_assert(((sizeof(NetS) + 127) & ~(size_t)127) + ((sizeof(FwdS) + 127) & ~(size_t)127) + sizeof(TrainS) <=
                  227 * 1024,
              "training shared memory");
static_assert(sizeof(NetS) == 19140 && sizeof(FwdS) == 71456 && sizeof(TrainS) == 121220,
              "layout the operand ranges were checked against");

// position of W2[co][ci][t] in TrainS::w2t (ci is the N index, co the K index)
__device__ __forceinline__ int W2Ti(int t, int co, int ci) {
  return t * 256 + (co >> 3) * 128 + (ci >> 3) * 64 + (ci & 7) * 8 + (co & 7);
}

__global__ void __launch_bounds__(TT, 1) k_cnn_train(const bf16 *__restrict__ X, const float *__restrict__ target,
                                                  const int *__restrict__ ids, int n, float inv_count,
                                                  const float *__restrict__ w, float *__restrict__ partial,
                                                  float *__restrict__ loss_partial, unsigned *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  const size_t o1 = (sizeof(NetS) + 127) & ~(size_t)127, o2 = o1 + ((sizeof(FwdS) + 127) & ~(size_t)127);
  NetS &N = *reinterpret_cast<NetS *>(smraw);
  FwdS &F = *reinterpret_cast<FwdS *>(smraw + o1);
  TrainS &S = *reinterpret_cast<TrainS *>(smraw + o2);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  TcState tc;
  tc_begin(tc, &mbar, &tslot, err, TRAIN_COLS);
  load_net(N, w);
  for (int i = t; i < 27 * 256; i += TT) {
    const int tp = i / 256, co = (i / 16) % 16, ci = i % 16;
    S.w2t[W2Ti(tp, co, ci)] = __float2bfloat16_rn(w[O_W2 + (co * 16 + ci) * 27 + tp]);
  }
  zero_acts(F);
  zero16(S.d2, sizeof(S.d2));
  for (int i = t; i < NG; i += TT) S.grad[i] = 0.0f;
  float my_loss = 0.0f;
  bool wg_acc = false;  // the backward-weight accumulators hold a sum
  __syncthreads();
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int s = ids[it];
    load_input(F, X + (size_t)s * NPOS * 2);
    if (!forward_box<TT>(N, F, tc, nullptr, nullptr, nullptr, nullptr)) break;
    const float *tg = target + (size_t)s * 512;
    for (int v = t; v < 512; v += TT) {
      const float e = F.out[v] - tg[v];
      my_loss += e * e * inv_count;
      S.g3[v] = 2.0f * inv_count * e;
    }
    __syncthreads();
    // layer 3 weights: warp w takes taps w, w + 8, ...; lane l the voxels
    // l + 32k, whose sums the warp then adds (fixed order); bias: warp 7
    for (int tp = warp; tp < 27; tp += TT / 32) {
      const int so = SOff(tp);
      float acc[16];
#pragma unroll
      for (int ci = 0; ci < 16; ++ci) acc[ci] = 0.0f;
      for (int v = lane; v < 512; v += 32) {
        float a[16];
        row16(F.a2, VS(v) + so, a);
        const float g = S.g3[v];
#pragma unroll
        for (int ci = 0; ci < 16; ++ci) acc[ci] += a[ci] * g;
      }
#pragma unroll
      for (int ci = 0; ci < 16; ++ci) acc[ci] = warp_sum(acc[ci]);
      if (lane == 0)
#pragma unroll
        for (int ci = 0; ci < 16; ++ci) S.grad[G_W3 + ci * 27 + tp] += acc[ci];
    }
    if (warp == TT / 32 - 1) {
      float acc = 0.0f;
      for (int v = lane; v < 512; v += 32) acc += S.g3[v];
      acc = warp_sum(acc);
      if (lane == 0) S.grad[G_B3] += acc;
    }
    // dL/dz2[u][c] = relu'(a2[u][c]) sum_t W3[c][t] g3[u - d_t] for voxels
    // t + r TT, stored as three BF16 terms h0 + h1 + h2 equal to the
    // FP32 value (each remainder is exact in FP32 and the last has at most 8
    // significant bits)
    {
      float bsum[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) bsum[c] = 0.0f;
#pragma unroll 1
      for (int r = 0; r < 512 / TT; ++r) {
        const int u = t + r * TT, ux = u & 7, uy = (u >> 3) & 7, uz = u >> 6;
        float acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.0f;
        for (int tp = 0; tp < 27; ++tp) {
          const int vx = ux - (tp % 3 - 1), vy = uy - ((tp / 3) % 3 - 1), vz = uz - (tp / 9 - 1);
          if (vx < 0 || vx > 7 || vy < 0 || vy > 7 || vz < 0 || vz > 7) continue;
          const float g = S.g3[vx + 8 * vy + 64 * vz];
          float wv[16];
          w16(N.w3 + 16 * tp, wv);
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[c] += wv[c] * g;
        }
        float a2v[16];
        row16(F.a2, VS(u), a2v);
        const int R = (uy + 1) + 10 * (uz + 1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t t0[4], t1[4], t2[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            bf16 hv[3][2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int c = 8 * h + 2 * k + e;
              const float d = a2v[c] > 0.0f ? acc[c] : 0.0f;
              bsum[c] += d;
              hv[0][e] = __float2bfloat16_rn(d);
              const float r1 = d - bf(hv[0][e]);
              hv[1][e] = __float2bfloat16_rn(r1);
              hv[2][e] = __float2bfloat16_rn(r1 - bf(hv[1][e]));
            }
            t0[k] = pack2(hv[0][0], hv[0][1]);
            t1[k] = pack2(hv[1][0], hv[1][1]);
            t2[k] = pack2(hv[2][0], hv[2][1]);
          }
          *reinterpret_cast<uint4 *>(S.d2 + 8 * D2S(ux + 1, 0, h, R)) = make_uint4(t0[0], t0[1], t0[2], t0[3]);
          *reinterpret_cast<uint4 *>(S.d2 + 8 * D2S(ux + 1, 1, h, R)) = make_uint4(t1[0], t1[1], t1[2], t1[3]);
          *reinterpret_cast<uint4 *>(S.d2 + 8 * D2S(ux + 1, 2, h, R)) = make_uint4(t2[0], t2[1], t2[2], t2[3]);
        }
      }
      // layer-2 bias: per warp, then the warps in order (below)
#pragma unroll
      for (int c = 0; c < 16; ++c) bsum[c] = warp_sum(bsum[c]);
      if (lane == 0)
#pragma unroll
        for (int c = 0; c < 16; ++c) S.part[16 * warp + c] = bsum[c];
    }
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    // backward-data and backward-weight of layer 2 on tcgen05 (described
    // above TC_TILES): lane 0 of warp j issues backward-data tile j and the
    // backward-weight accumulators j and j + 5, then commits
    if ((t & 31) == 0 && (t >> 5) < TC_TILES) {
      tc_fence_after();
      const int j = t >> 5, R0 = 11 + 16 * j;
      const uint32_t a0 = smem_u32(F.a1), d0 = smem_u32(S.d2), b0 = smem_u32(S.w2t);
      for (int tp = 0; tp < 27; ++tp) {
        const int dx = tp % 3 - 1, dy = (tp / 3) % 3 - 1, dz = tp / 9 - 1;
        const uint64_t bd = tc_desc(b0 + 512 * tp, 256, 128);
        for (int m = 0; m < 3; ++m)
          tc_mma(tc.taddr + 16 * j, tc_desc(d0 + 16 * D2S(1 - dx, m, 0, R0 - dy - 10 * dz), 160, 960), bd,
                 TC_IDESC, tp > 0 || m > 0);
      }
      for (int c = j; c < 9; c += TC_TILES) {
        const int dy = c % 3 - 1, dz = c / 3 - 1;
        for (int p = 0; p < 32; ++p) {
          const int R = (2 * (p & 3) + 1) + 10 * ((p >> 2) + 1);  // x rows y = 2 (p % 4), +1 of plane z = p / 4
          tc_mma(tc.taddr + WG_COL0 + 48 * c, tc_desc(a0 + 16 * A1S(0, 0, R + dy + 10 * dz), 320, 16),
                 tc_desc(d0 + 16 * D2S(1, 0, 0, R), 960, 160), TC_IDESC_WG, wg_acc || p > 0);
        }
      }
      tc_commit(tc.mbar);
    }
    wg_acc = true;
    if (t < 16) {
      float acc = 0.0f;
      for (int i = 0; i < TT / 32; ++i) acc += S.part[16 * i + t];
      S.grad[G_B2 + t] += acc;
    }
    if (!tc_wait_all(tc)) break;
    // dL/dz1 = relu'(a1) dA1 on the interior voxels, into the a2 space
    // ([channel][voxel]: the lanes of a warp touch consecutive words)
    {
      float *d1 = reinterpret_cast<float *>(F.a2);
      const int q = warp & 3, r = 32 * q + lane;
      for (int j = warp >> 2; j < TC_TILES; j += TT / 128) {
        float acc[16];
        tc_ld16(tc.taddr + ((uint32_t)(32 * q) << 16) + 16 * j, acc);
        const int R = 11 + 16 * j + (r >> 3), x = r & 7, y = R % 10 - 1, z = R / 10 - 1;
        if (y < 0 || y > 7 || z < 0 || z > 7) continue;
        const int v = x + 8 * y + 64 * z;
        const bf16 *a1v = F.a1 + 8 * A1S(x + 1, 0, R);
#pragma unroll
        for (int ci = 0; ci < 16; ++ci) d1[ci * 512 + v] = bf(a1v[ci < 8 ? ci : 80 + (ci - 8)]) > 0.0f ? acc[ci] : 0.0f;
      }
    }
    tc_fence_before();
    __syncthreads();
    // layer 1 weights (valid conv on the 10^3 input): warp w takes taps
    // w, w + 8, ...; lane l the voxels l + 32k, whose sums the warp adds
    {
      const float *d1 = reinterpret_cast<const float *>(F.a2);
      for (int tp = warp; tp < 27; tp += TT / 32) {
        const int off = Off(tp);
        float acc[32];  // [co][ci]
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
        for (int v = lane; v < 512; v += 32) {
          const float2 xv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(F.x + 2 * (Pos(v) + off)));
          float dv[16];
#pragma unroll
          for (int co = 0; co < 16; ++co) dv[co] = d1[co * 512 + v];
#pragma unroll
          for (int co = 0; co < 16; ++co) {
            acc[2 * co] += xv.x * dv[co];
            acc[2 * co + 1] += xv.y * dv[co];
          }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = warp_sum(acc[i]);
        if (lane == 0)
#pragma unroll
          for (int i = 0; i < 32; ++i) S.grad[G_W1 + i * 27 + tp] += acc[i];
      }
      // layer-1 bias: thread t sums channel t / G over the voxels t % G +
      // G i (G = TT / 16), then the G partial sums of a channel in order
      {
        constexpr int G = TT / 16;
        const int c = t / G, g = t % G;
        float acc = 0.0f;
        for (int v = g; v < 512; v += G) acc += d1[c * 512 + v];
        S.part[t] = acc;
      }
      __syncthreads();
      if (t < 16) {
        float acc = 0.0f;
        for (int g = 0; g < TT / 16; ++g) acc += S.part[(TT / 16) * t + g];
        S.grad[G_B1 + t] += acc;
      }
    }
    __syncthreads();
    zero16(F.a2, sizeof(F.a2));  // layer 3 of the next box reads zeros outside the interior
    __syncthreads();
  }
  float *dst = partial + (size_t)blockIdx.x * NP;
  // W2 gradient: the three terms' columns of the useful rows of each
  // backward-weight accumulator (lanes 0-23 and 80-103: warps 0, 2, 3)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  {
    const int q = warp & 3;
    if (warp < 4 && q != 1) {
      const int L = 32 * q + lane, g = L >> 3, c8 = L & 7;
      const bool use = g <= 2 || (g >= 10 && g <= 12);
      const int ci = g <= 2 ? c8 : 8 + c8, dx = g <= 2 ? g - 1 : g - 11;
      for (int c = 0; c < 9; ++c) {
        float sum[16];
#pragma unroll
        for (int co = 0; co < 16; ++co) sum[co] = 0.0f;
        if (wg_acc) {
          for (int m = 0; m < 3; ++m) {
            float v[16];
            tc_ld16(tc.taddr + ((uint32_t)(32 * q) << 16) + WG_COL0 + 48 * c + 16 * m, v);
#pragma unroll
            for (int co = 0; co < 16; ++co) sum[co] += v[co];
          }
        }
        if (use) {
          const int tp = (dx + 1) + 3 * c;
#pragma unroll
          for (int co = 0; co < 16; ++co) dst[O_W2 + (co * 16 + ci) * 27 + tp] = sum[co];
        }
      }
    }
  }
  tc_end(tc);
  for (int i = t; i < NG; i += TT) dst[g_to_param(i)] = S.grad[i];
  // this CTA's loss
  float v = my_loss;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((t & 31) == 0) S.red[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    float s = 0.0f;
    for (int i = 0; i < TT / 32; ++i) s += S.red[i];
    loss_partial[blockIdx.x] = s;
  }
}

// gradient = sum of the CTA partials in CTA order (deterministic)
__global__ void k_cnn_reduce(const float *__restrict__ partial, int nblk, float *__restrict__ grad,
                             const float *__restrict__ loss_partial, float *__restrict__ loss) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NP) {
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * NP + i];
    grad[i] = s;
  }
  if (i == 0) {
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += loss_partial[b];
    *loss = s;
  }
}

// Adam on the FP32 master weights (bias-corrected moments)
__global__ void k_cnn_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ g, float lr, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float gi = g[i];
  float mi = b1 * m[i] + (1.0f - b1) * gi;
  float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Inputs of the listed boxes from the solver state, on the 10^3 box-with-
// ghosts positions (positions outside the box repeat the nearest interior
// cell): channel 0 = h^2 r with r = f - L phi the FP64 residual of the
// plain warm start, divided by the box scale s = max |h^2 r|; channel 1 =
// h^2 f divided by its own box maximum (where the charge is).  The residual
// is formed in FP64 before any rounding: it is ~1e-3 of f, below BF16
// resolution, so the network could not form it from rounded inputs.
__global__ void __launch_bounds__(CT) k_cnn_gather(const int *__restrict__ boxes, int n,
                                                   const double *__restrict__ phi, const double *__restrict__ rhs,
                                                   const double *__restrict__ gh, const int32_t *__restrict__ nbr6,
                                                   const int32_t *__restrict__ level,
                                                   const int32_t *__restrict__ child, Bc bc, LevelH lh,
                                                   bf16 *__restrict__ X, float *__restrict__ scale,
                                                   double *__restrict__ phi_prev, int slot0) {
  __shared__ double vr[CELLS], vf[CELLS], red[2][CT / 32];
  int b = boxes[blockIdx.x], slot = slot0 + blockIdx.x;
  int l = level[b];
  double h2 = lh.h2[l], inv_h2 = lh.inv_h2[l];
  const double *pb = phi + (size_t)b * CELLS, *fb = rhs + (size_t)b * CELLS;
  double mr = 0.0, mf = 0.0;
  for (int v = threadIdx.x; v < CELLS; v += CT) {
    double p = pb[v];
    double sum = nb_sum(phi, nbr6, gh, b, v & 7, (v >> 3) & 7, v >> 6, p, bc, 0);
    double r = fb[v] - (sum - 6.0 * p) * inv_h2;
    vr[v] = h2 * r;
    vf[v] = h2 * fb[v];
    mr = fmax(mr, fabs(vr[v]));
    mf = fmax(mf, fabs(vf[v]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mf = fmax(mf, __shfl_xor_sync(0xffffffffu, mf, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = mr;
    red[1][threadIdx.x >> 5] = mf;
  }
  __syncthreads();
  double sr = 0.0, sf = 0.0;
  for (int i = 0; i < CT / 32; ++i) {
    sr = fmax(sr, red[0][i]);
    sf = fmax(sf, red[1][i]);
  }
  double ir = sr > 0.0 ? 1.0 / sr : 0.0, iff = sf > 0.0 ? 1.0 / sf : 0.0;
  bf16 *xo = X + (size_t)slot * NPOS * 2;
  for (int q = threadIdx.x; q < NPOS; q += CT) {
    int cx = min(max(q % 10 - 1, 0), NC - 1), cy = min(max((q / 10) % 10 - 1, 0), NC - 1),
        cz = min(max(q / 100 - 1, 0), NC - 1);
    int v = cidx(cx, cy, cz);
    xo[2 * q] = __float2bfloat16_rn((float)(vr[v] * ir));
    xo[2 * q + 1] = __float2bfloat16_rn((float)(vf[v] * iff));
  }
  if (threadIdx.x == 0) scale[slot] = (float)sr;
  if (phi_prev)  // indexed by position in the box list
    for (int v = threadIdx.x; v < CELLS; v += CT) phi_prev[(size_t)blockIdx.x * CELLS + v] = pb[v];
}

// training target (phi_new - phi_prev) / s of recorded boxes, clipped to
// +-8: a box whose change is mostly driven by charge elsewhere cannot be
// predicted from its own residual and is taught a bounded correction
__global__ void k_cnn_target(const int *__restrict__ boxes, int n, const double *__restrict__ phi,
                             const double *__restrict__ phi_prev, const float *__restrict__ scale,
                             float *__restrict__ target, int slot0) {
  int i = blockIdx.x, slot = slot0 + i, b = boxes[i];
  double s = (double)scale[slot];
  for (int v = threadIdx.x; v < CELLS; v += blockDim.x) {
    double d = phi[(size_t)b * CELLS + v] - phi_prev[(size_t)i * CELLS + v];
    double t = s > 0.0 ? d / s : 0.0;
    target[(size_t)slot * CELLS + v] = (float)fmin(8.0, fmax(-8.0, t));
  }
}

// phi += s * w * prediction on the listed boxes; with taper, w falls from
// 1 in the 4^3 core to 3/4 and 1/4 on the two outer cell layers per axis
// (so neighbouring boxes' independent predictions do not meet in jumps)
__device__ __forceinline__ double taper1(int i) { return i == 0 || i == 7 ? 0.25 : (i == 1 || i == 6 ? 0.75 : 1.0); }

__global__ void k_cnn_apply(const int *__restrict__ boxes, int n, const float *__restrict__ out,
                            const float *__restrict__ scale, double *__restrict__ phi, int taper) {
  int i = blockIdx.x, b = boxes[i];
  for (int v = threadIdx.x; v < CELLS; v += blockDim.x) {
    double w = taper ? taper1(v & 7) * taper1((v >> 3) & 7) * taper1(v >> 6) : 1.0;
    phi[(size_t)b * CELLS + v] += w * (double)scale[i] * (double)out[(size_t)i * CELLS + v];
  }
}

size_t fwd_smem() { return ((sizeof(NetS) + 127) & ~(size_t)127) + ((sizeof(FwdS) + 127) & ~(size_t)127); }
size_t train_smem() { return fwd_smem() + sizeof(TrainS); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct sm_cnn {
  cudaStream_t stream = nullptr;
  int max_samples = 0, max_boxes = 0, sms = 148;
  int n_samples = 0;
  char *arena = nullptr;
  float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *partial = nullptr, *lossp = nullptr,
        *loss = nullptr;
  unsigned *derr = nullptr;     // device error word of the network kernels
  bf16 *X = nullptr;            // samples [max_samples][1000][2]
  float *target = nullptr;      // [max_samples][512]
  float *scale = nullptr;       // [max_samples]
  double *phi_prev = nullptr;   // [max_boxes][512] boxes of the pending record
  bf16 *Xp = nullptr;           // prediction inputs [max_boxes][1000][2]
  float *out = nullptr, *sc_p = nullptr;  // prediction outputs and scales
  float *dbg = nullptr;         // [MAX_DEBUG][4][16][512]
  int *ids = nullptr, *boxes = nullptr;
  int adam_step = 0;
  // attached solver
  int mode = 0, stride = 1, per_solve = 0, taper = 0;
  double accept = 1.0;  // keep a prediction when rel_cnn < accept * rel_plain
  std::vector<int> pending;     // boxes recorded by the last pre-solve hook
  int pending_slot = 0;
  long long predictions = 0, kept = 0;
  double last_rel_plain = 0.0, last_rel_cnn = 0.0;
  std::string err;
};

static int cfail(sm_cnn *c, int code, const char *msg) {
  if (c) c->err = msg;
  return code;
}
#define CCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return SM_ECUDA;                                                     \
    }                                                                      \
  } while (0)

struct CLayout {
  size_t w, m, v, grad, partial, lossp, loss, derr, X, target, scale, phi_prev, Xp, out, sc_p, dbg, ids, boxes,
      total;
};

static CLayout clayout(int max_samples, int max_boxes, int sms) {
  CLayout L;
  size_t t = 0;
  auto take = [&](size_t bytes) {
    size_t at = t;
    t = (t + bytes + 255) & ~(size_t)255;
    return at;
  };
  L.w = take(4 * NP);
  L.m = take(4 * NP);
  L.v = take(4 * NP);
  L.grad = take(4 * NP);
  L.partial = take(4 * (size_t)NP * sms);
  L.lossp = take(4 * (size_t)sms);
  L.loss = take(4);
  L.derr = take(4);
  L.X = take(2 * (size_t)NPOS * 2 * max_samples);
  L.target = take(4 * (size_t)512 * max_samples);
  L.scale = take(4 * (size_t)max_samples);
  L.phi_prev = take(8 * (size_t)512 * max_boxes);
  L.Xp = take(2 * (size_t)NPOS * 2 * max_boxes);
  L.out = take(4 * (size_t)512 * max_boxes);
  L.sc_p = take(4 * (size_t)max_boxes);
  L.dbg = take(4 * (size_t)MAX_DEBUG * 4 * 16 * 512);
  L.ids = take(4 * (size_t)max_samples);
  L.boxes = take(4 * (size_t)max_boxes);
  L.total = t;
  return L;
}

extern "C" int sm_cnn_create(sm_cnn **out, int max_samples, int max_boxes, void *stream) {
  if (!out || max_samples < MAX_DEBUG || max_boxes < 1) return SM_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return SM_ECUDA;
  }
  sm_cnn *c = new sm_cnn();
  c->stream = (cudaStream_t)stream;
  c->max_samples = max_samples;
  c->max_boxes = max_boxes;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  *out = c;
  return SM_OK;
}

extern "C" int sm_cnn_destroy(sm_cnn *c) {
  delete c;
  return SM_OK;
}

extern "C" int sm_cnn_arena_size(const sm_cnn *c, size_t *bytes) {
  if (!c || !bytes) return SM_EINVAL;
  *bytes = clayout(c->max_samples, c->max_boxes, c->sms).total;
  return SM_OK;
}

extern "C" int sm_cnn_bind_arena(sm_cnn *c, void *dev_ptr, size_t bytes) {
  if (!c || !dev_ptr) return SM_EINVAL;
  CLayout L = clayout(c->max_samples, c->max_boxes, c->sms);
  if (bytes < L.total) return cfail(c, SM_ENOMEM, "arena too small");
  if (((uintptr_t)dev_ptr & 255) != 0) return cfail(c, SM_EINVAL, "arena not 256-byte aligned");
  char *a = (char *)dev_ptr;
  c->arena = a;
  c->w = (float *)(a + L.w);
  c->m = (float *)(a + L.m);
  c->v = (float *)(a + L.v);
  c->grad = (float *)(a + L.grad);
  c->partial = (float *)(a + L.partial);
  c->lossp = (float *)(a + L.lossp);
  c->loss = (float *)(a + L.loss);
  c->derr = (unsigned *)(a + L.derr);
  c->X = (bf16 *)(a + L.X);
  c->target = (float *)(a + L.target);
  c->scale = (float *)(a + L.scale);
  c->phi_prev = (double *)(a + L.phi_prev);
  c->Xp = (bf16 *)(a + L.Xp);
  c->out = (float *)(a + L.out);
  c->sc_p = (float *)(a + L.sc_p);
  c->dbg = (float *)(a + L.dbg);
  c->ids = (int *)(a + L.ids);
  c->boxes = (int *)(a + L.boxes);
  CCK(cudaMemsetAsync(a, 0, L.total, c->stream));
  CCK(cudaFuncSetAttribute(k_cnn_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem()));
  CCK(cudaFuncSetAttribute(k_cnn_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem()));
  c->n_samples = 0;
  c->adam_step = 0;
  return SM_OK;
}

extern "C" int sm_cnn_set_params(sm_cnn *c, const float *host, int n) {
  if (!c || !host || n != NP || !c->arena) return SM_EINVAL;
  CCK(cudaMemcpyAsync(c->w, host, 4 * NP, cudaMemcpyHostToDevice, c->stream));
  CCK(cudaMemsetAsync(c->m, 0, 4 * NP, c->stream));
  CCK(cudaMemsetAsync(c->v, 0, 4 * NP, c->stream));
  CCK(cudaStreamSynchronize(c->stream));
  c->adam_step = 0;
  return SM_OK;
}

extern "C" int sm_cnn_get_params(sm_cnn *c, float *host, int n) {
  if (!c || !host || n != NP || !c->arena) return SM_EINVAL;
  CCK(cudaMemcpyAsync(host, c->w, 4 * NP, cudaMemcpyDeviceToHost, c->stream));
  CCK(cudaStreamSynchronize(c->stream));
  return SM_OK;
}

// synchronise and read the network kernels' error word (cleared after
// reading): a tensor-core completion wait that ran out is SM_ETIMEOUT
static int check_derr(sm_cnn *c) {
  unsigned e = 0;
  CCK(cudaMemcpyAsync(&e, c->derr, 4, cudaMemcpyDeviceToHost, c->stream));
  CCK(cudaStreamSynchronize(c->stream));
  if (e) {
    CCK(cudaMemsetAsync(c->derr, 0, 4, c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    return cfail(c, SM_ETIMEOUT, "tensor-core completion wait ran out");
  }
  return SM_OK;
}

// forward of n explicit inputs (host [n][1000][2] floats, rounded to BF16
// on upload); out [n][512] and optional per-layer activations of the first
// min(n, 16) boxes ([n][4][16][512]: z1, a1, z2, a2)
extern "C" int sm_cnn_forward(sm_cnn *c, const float *x_host, int n, float *out_host, float *acts_host) {
  SM_RANGE();
  if (!c || !x_host || !out_host || n < 1 || n > c->max_boxes || !c->arena) return SM_EINVAL;
  std::vector<bf16> xb((size_t)n * NPOS * 2);
  for (size_t i = 0; i < xb.size(); ++i) xb[i] = __float2bfloat16_rn(x_host[i]);
  CCK(cudaMemcpyAsync(c->Xp, xb.data(), 2 * xb.size(), cudaMemcpyHostToDevice, c->stream));
  int grid = std::min(n, 4 * c->sms);
  k_cnn_forward<<<grid, CT, fwd_smem(), c->stream>>>(c->Xp, n, c->w, c->out, acts_host ? c->dbg : nullptr,
                                                     c->derr);
  CCK(cudaGetLastError());
  CCK(cudaMemcpyAsync(out_host, c->out, 4 * (size_t)512 * n, cudaMemcpyDeviceToHost, c->stream));
  if (acts_host)
    CCK(cudaMemcpyAsync(acts_host, c->dbg, 4 * (size_t)std::min(n, MAX_DEBUG) * 4 * 16 * 512,
                        cudaMemcpyDeviceToHost, c->stream));
  return check_derr(c);
}

static int grad_step(sm_cnn *c, int n, const int *ids_host) {
  CCK(cudaMemcpyAsync(c->ids, ids_host, 4 * (size_t)n, cudaMemcpyHostToDevice, c->stream));
  int nblk = std::min(n, c->sms);
  k_cnn_train<<<nblk, TT, train_smem(), c->stream>>>(c->X, c->target, c->ids, n, 1.0f / (512.0f * n), c->w,
                                                     c->partial, c->lossp, c->derr);
  k_cnn_reduce<<<(NP + 255) / 256, 256, 0, c->stream>>>(c->partial, nblk, c->grad, c->lossp, c->loss);
  CCK(cudaGetLastError());
  return SM_OK;
}

static int adam(sm_cnn *c, float lr) {
  ++c->adam_step;
  float c1 = 1.0f - powf(0.9f, (float)c->adam_step), c2 = 1.0f - powf(0.999f, (float)c->adam_step);
  k_cnn_adam<<<(NP + 255) / 256, 256, 0, c->stream>>>(c->w, c->m, c->v, c->grad, lr, c1, c2);
  CCK(cudaGetLastError());
  return SM_OK;
}

// gradient of the mean squared error over n explicit (input, target)
// pairs (host [n][1000][2] and [n][512]); overwrites sample slots 0..n-1
extern "C" int sm_cnn_gradient(sm_cnn *c, const float *x_host, const float *t_host, int n, float *grad_host,
                               float *loss) {
  if (!c || !x_host || !t_host || !grad_host || n < 1 || n > c->max_samples || !c->arena) return SM_EINVAL;
  std::vector<bf16> xb((size_t)n * NPOS * 2);
  for (size_t i = 0; i < xb.size(); ++i) xb[i] = __float2bfloat16_rn(x_host[i]);
  CCK(cudaMemcpyAsync(c->X, xb.data(), 2 * xb.size(), cudaMemcpyHostToDevice, c->stream));
  CCK(cudaMemcpyAsync(c->target, t_host, 4 * (size_t)512 * n, cudaMemcpyHostToDevice, c->stream));
  std::vector<int> ids(n);
  for (int i = 0; i < n; ++i) ids[i] = i;
  int st = grad_step(c, n, ids.data());
  if (st) return st;
  CCK(cudaMemcpyAsync(grad_host, c->grad, 4 * NP, cudaMemcpyDeviceToHost, c->stream));
  float l = 0.0f;
  CCK(cudaMemcpyAsync(&l, c->loss, 4, cudaMemcpyDeviceToHost, c->stream));
  if ((st = check_derr(c))) return st;
  if (loss) *loss = l;
  c->n_samples = 0;
  return SM_OK;
}

// explicit (input, target) pairs as the recorded samples
extern "C" int sm_cnn_load_samples(sm_cnn *c, const float *x_host, const float *t_host, int n) {
  if (!c || !x_host || !t_host || n < 1 || n > c->max_samples || !c->arena) return SM_EINVAL;
  std::vector<bf16> xb((size_t)n * NPOS * 2);
  for (size_t i = 0; i < xb.size(); ++i) xb[i] = __float2bfloat16_rn(x_host[i]);
  CCK(cudaMemcpyAsync(c->X, xb.data(), 2 * xb.size(), cudaMemcpyHostToDevice, c->stream));
  CCK(cudaMemcpyAsync(c->target, t_host, 4 * (size_t)512 * n, cudaMemcpyHostToDevice, c->stream));
  CCK(cudaStreamSynchronize(c->stream));
  c->n_samples = n;
  return SM_OK;
}

// one Adam step with an explicit gradient (host [NP])
extern "C" int sm_cnn_adam_step(sm_cnn *c, const float *grad_host, float lr) {
  if (!c || !grad_host || !c->arena) return SM_EINVAL;
  CCK(cudaMemcpyAsync(c->grad, grad_host, 4 * NP, cudaMemcpyHostToDevice, c->stream));
  int st = adam(c, lr);
  if (st) return st;
  CCK(cudaStreamSynchronize(c->stream));
  return SM_OK;
}

static uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// epochs over the recorded samples in minibatches, Adam after each; the
// sample order of each epoch is a seeded shuffle (SplitMix64 keys).
// Out: mean loss of the last epoch.
extern "C" int sm_cnn_train(sm_cnn *c, int epochs, int batch, float lr, unsigned long long seed, float *loss) {
  SM_RANGE();
  if (!c || epochs < 1 || batch < 1 || !c->arena) return SM_EINVAL;
  if (c->n_samples < 1) return cfail(c, SM_ESTATE, "no recorded samples");
  int n = c->n_samples;
  std::vector<int> order(n);
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    std::vector<std::pair<uint64_t, int>> key(n);
    for (int i = 0; i < n; ++i) key[i] = {splitmix(seed ^ ((uint64_t)ep << 32) ^ (uint64_t)i), i};
    std::sort(key.begin(), key.end());
    for (int i = 0; i < n; ++i) order[i] = key[i].second;
    double acc = 0.0;
    int nb = 0;
    for (int s = 0; s < n; s += batch) {
      int k = std::min(batch, n - s);
      int st = grad_step(c, k, order.data() + s);
      if (st) return st;
      if ((st = adam(c, lr))) return st;
      float l = 0.0f;
      CCK(cudaMemcpyAsync(&l, c->loss, 4, cudaMemcpyDeviceToHost, c->stream));
      if ((st = check_derr(c))) return st;
      acc += l;
      ++nb;
    }
    last = acc / nb;
  }
  if (loss) *loss = (float)last;
  return SM_OK;
}

// Average duration of one launch over the first n recorded samples: kind 0
// the forward kernel (inference), kind 1 a training gradient pass (forward,
// backward, partial gradients, reduction).  FLOPs per launch from the
// network's model: 16416 per voxel forward (layers of 1728, 13824 and 864),
// twice that backward; tensor-core FLOPs: those of the MMAs issued,
// discarded tile rows included.
extern "C" int sm_cnn_kernel_bench(sm_cnn *c, int kind, int n, int reps, double *us_per_launch, double *flops,
                                   double *tensor_flops) {
  if (!c || !c->arena || (kind != 0 && kind != 1) || n < 1 || reps < 1) return SM_EINVAL;
  if (n > c->n_samples) return cfail(c, SM_ESTATE, "fewer recorded samples than requested");
  if (kind == 0 && n > c->max_boxes) return SM_EINVAL;
  std::vector<int> ids(n);
  for (int i = 0; i < n; ++i) ids[i] = i;
  CCK(cudaMemcpyAsync(c->ids, ids.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, c->stream));
  auto launch = [&]() -> int {
    if (kind == 0) {
      k_cnn_forward<<<std::min(n, 4 * c->sms), CT, fwd_smem(), c->stream>>>(c->X, n, c->w, c->out, nullptr,
                                                                            c->derr);
      CCK(cudaGetLastError());
      return SM_OK;
    }
    return grad_step(c, n, ids.data());
  };
  int st = launch();  // warm-up
  if (st) return st;
  cudaEvent_t a, b;
  CCK(cudaEventCreate(&a));
  CCK(cudaEventCreate(&b));
  CCK(cudaEventRecord(a, c->stream));
  for (int r = 0; r < reps && !st; ++r) st = launch();
  CCK(cudaEventRecord(b, c->stream));
  CCK(cudaEventSynchronize(b));
  float ms = 0.f;
  CCK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st) return st;
  if ((st = check_derr(c))) return st;
  // tensor-core work per box: forward 135 MMAs of 128 x 16 x 16; training
  // adds backward-data (405 of 128 x 16 x 16) and backward-weight (288 of
  // 128 x 48 x 16)
  const double fwd = 16416.0 * 512.0 * n, mma16 = 2.0 * 128 * 16 * 16, mma48 = 2.0 * 128 * 48 * 16;
  const double tc = kind == 0 ? 135.0 * mma16 * n : (540.0 * mma16 + 288.0 * mma48) * n;
  if (us_per_launch) *us_per_launch = 1e3 * ms / reps;
  if (flops) *flops = kind == 0 ? fwd : 3.0 * fwd;
  if (tensor_flops) *tensor_flops = tc;
  return SM_OK;
}

// ---- coupling to a solver ---------------------------------------------------

// leaf boxes of the two finest levels, every stride-th, at most per_solve
static int sample_boxes(sm_cnn *c, sm_ctx *ctx, std::vector<int> &boxes) {
  boxes.clear();
  int lo = ctx->n_levels >= 2 ? ctx->leaf_level_off[ctx->n_levels - 2] : 0;
  int hi = ctx->n_leaves;
  std::vector<int32_t> leaf(hi - lo);
  if (hi > lo)
    CCK(cudaMemcpyAsync(leaf.data(), ctx->leaf + lo, 4 * (size_t)(hi - lo), cudaMemcpyDeviceToHost, ctx->stream));
  CCK(cudaStreamSynchronize(ctx->stream));
  for (size_t i = 0; i < leaf.size() && (int)boxes.size() < c->per_solve; i += c->stride) boxes.push_back(leaf[i]);
  return SM_OK;
}

static int cnn_pre_solve(void *obj, sm_ctx *ctx) {
  sm_cnn *c = (sm_cnn *)obj;
  int st = sm_fill_all_cf(ctx, ctx->phi);
  if (st) return st;
  if (c->mode == 1) {  // record inputs and the previous potential
    std::vector<int> boxes;
    if ((st = sample_boxes(c, ctx, boxes))) return st;
    int k = std::min((int)boxes.size(), c->max_samples - c->n_samples);
    c->pending.assign(boxes.begin(), boxes.begin() + std::max(k, 0));
    c->pending_slot = c->n_samples;
    if (k <= 0) return SM_OK;
    CCK(cudaMemcpyAsync(c->boxes, boxes.data(), 4 * (size_t)k, cudaMemcpyHostToDevice, ctx->stream));
    k_cnn_gather<<<k, CT, 0, ctx->stream>>>(c->boxes, k, ctx->phi, ctx->rhs, ctx->gh, ctx->nbr6, ctx->level,
                                            ctx->child, ctx->bc, ctx->lh, c->X, c->scale, c->phi_prev,
                                            c->pending_slot);
    ++ctx->n_launch;
    CCK(cudaGetLastError());
    return SM_OK;
  }
  if (c->mode == 2) {  // predict, keep the prediction only if it helps
    std::vector<int> boxes;
    if ((st = sample_boxes(c, ctx, boxes))) return st;
    int k = std::min((int)boxes.size(), c->max_boxes);
    if (k <= 0) return SM_OK;
    double rel_plain = 0.0, rel_cnn = 0.0;
    if ((st = sm_rel_residual_now(ctx, &rel_plain))) return st;
    CCK(cudaMemcpyAsync(ctx->res, ctx->phi, sizeof(double) * CELLS * (size_t)ctx->n_boxes,
                        cudaMemcpyDeviceToDevice, ctx->stream));
    CCK(cudaMemcpyAsync(c->boxes, boxes.data(), 4 * (size_t)k, cudaMemcpyHostToDevice, ctx->stream));
    k_cnn_gather<<<k, CT, 0, ctx->stream>>>(c->boxes, k, ctx->phi, ctx->rhs, ctx->gh, ctx->nbr6, ctx->level,
                                            ctx->child, ctx->bc, ctx->lh, c->Xp, c->sc_p, nullptr, 0);
    k_cnn_forward<<<std::min(k, 4 * c->sms), CT, fwd_smem(), ctx->stream>>>(c->Xp, k, c->w, c->out, nullptr,
                                                                            c->derr);
    k_cnn_apply<<<k, CT, 0, ctx->stream>>>(c->boxes, k, c->out, c->sc_p, ctx->phi, c->taper);
    ctx->n_launch += 3;
    CCK(cudaGetLastError());
    if ((st = sm_restrict_pair(ctx, ctx->phi, nullptr))) return st;
    if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
    if ((st = sm_rel_residual_now(ctx, &rel_cnn))) return st;
    ++c->predictions;
    c->last_rel_plain = rel_plain;
    c->last_rel_cnn = rel_cnn;
    if (rel_cnn < c->accept * rel_plain) {
      ++c->kept;
    } else {  // the residual test rejects the prediction: plain warm start
      CCK(cudaMemcpyAsync(ctx->phi, ctx->res, sizeof(double) * CELLS * (size_t)ctx->n_boxes,
                          cudaMemcpyDeviceToDevice, ctx->stream));
      if ((st = sm_fill_all_cf(ctx, ctx->phi))) return st;
    }
  }
  return SM_OK;
}

static int cnn_post_solve(void *obj, sm_ctx *ctx) {
  sm_cnn *c = (sm_cnn *)obj;
  if (c->mode != 1 || c->pending.empty()) return SM_OK;
  int k = (int)c->pending.size();
  CCK(cudaMemcpyAsync(c->boxes, c->pending.data(), 4 * (size_t)k, cudaMemcpyHostToDevice, ctx->stream));
  k_cnn_target<<<k, CT, 0, ctx->stream>>>(c->boxes, k, ctx->phi, c->phi_prev, c->scale, c->target,
                                          c->pending_slot);
  ++ctx->n_launch;
  CCK(cudaGetLastError());
  c->n_samples += k;
  c->pending.clear();
  return SM_OK;
}

extern "C" int sm_cnn_attach(sm_ctx *ctx, sm_cnn *c, int mode, int per_solve, int stride, int taper,
                             double accept) {
  if (!ctx) return SM_EINVAL;
  if (mode == 0 || !c) {
    ctx->hook_obj = nullptr;
    ctx->pre_solve = nullptr;
    ctx->post_solve = nullptr;
    return SM_OK;
  }
  if ((mode != 1 && mode != 2) || per_solve < 1 || stride < 1 || !c->arena || !(accept > 0.0)) return SM_EINVAL;
  if (per_solve > c->max_boxes) return SM_EINVAL;
  c->mode = mode;
  c->per_solve = per_solve;
  c->stride = stride;
  c->taper = taper != 0;
  c->accept = accept;
  ctx->hook_obj = c;
  ctx->pre_solve = cnn_pre_solve;
  ctx->post_solve = cnn_post_solve;
  return SM_OK;
}

extern "C" int sm_cnn_stats(const sm_cnn *c, int *n_samples, long long *predictions, long long *kept,
                            double *last_rel) {
  if (!c) return SM_EINVAL;
  if (n_samples) *n_samples = c->n_samples;
  if (predictions) *predictions = c->predictions;
  if (kept) *kept = c->kept;
  if (last_rel) {
    last_rel[0] = c->last_rel_plain;
    last_rel[1] = c->last_rel_cnn;
  }
  return SM_OK;
}

extern "C" const char *sm_cnn_last_error(const sm_cnn *c) { return c ? c->err.c_str() : "null network"; }
