// regrid.cu -- refinement criterion (Sec. 2.5, Eq. 8) and regridding of
// the octree: per-box flags from |E| computed on the GPU, a new box set
// under proper nesting (Sec. 2.1.1), field data carried over to the new box
// numbering and prolonged into new boxes.
#include <string.h>

#include <vector>

#include "sm_internal.cuh"
#include "sm_nvtx.h"

using namespace sm;

namespace {

// Flag-mask bits of a leaf box: bit d (d < 26) -- a cell that needs
// refinement lies within the buffer distance of the neighbour in direction
// d; NEED -- some cell needs refinement; COARSE -- some cell fails the
// derefinement criterion.
constexpr unsigned NEED = 1u << 26, COARSE = 1u << 27;

struct LevelDx {
  double v[SM_MAX_LEVELS + 1];
};

// alpha(e) from the table sampled at E_k = k e_max/(n-1): linear
// interpolation, clamped at the ends.  Every operation is rounded on its
// own (no fused multiply-add), so the Eq. 8 threshold decision is the same
// in any implementation that evaluates the same formula.
__device__ __forceinline__ double alpha_rn(const double *__restrict__ t, int n, double de, double e) {
  const double x = __ddiv_rn(e, de);
  if (x <= 0.0) return t[0];
  if (x >= (double)(n - 1)) return t[n - 1];
  const int i = (int)x;
  const double w = __dsub_rn(x, (double)i);
  return __dadd_rn(t[i], __dmul_rn(w, __dsub_rn(t[i + 1], t[i])));
}

// Eq. 8 cell by cell on every leaf box (one block per box, one thread per
// cell): a cell needs refinement where alpha(c1 |E|) dx >= c0 c1; the box
// mask collects NEED, COARSE (alpha(c1 |E|) dx < c0_deref c1 fails) and,
// per neighbour direction, whether a needing cell is within `buffer` cells
// of that neighbour (Chebyshev distance).
__global__ void __launch_bounds__(512) k_ref_mask(const int32_t *__restrict__ leaf, const int32_t *__restrict__ level,
                                                  const double *__restrict__ emag, const double *__restrict__ alpha,
                                                  int tab_n, double de, double c1, double c0c1, double c0dc1,
                                                  LevelDx dxl, int buffer, uint32_t *__restrict__ mask) {
  __shared__ uint32_t acc;
  const int b = leaf[blockIdx.x], c = threadIdx.x;
  if (c == 0) acc = 0u;
  __syncthreads();
  const int ic[3] = {c & 7, (c >> 3) & 7, c >> 6};
  const double dx = dxl.v[level[b]];
  const double ad = __dmul_rn(alpha_rn(alpha, tab_n, de, __dmul_rn(c1, emag[(size_t)b * CELLS + c])), dx);
  uint32_t m = 0u;
  if (ad >= c0c1) {
    m |= NEED;
    for (int d = 0; d < 26; ++d) {
      const int dd = d < 13 ? d : d + 1;
      const int s[3] = {dd % 3 - 1, (dd / 3) % 3 - 1, dd / 9 - 1};
      bool in = true;
      for (int a = 0; a < 3; ++a) {
        if (s[a] > 0 && NC - ic[a] > buffer) in = false;
        if (s[a] < 0 && ic[a] + 1 > buffer) in = false;
      }
      if (in) m |= 1u << d;
    }
  }
  if (!(ad < c0dc1)) m |= COARSE;
  m = __reduce_or_sync(0xffffffffu, m);
  if ((c & 31) == 0 && m) atomicOr(&acc, m);
  __syncthreads();
  if (c == 0) mask[b] = acc;
}

// Per leaf: refine (+1) when a needing cell is in the box or within the
// buffer in a same-level leaf neighbour and the level is below the
// maximum; derefinable (-1) when nothing marks it, every cell meets the
// derefinement criterion, dx < dx_deref and the box is above the base grid.
__global__ void k_ref_flags(const int32_t *__restrict__ leaf, int n_leaves, const int32_t *__restrict__ level,
                            const int32_t *__restrict__ nbr, const int32_t *__restrict__ child,
                            const uint32_t *__restrict__ mask, int lbase, int lmax, LevelDx dxl, double dx_deref,
                            int8_t *__restrict__ flags) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_leaves) return;
  const int b = leaf[t];
  const uint32_t m = mask[b];
  bool marked = (m & NEED) != 0u;
  for (int d = 0; d < 26 && !marked; ++d) {
    const int nb = nbr[26 * b + d];
    // the neighbour's slab facing this box is the opposite direction
    if (nb >= 0 && child[8 * nb] < 0 && ((mask[nb] >> (25 - d)) & 1u)) marked = true;
  }
  const int l = level[b];
  int8_t f = 0;
  if (marked) f = l < lmax ? 1 : 0;
  else if (!(m & COARSE) && dxl.v[l] < dx_deref && l > lbase) f = -1;
  flags[b] = f;
}

__global__ void __launch_bounds__(512) k_regrid_gather(const int32_t *__restrict__ src, const double *__restrict__ x,
                                                       double *__restrict__ y) {
  const int s = src[blockIdx.x];
  y[(size_t)blockIdx.x * CELLS + threadIdx.x] = s >= 0 ? x[(size_t)s * CELLS + threadIdx.x] : 0.0;
}

// New boxes: (c + c_sx + c_sy + c_sz)/4 of the parent's cells, s the
// direction of the fine cell inside its coarse cell, for the potential
// (wall ghosts 2g - c or c) and the densities (mirror ghosts c, result
// limited to 2c), summed in the order c, x, y, z.
__global__ void __launch_bounds__(512) k_regrid_prolong(const int32_t *__restrict__ list,
                                                        const int32_t *__restrict__ parent,
                                                        const int32_t *__restrict__ ijk,
                                                        const int32_t *__restrict__ nbr6, Bc bc, double *phi,
                                                        double *ne, double *ni, unsigned long long *err) {
  const int b = list[blockIdx.x], p = parent[b], c = threadIdx.x;
  const int ic[3] = {c & 7, (c >> 3) & 7, c >> 6};
  int cl[3], s[3];
  for (int a = 0; a < 3; ++a) {
    cl[a] = ((ijk[3 * b + a] & 1) * NC + ic[a]) >> 1;
    s[a] = (ic[a] & 1) ? 1 : -1;
  }
  double *vars[3] = {phi, ne, ni};
  for (int v = 0; v < 3; ++v) {
    double *X = vars[v];
    const double cval = X[(size_t)p * CELLS + cl[0] + NC * cl[1] + FACE * cl[2]];
    double sum = cval;
    for (int a = 0; a < 3; ++a) {
      int q[3] = {cl[0], cl[1], cl[2]};
      q[a] += s[a];
      double nv;
      if (q[a] >= 0 && q[a] < NC) {
        nv = X[(size_t)p * CELLS + q[0] + NC * q[1] + FACE * q[2]];
      } else {
        const int f = 2 * a + (s[a] > 0 ? 1 : 0), nb = nbr6[6 * p + f];
        if (nb >= 0) {
          q[a] = s[a] > 0 ? 0 : NC - 1;
          nv = X[(size_t)nb * CELLS + q[0] + NC * q[1] + FACE * q[2]];
        } else if (nb == -1) {
          nv = (v == 0 && bc.type[f]) ? bc.g2[f] - cval : cval;
        } else {
          atomicOr(err, 16ull);  // nesting violated: the parent lacks a face neighbour
          nv = cval;
        }
      }
      sum += nv;
    }
    double val = 0.25 * sum;
    if (v > 0 && val > 2.0 * cval) val = 2.0 * cval;
    X[(size_t)b * CELLS + c] = val;
  }
}

static LevelDx level_dx(const sm_ctx *ctx) {
  LevelDx d;
  for (int l = 0; l <= SM_MAX_LEVELS; ++l) d.v[l] = ctx->dom.length / (NC * (double)(1 << l));
  return d;
}

// ---- the new box set on the device --------------------------------------
//
// Old boxes are stored level by level in Morton order.  The new set keeps
// every box but the children of derefined boxes and adds 8 children per
// refined box; at each level it is the merge of two Morton-sorted lists
// (the kept boxes of the level and the children of the refined boxes of the
// level below, whose keys are parent key * 8 + child), so a box's new index
// is its rank in its own list plus the number of keys of the other list
// below its own (binary searches).  Parents and children follow by binary
// search in the new levels' keys.

// per-level offsets of the compacted lists and of the new levels
struct RgLevels {
  int kept[SM_MAX_LEVELS + 2];   // start of level l in the kept list
  int ref[SM_MAX_LEVELS + 2];    // start of level l in the refined list
  int nw[SM_MAX_LEVELS + 2];     // start of level l in the new numbering
};

// first index in [lo, hi) whose key is >= x
__device__ __forceinline__ int lower_bound_u64(const uint64_t *__restrict__ a, int lo, int hi, uint64_t x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// refinement: a flagged leaf below the maximum level whose 26 neighbour
// positions of its level hold a box or lie outside the domain (else the
// request is dropped, cnt[0])
__global__ void k_rg_refine(int n, const int32_t *__restrict__ level, const int32_t *__restrict__ child,
                            const int32_t *__restrict__ nbr, const int8_t *__restrict__ flags, int lmax,
                            int32_t *__restrict__ refv, int32_t *cnt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  int r = 0;
  if (child[8 * b] < 0 && flags[b] > 0 && level[b] < lmax) {
    bool ok = true;
    for (int d = 0; d < 26; ++d) ok = ok && nbr[26 * b + d] != -2;
    if (ok) r = 1;
    else atomicAdd(cnt, 1);
  }
  refv[b] = r;
}

// derefinement of box p: its 8 children are leaves flagged < 0, and no
// non-sibling neighbour of a child has or gets children (cnt[1] counts);
// then keep[b] = b is not a child of a derefined box
__global__ void k_rg_derefine(int n, const int32_t *__restrict__ child, const int32_t *__restrict__ parent,
                              const int32_t *__restrict__ nbr, const int8_t *__restrict__ flags,
                              const int32_t *__restrict__ refv, int8_t *__restrict__ derv, int32_t *cnt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  bool ok = child[8 * p] >= 0;
  for (int c = 0; c < 8 && ok; ++c) {
    const int ch = child[8 * p + c];
    ok = child[8 * ch] < 0 && flags[ch] < 0;
  }
  for (int c = 0; c < 8 && ok; ++c) {
    const int ch = child[8 * p + c];
    for (int d = 0; d < 26 && ok; ++d) {
      const int nb = nbr[26 * ch + d];
      if (nb >= 0 && parent[nb] != p && (child[8 * nb] >= 0 || refv[nb])) ok = false;
    }
  }
  derv[p] = ok ? 1 : 0;
  if (ok) atomicAdd(cnt + 1, 1);
}

__global__ void k_rg_keep(int n, const int32_t *__restrict__ parent, const int8_t *__restrict__ derv,
                          int32_t *__restrict__ keepv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int p = parent[b];
  keepv[b] = (p >= 0 && derv[p]) ? 0 : 1;
}

// the Morton keys of the kept and of the refined boxes, compacted
__global__ void k_rg_keys(int n, const uint64_t *__restrict__ morton, const int32_t *__restrict__ keepv,
                          const int32_t *__restrict__ keep_pos, const int32_t *__restrict__ refv,
                          const int32_t *__restrict__ ref_pos, uint64_t *__restrict__ kept_keys,
                          uint64_t *__restrict__ ref_keys) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  if (keepv[b]) kept_keys[keep_pos[b]] = morton[b];
  if (refv[b]) ref_keys[ref_pos[b]] = morton[b];
}

// new index, level, coordinates, key and source of every kept box and of
// the 8 children of every refined box (8 threads per old box: thread 0
// places the box itself when kept, thread c its child c when refined)
__global__ void k_rg_place(int n, const int32_t *__restrict__ level, const int32_t *__restrict__ ijk,
                           const uint64_t *__restrict__ morton, const int32_t *__restrict__ keepv,
                           const int32_t *__restrict__ keep_pos, const int32_t *__restrict__ refv,
                           const int32_t *__restrict__ ref_pos, const uint64_t *__restrict__ kept_keys,
                           const uint64_t *__restrict__ ref_keys, RgLevels L, int32_t *__restrict__ nlev,
                           int32_t *__restrict__ nijk, uint64_t *__restrict__ nkey, int32_t *__restrict__ nsrc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = t >> 3, c = t & 7;
  if (b >= n) return;
  const int l = level[b];
  const uint64_t key = morton[b];
  if (c == 0 && keepv[b]) {
    // refined boxes of level l-1 whose key is below this box's parent key
    const int below = l > 0 ? lower_bound_u64(ref_keys, L.ref[l - 1], L.ref[l], key >> 3) - L.ref[l - 1] : 0;
    const int x = L.nw[l] + (keep_pos[b] - L.kept[l]) + 8 * below;
    nlev[x] = l;
    nijk[3 * x] = ijk[3 * b];
    nijk[3 * x + 1] = ijk[3 * b + 1];
    nijk[3 * x + 2] = ijk[3 * b + 2];
    nkey[x] = key;
    nsrc[x] = b;
  }
  if (refv[b]) {
    const uint64_t ck = (key << 3) | (uint64_t)c;
    const int below = lower_bound_u64(kept_keys, L.kept[l + 1], L.kept[l + 2], ck) - L.kept[l + 1];
    const int x = L.nw[l + 1] + 8 * (ref_pos[b] - L.ref[l]) + c + below;
    nlev[x] = l + 1;
    nijk[3 * x] = 2 * ijk[3 * b] + (c & 1);
    nijk[3 * x + 1] = 2 * ijk[3 * b + 1] + ((c >> 1) & 1);
    nijk[3 * x + 2] = 2 * ijk[3 * b + 2] + (c >> 2);
    nkey[x] = ck;
    nsrc[x] = -1;
  }
}

// parent and children of every new box by binary search in the new keys
__global__ void k_rg_links(int m, const int32_t *__restrict__ nlev, const uint64_t *__restrict__ nkey, RgLevels L,
                           int nlevels, int32_t *__restrict__ npar, int32_t *__restrict__ nchl) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m) return;
  const int l = nlev[b];
  const uint64_t key = nkey[b];
  int p = -1;
  if (l > 0) {
    const int i = lower_bound_u64(nkey, L.nw[l - 1], L.nw[l], key >> 3);
    if (i < L.nw[l] && nkey[i] == key >> 3) p = i;
  }
  npar[b] = p;
  int c0 = -1;
  if (l + 1 < nlevels) {
    const int i = lower_bound_u64(nkey, L.nw[l + 1], L.nw[l + 2], key << 3);
    if (i < L.nw[l + 2] && nkey[i] == key << 3) c0 = i;
  }
  for (int c = 0; c < 8; ++c) nchl[8 * b + c] = c0 >= 0 ? c0 + c : -1;
}

// boxes without a source (new children), compacted
__global__ void k_rg_fresh_flag(int m, const int32_t *__restrict__ nsrc, int32_t *__restrict__ f) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < m) f[b] = nsrc[b] < 0 ? 1 : 0;
}

__global__ void k_rg_compact(int m, const int32_t *__restrict__ f, const int32_t *__restrict__ pos,
                             int32_t *__restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < m && f[b]) out[pos[b]] = b;
}

}  // namespace

extern "C" int sm_refine_flags(sm_ctx *ctx, double c0, double c1, double c0_deref, double dx_deref, int buffer,
                               int8_t *flags) {
  SM_RANGE();
  if (!ctx || !flags || buffer < 0 || buffer > NC) return SM_EINVAL;
  if (!ctx->arena || ctx->n_levels == 0) return sm_fail(ctx, SM_ESTATE, "octree not built");
  if (ctx->tab_n < 2) return sm_fail(ctx, SM_ESTATE, "no coefficient table");
  const int n = ctx->n_boxes;
  uint32_t *mask = reinterpret_cast<uint32_t *>(ctx->scan_a);
  SM_CK(cudaMemsetAsync(mask, 0, sizeof(uint32_t) * n, ctx->stream));
  SM_CK(cudaMemsetAsync(ctx->dev_flags, 0, n, ctx->stream));
  const LevelDx dxl = level_dx(ctx);
  const double de = ctx->tab_emax / (ctx->tab_n - 1);
  if (ctx->n_leaves > 0) {
    k_ref_mask<<<ctx->n_leaves, CELLS, 0, ctx->stream>>>(ctx->leaf, ctx->level, ctx->emag, ctx->tab + 8192,
                                                         ctx->tab_n, de, c1, c0 * c1, c0_deref * c1, dxl, buffer,
                                                         mask);
    ++ctx->n_launch;
    k_ref_flags<<<(ctx->n_leaves + 255) / 256, 256, 0, ctx->stream>>>(ctx->leaf, ctx->n_leaves, ctx->level,
                                                                       ctx->nbr, ctx->child, mask, ctx->lbase,
                                                                       ctx->lmax, dxl, dx_deref, ctx->dev_flags);
    ++ctx->n_launch;
    SM_CKL("refine flags");
  }
  SM_CK(cudaMemcpyAsync(flags, ctx->dev_flags, n, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  return SM_OK;
}

int sm_regrid_impl(sm_ctx *ctx, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped);

extern "C" int sm_regrid(sm_ctx *ctx, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped) {
  return sm_regrid_impl(ctx, flags, n_refined, n_derefined, n_dropped);
}

extern "C" int sm_refine(sm_ctx *ctx, const int8_t *flags, int *n_boxes) {
  const int st = sm_regrid_impl(ctx, flags, nullptr, nullptr, nullptr);
  if (st == SM_OK && n_boxes) *n_boxes = ctx->n_boxes;
  return st;
}

int sm_regrid_impl(sm_ctx *ctx, const int8_t *flags, int *n_refined, int *n_derefined, int *n_dropped) {
  SM_RANGE();
  if (!ctx) return SM_EINVAL;
  if (!ctx->arena || ctx->n_levels == 0) return sm_fail(ctx, SM_ESTATE, "octree not built");
  int st;
  // densities of refined boxes = mean of their children, on the old mesh
  if ((st = sm_restrict_pair(ctx, ctx->nbuf[ctx->ncur], ctx->ibuf[ctx->ncur]))) return st;
  const int n = ctx->n_boxes, M = ctx->cfg.max_boxes, T = 256;
  // flags: from the host, or (NULL) those the last sm_refine_flags left on the device
  if (flags) SM_CK(cudaMemcpyAsync(ctx->dev_flags, flags, n, cudaMemcpyHostToDevice, ctx->stream));
  // scratch in the residual array (not carried over by a regrid)
  char *w = reinterpret_cast<char *>(ctx->res);
  auto take = [&](size_t bytes) {
    char *p = w;
    w += (bytes + 255) & ~(size_t)255;
    return p;
  };
  int32_t *refv = (int32_t *)take(4 * (size_t)n), *keepv = (int32_t *)take(4 * (size_t)n);
  int32_t *ref_pos = (int32_t *)take(4 * ((size_t)n + 1)), *keep_pos = (int32_t *)take(4 * ((size_t)n + 1));
  int8_t *derv = (int8_t *)take((size_t)n);
  uint64_t *ref_keys = (uint64_t *)take(8 * (size_t)n), *kept_keys = (uint64_t *)take(8 * (size_t)n);
  int32_t *nlev = (int32_t *)take(4 * (size_t)M), *nijk = (int32_t *)take(12 * (size_t)M);
  uint64_t *nkey = (uint64_t *)take(8 * (size_t)M);
  int32_t *nsrc = (int32_t *)take(4 * (size_t)M), *npar = (int32_t *)take(4 * (size_t)M);
  int32_t *nchl = (int32_t *)take(32 * (size_t)M);
  int32_t *ff = (int32_t *)take(4 * (size_t)M), *fpos = (int32_t *)take(4 * ((size_t)M + 1));
  int32_t *cnt = ctx->dev_count;
  SM_CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(int32_t), ctx->stream));
  const int gb = (n + T - 1) / T;
  k_rg_refine<<<gb, T, 0, ctx->stream>>>(n, ctx->level, ctx->child, ctx->nbr, ctx->dev_flags, ctx->lmax, refv, cnt);
  k_rg_derefine<<<gb, T, 0, ctx->stream>>>(n, ctx->child, ctx->parent, ctx->nbr, ctx->dev_flags, refv, derv, cnt);
  k_rg_keep<<<gb, T, 0, ctx->stream>>>(n, ctx->parent, derv, keepv);
  ctx->n_launch += 3;
  SM_CKL("regrid decisions");
  if ((st = sm_exclusive_scan(ctx, refv, ref_pos, n))) return st;
  if ((st = sm_exclusive_scan(ctx, keepv, keep_pos, n))) return st;
  // counts: dropped, derefined, and the list offsets at the old level offsets
  const int L0 = ctx->n_levels;
  std::vector<int32_t> hk(L0 + 1), hr(L0 + 1);
  int32_t hc[2];
  SM_CK(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, ctx->stream));
  for (int l = 0; l <= L0; ++l) {
    SM_CK(cudaMemcpyAsync(&hk[l], keep_pos + ctx->level_off[l], 4, cudaMemcpyDeviceToHost, ctx->stream));
    SM_CK(cudaMemcpyAsync(&hr[l], ref_pos + ctx->level_off[l], 4, cudaMemcpyDeviceToHost, ctx->stream));
  }
  SM_CK(cudaStreamSynchronize(ctx->stream));
  const int nref = hr[L0], nder = hc[1];
  if (n_refined) *n_refined = nref;
  if (n_derefined) *n_derefined = nder;
  if (n_dropped) *n_dropped = hc[0];
  if (nref == 0 && nder == 0) return SM_OK;
  RgLevels L;
  int nlevels = 0, m = 0;
  for (int l = 0; l < SM_MAX_LEVELS + 2; ++l) {
    const int kept = l < L0 ? hk[l + 1] - hk[l] : 0;
    const int born = (l >= 1 && l - 1 < L0) ? 8 * (hr[l] - hr[l - 1]) : 0;
    L.kept[l] = l <= L0 ? hk[l] : hk[L0];
    L.ref[l] = l <= L0 ? hr[l] : hr[L0];
    L.nw[l] = m;
    m += kept + born;
    if (kept + born > 0) nlevels = l + 1;
  }
  if (m > M) return sm_fail(ctx, SM_ENOMEM, "max_boxes %d exceeded (%d needed)", M, m);
  if (nlevels > SM_MAX_LEVELS) return sm_fail(ctx, SM_EINVAL, "more than %d levels", SM_MAX_LEVELS);
  k_rg_keys<<<gb, T, 0, ctx->stream>>>(n, ctx->morton, keepv, keep_pos, refv, ref_pos, kept_keys, ref_keys);
  k_rg_place<<<(8 * n + T - 1) / T, T, 0, ctx->stream>>>(n, ctx->level, ctx->ijk, ctx->morton, keepv, keep_pos, refv,
                                                         ref_pos, kept_keys, ref_keys, L, nlev, nijk, nkey, nsrc);
  k_rg_links<<<(m + T - 1) / T, T, 0, ctx->stream>>>(m, nlev, nkey, L, nlevels, npar, nchl);
  k_rg_fresh_flag<<<(m + T - 1) / T, T, 0, ctx->stream>>>(m, nsrc, ff);
  ctx->n_launch += 4;
  SM_CKL("regrid box set");
  if ((st = sm_exclusive_scan(ctx, ff, fpos, m))) return st;
  k_rg_compact<<<(m + T - 1) / T, T, 0, ctx->stream>>>(m, ff, fpos, ctx->scan_a);
  ++ctx->n_launch;
  sm_drop_graphs(ctx);
  // fields to the new numbering (new boxes zero), through the scratch array
  // of the previous cycle's potential
  double *vars[6] = {ctx->phi, ctx->rhs, ctx->emag, ctx->rho, ctx->nbuf[ctx->ncur], ctx->ibuf[ctx->ncur]};
  for (double *x : vars) {
    k_regrid_gather<<<m, CELLS, 0, ctx->stream>>>(nsrc, x, ctx->old);
    ++ctx->n_launch;
    SM_CK(cudaMemcpyAsync(x, ctx->old, sizeof(double) * CELLS * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  SM_CKL("regrid gather");
  // tables of the new mesh; neighbours and the leaf list from them
  SM_CK(cudaMemcpyAsync(ctx->level, nlev, 4 * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
  SM_CK(cudaMemcpyAsync(ctx->ijk, nijk, 12 * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
  SM_CK(cudaMemcpyAsync(ctx->morton, nkey, 8 * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
  SM_CK(cudaMemcpyAsync(ctx->parent, npar, 4 * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
  SM_CK(cudaMemcpyAsync(ctx->child, nchl, 32 * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->n_boxes = m;
  ctx->n_levels = nlevels;
  for (int l = 0; l <= SM_MAX_LEVELS; ++l) ctx->level_off[l] = L.nw[l];
  for (int l = 0; l < nlevels; ++l)
    if ((st = sm_build_neighbours(ctx, l))) return st;
  // the fresh-box list (scan_a) is read before the leaf rebuild reuses it
  if (nref > 0) {
    k_regrid_prolong<<<8 * nref, CELLS, 0, ctx->stream>>>(ctx->scan_a, ctx->parent, ctx->ijk, ctx->nbr6, ctx->bc,
                                                         ctx->phi, ctx->nbuf[ctx->ncur], ctx->ibuf[ctx->ncur],
                                                         ctx->dscal + SC_ERR);
    ++ctx->n_launch;
    SM_CKL("regrid prolong");
  }
  if ((st = sm_rebuild_leaves(ctx))) return st;
  SM_CK(cudaStreamSynchronize(ctx->stream));
  return SM_OK;
}
