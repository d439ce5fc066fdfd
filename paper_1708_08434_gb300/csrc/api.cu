// api.cu -- context, arena, octree tables (Sec. 2.1.1), field transfer and
// diagnostics of the C ABI declared in sm_streamer.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "sm_internal.cuh"
#include "sm_nvtx.h"

using namespace sm;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
int sm_fail(sm_ctx *ctx, int code, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int sm_cuda_check(sm_ctx *ctx, cudaError_t e, const char *what) {
  return sm_fail(ctx, SM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" int sm_launch_count(const sm_ctx *ctx, long long *n) {
  if (!ctx || !n) return SM_EINVAL;
  *n = ctx->n_launch;
  return SM_OK;
}

extern "C" const char *sm_last_error(const sm_ctx *ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

// ---------------------------------------------------------------------------
// lifetime and arena
// ---------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct ArenaPlan {
  size_t total = 0;
  template <typename T>
  size_t take(size_t count) {
    size_t at = total;
    total = align256(total + count * sizeof(T));
    return at;
  }
};

// layout shared by sm_arena_size and sm_bind_arena
struct Layout {
  size_t level, ijk, parent, child, nbr, nbr6, leaf, cf_leaf, morton, scan_a, scan_b, count, flags;
  size_t phi, rhs, res, old, rho, emag, nb[3], ib[3], gh, cflux, basis, tab, dscal, hist, e32, f32, old32, gh32,
      phx, gx, ghx, total;
};

static Layout plan(int cap, bool mixed) {
  ArenaPlan p;
  Layout L;
  size_t nc = (size_t)cap * CELLS;
  L.level = p.take<int32_t>(cap);
  L.ijk = p.take<int32_t>((size_t)cap * 3);
  L.parent = p.take<int32_t>(cap);
  L.child = p.take<int32_t>((size_t)cap * 8);
  L.nbr = p.take<int32_t>((size_t)cap * 26);
  L.nbr6 = p.take<int32_t>((size_t)cap * 6);
  L.leaf = p.take<int32_t>(cap);
  L.cf_leaf = p.take<int32_t>(cap);
  L.morton = p.take<uint64_t>(cap);
  L.scan_a = p.take<int32_t>(cap + 1);
  L.scan_b = p.take<int32_t>(cap + 1);
  L.count = p.take<int32_t>(64);
  L.flags = p.take<int8_t>(cap);
  L.phi = p.take<double>(nc);
  L.rhs = p.take<double>(nc);
  L.res = p.take<double>(nc);
  L.old = p.take<double>(nc);
  L.rho = p.take<double>(nc);
  L.emag = p.take<double>(nc);
  for (int i = 0; i < 3; ++i) L.nb[i] = p.take<double>(nc);
  for (int i = 0; i < 3; ++i) L.ib[i] = p.take<double>(nc);
  L.gh = p.take<double>((size_t)cap * 6 * FACE);
  L.cflux = p.take<double>((size_t)cap * 6 * FACE);
  L.basis = p.take<double>(3 * 64 + 3 * 8);
  L.tab = p.take<double>(6 * 4096);  // mu, D, alpha and their slopes t[i+1] - t[i]
  L.dscal = p.take<unsigned long long>(SC_N);
  L.hist = p.take<double>(SM_HIST);
  L.phx = p.take<long long>(nc);
  L.gx = p.take<long long>(nc);
  L.ghx = p.take<long long>((size_t)cap * 6 * FACE);
  if (mixed) {
    L.e32 = p.take<float>(nc);
    L.f32 = p.take<float>(nc);
    L.old32 = p.take<float>(nc);
    L.gh32 = p.take<float>((size_t)cap * 6 * FACE);
  } else {
    L.e32 = L.f32 = L.old32 = L.gh32 = 0;
  }
  L.total = p.total;
  return L;
}

static int uniform_boxes(int lbase) {
  int n = 0;
  for (int l = 0; l <= lbase; ++l) n += 1 << (3 * l);
  return n;
}

extern "C" int sm_create(sm_ctx **out, const sm_config *cfg, const sm_domain *dom, void *stream) {
  if (!out || !cfg || !dom) return SM_EINVAL;
  *out = nullptr;
  int lb = 0;
  while ((1 << lb) < dom->nb) ++lb;
  if (dom->nb < 1 || (1 << lb) != dom->nb) return SM_EINVAL;
  if (dom->max_level < 0 || lb + dom->max_level >= SM_MAX_LEVELS) return SM_EINVAL;
  if (cfg->nu1 < 1 || cfg->nu2 < 1 || cfg->max_boxes < uniform_boxes(lb)) return SM_EINVAL;
  if (!(dom->length > 0.0)) return SM_EINVAL;
  bool any_dirichlet = false;
  for (int f = 0; f < 6; ++f) {
    if (dom->bc_type[f] != 0 && dom->bc_type[f] != 1) return SM_EINVAL;
    any_dirichlet |= dom->bc_type[f] == 1;
  }
  if (!any_dirichlet) return SM_EINVAL;
  if (cfg->precision != SM_FP64 && cfg->precision != SM_MIXED) return SM_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return SM_ECUDA;
  }
  sm_ctx *ctx = new sm_ctx();
  ctx->cfg = *cfg;
  ctx->dom = *dom;
  ctx->lbase = lb;
  ctx->lmax = lb + dom->max_level;
  ctx->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    delete ctx;
    return SM_ECUDA;
  }
  for (int f = 0; f < 6; ++f) {
    ctx->bc.type[f] = dom->bc_type[f];
    ctx->bc.val[f] = dom->bc_val[f];
  }
  bc_finish(ctx->bc);
  for (int l = 0; l < MAXL; ++l) {
    double h = dom->length / (NC * (double)(1 << l));
    ctx->lh.h[l] = h;
    ctx->lh.inv_h[l] = 1.0 / h;
    ctx->lh.h2[l] = h * h;
    ctx->lh.inv_h2[l] = 1.0 / (h * h);
  }
  if (cudaMallocHost((void **)&ctx->hscal, sizeof(double) * 2 * SC_N) != cudaSuccess) {  // + staged copy
    delete ctx;
    return SM_ECUDA;
  }
  *out = ctx;
  return SM_OK;
}

extern "C" int sm_destroy(sm_ctx *ctx) {
  if (!ctx) return SM_OK;
  sm_drop_graphs(ctx);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  if (ctx->cap2) cudaStreamDestroy(ctx->cap2);
  if (ctx->hscal) cudaFreeHost(ctx->hscal);
  if (ctx->mlog) fclose(ctx->mlog);
  for (cudaEvent_t e : ctx->mlog_ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return SM_OK;
}

extern "C" int sm_arena_size(const sm_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return SM_EINVAL;
  *bytes = plan(ctx->cfg.max_boxes, ctx->cfg.precision == SM_MIXED).total;
  return SM_OK;
}

extern "C" int sm_bind_arena(sm_ctx *ctx, void *dev_ptr, size_t bytes) {
  if (!ctx || !dev_ptr) return SM_EINVAL;
  Layout L = plan(ctx->cfg.max_boxes, ctx->cfg.precision == SM_MIXED);
  if (bytes < L.total) return sm_fail(ctx, SM_ENOMEM, "arena %zu bytes < needed %zu", bytes, L.total);
  if (((uintptr_t)dev_ptr & 255) != 0) return sm_fail(ctx, SM_EINVAL, "arena not 256-byte aligned");
  char *a = (char *)dev_ptr;
  ctx->arena = a;
  ctx->arena_bytes = bytes;
  ctx->level = (int32_t *)(a + L.level);
  ctx->ijk = (int32_t *)(a + L.ijk);
  ctx->parent = (int32_t *)(a + L.parent);
  ctx->child = (int32_t *)(a + L.child);
  ctx->nbr = (int32_t *)(a + L.nbr);
  ctx->nbr6 = (int32_t *)(a + L.nbr6);
  ctx->leaf = (int32_t *)(a + L.leaf);
  ctx->cf_leaf = (int32_t *)(a + L.cf_leaf);
  ctx->morton = (uint64_t *)(a + L.morton);
  ctx->scan_a = (int32_t *)(a + L.scan_a);
  ctx->scan_b = (int32_t *)(a + L.scan_b);
  ctx->dev_count = (int32_t *)(a + L.count);
  ctx->dev_flags = (int8_t *)(a + L.flags);
  ctx->phi = (double *)(a + L.phi);
  ctx->rhs = (double *)(a + L.rhs);
  ctx->res = (double *)(a + L.res);
  ctx->old = (double *)(a + L.old);
  ctx->rho = (double *)(a + L.rho);
  ctx->emag = (double *)(a + L.emag);
  for (int i = 0; i < 3; ++i) {
    ctx->nbuf[i] = (double *)(a + L.nb[i]);
    ctx->ibuf[i] = (double *)(a + L.ib[i]);
  }
  ctx->gh = (double *)(a + L.gh);
  ctx->cflux = (double *)(a + L.cflux);
  ctx->basis = (double *)(a + L.basis);
  ctx->tab = (double *)(a + L.tab);
  ctx->dscal = (unsigned long long *)(a + L.dscal);
  ctx->hist = (double *)(a + L.hist);
  ctx->phx = (long long *)(a + L.phx);
  ctx->gx = (long long *)(a + L.gx);
  ctx->ghx = (long long *)(a + L.ghx);
  if (ctx->cfg.precision == SM_MIXED) {
    ctx->e32 = (float *)(a + L.e32);
    ctx->f32 = (float *)(a + L.f32);
    ctx->old32 = (float *)(a + L.old32);
    ctx->gh32 = (float *)(a + L.gh32);
  }
  SM_CK(cudaMemsetAsync(a, 0, L.total, ctx->stream));
  sm_drop_graphs(ctx);
  ctx->n_boxes = ctx->n_levels = ctx->n_leaves = ctx->n_cf_leaves = 0;
  ctx->basis_ready = false;
  return SM_OK;
}

// ---------------------------------------------------------------------------
// octree kernels (Sec. 2.1.1): Morton-sorted levels, parent/child links,
// 26-neighbour table by binary search in the sorted keys of a level
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t d_morton(int i, int j, int k) {
  uint64_t key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= (uint64_t)((i >> b) & 1) << (3 * b);
    key |= (uint64_t)((j >> b) & 1) << (3 * b + 1);
    key |= (uint64_t)((k >> b) & 1) << (3 * b + 2);
  }
  return key;
}

struct LevelOffsets {
  int off[SM_MAX_LEVELS + 1];
};

// all boxes of the uniform levels 0..lbase (level l: key = index - off[l])
__global__ void k_build_uniform(int total, int lbase, LevelOffsets lo, int32_t *level, int32_t *ijk,
                                uint64_t *morton, int32_t *parent, int32_t *child) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= total) return;
  int l = 0;
  while (b >= lo.off[l + 1]) ++l;
  uint64_t key = (uint64_t)(b - lo.off[l]);
  int c[3] = {0, 0, 0};
  for (int bit = 0; bit < 21; ++bit)
    for (int d = 0; d < 3; ++d) c[d] |= (int)((key >> (3 * bit + d)) & 1) << bit;
  level[b] = l;
  ijk[3 * b] = c[0];
  ijk[3 * b + 1] = c[1];
  ijk[3 * b + 2] = c[2];
  morton[b] = key;
  parent[b] = l ? lo.off[l - 1] + (int)(key >> 3) : -1;
  for (int q = 0; q < 8; ++q) child[8 * b + q] = l < lbase ? lo.off[l + 1] + (int)((key << 3) | q) : -1;
}

// neighbour tables of the boxes [lo, hi) of level l
__global__ void k_neighbours(int lo, int hi, int l, const int32_t *__restrict__ ijk,
                             const uint64_t *__restrict__ morton, int32_t *nbr, int32_t *nbr6) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int b = lo + t / 26, d = t % 26;
  if (b >= hi) return;
  int dd = d < 13 ? d : d + 1;
  int dx = dd % 3 - 1, dy = (dd / 3) % 3 - 1, dz = dd / 9 - 1;
  int q[3] = {ijk[3 * b] + dx, ijk[3 * b + 1] + dy, ijk[3 * b + 2] + dz};
  int side = 1 << l;
  int res;
  if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= side || q[1] >= side || q[2] >= side) {
    res = -1;
  } else {
    uint64_t key = d_morton(q[0], q[1], q[2]);
    int a = lo, z = hi - 1;
    res = -2;
    while (a <= z) {
      int m = (a + z) >> 1;
      uint64_t km = morton[m];
      if (km == key) { res = m; break; }
      if (km < key) a = m + 1; else z = m - 1;
    }
  }
  nbr[26 * b + d] = res;
  // faces -x,+x,-y,+y,-z,+z sit at 26-list positions 12,13,10,15,4,21
  int f = -1;
  if (d == 12) f = 0; else if (d == 13) f = 1; else if (d == 10) f = 2;
  else if (d == 15) f = 3; else if (d == 4) f = 4; else if (d == 21) f = 5;
  if (f >= 0) nbr6[6 * b + f] = res;
}

// refinement request of box lo+t accepted when flagged and all 26
// neighbour positions of its level hold a box or lie outside the domain
__global__ void k_refine_accept(int lo, int n, const int8_t *__restrict__ flags,
                                const int32_t *__restrict__ nbr, int32_t *accept, int32_t *count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int ok = 0;
  if (flags[t] > 0) {
    ok = 1;
    for (int d = 0; d < 26; ++d)
      if (nbr[26 * (lo + t) + d] == -2) ok = 0;
    if (!ok) atomicAdd(count + 1, 1);
  }
  accept[t] = ok;
}

// exclusive prefix sum of n ints in one block (sizes here are <= ~1e6),
// total written to out[n]
__global__ void k_scan(const int32_t *__restrict__ in, int32_t *out, int n) {
  __shared__ int32_t s[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int x = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += x;
      __syncthreads();
    }
    if (i < n) out[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// append 8 children per accepted box of level l (boxes [lo, lo+n)), in
// parent order then child order: Morton order of the new level
__global__ void k_make_children(int lo, int n, int new_lo, int l, const int32_t *__restrict__ accept,
                                const int32_t *__restrict__ pos, int32_t *level, int32_t *ijk,
                                uint64_t *morton, int32_t *parent, int32_t *child) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int p = t >> 3, c = t & 7;
  if (p >= n || !accept[p]) return;
  int pb = lo + p;
  int b = new_lo + 8 * pos[p] + c;
  int q[3] = {2 * ijk[3 * pb] + (c & 1), 2 * ijk[3 * pb + 1] + ((c >> 1) & 1), 2 * ijk[3 * pb + 2] + (c >> 2)};
  level[b] = l + 1;
  ijk[3 * b] = q[0];
  ijk[3 * b + 1] = q[1];
  ijk[3 * b + 2] = q[2];
  morton[b] = (morton[pb] << 3) | (uint64_t)c;
  parent[b] = pb;
  child[8 * pb + c] = b;
  for (int r = 0; r < 8; ++r) child[8 * b + r] = -1;
}

__global__ void k_mark_leaves(int n, const int32_t *__restrict__ child, int32_t *is_leaf) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) is_leaf[b] = child[8 * b] < 0 ? 1 : 0;
}

// leaf boxes with a refinement face: a face whose same-level neighbour is
// missing inside the domain (nbr6 == -2)
__global__ void k_mark_cf_leaves(int n, const int32_t *__restrict__ child, const int32_t *__restrict__ nbr6,
                                 int32_t *flag) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  int f = 0;
  if (child[8 * b] < 0)
    for (int k = 0; k < 6; ++k) f |= nbr6[6 * b + k] == -2;
  flag[b] = f;
}

__global__ void k_compact(int n, const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                          int32_t *out) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n && flag[b]) out[pos[b]] = b;
}

// exclusive prefix sum of n ints on the context stream; out[n] = total
int sm_exclusive_scan(sm_ctx *ctx, const int32_t *in, int32_t *out, int n) {
  k_scan<<<1, 1024, 0, ctx->stream>>>(in, out, n);
  ++ctx->n_launch;
  SM_CKL("scan");
  return SM_OK;
}

int sm_rebuild_leaves(sm_ctx *ctx) {
  int n = ctx->n_boxes;
  k_mark_leaves<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, ctx->child, ctx->scan_a);
  ++ctx->n_launch;
  k_scan<<<1, 1024, 0, ctx->stream>>>(ctx->scan_a, ctx->scan_b, n);
  ++ctx->n_launch;
  k_compact<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, ctx->scan_a, ctx->scan_b, ctx->leaf);
  ++ctx->n_launch;
  SM_CKL("leaf list");
  // leaf count and per-level leaf offsets from the prefix sums at level offsets
  std::vector<int32_t> h(ctx->n_levels + 2);
  for (int l = 0; l <= ctx->n_levels; ++l) {
    SM_CK(cudaMemcpyAsync(&h[l], ctx->scan_b + ctx->level_off[l], sizeof(int32_t),
                          cudaMemcpyDeviceToHost, ctx->stream));
  }
  // the leaves with a refinement face (the fluid step's refinement fluxes);
  // the scan buffers are reused after the copies above in stream order
  k_mark_cf_leaves<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, ctx->child, ctx->nbr6, ctx->scan_a);
  ++ctx->n_launch;
  k_scan<<<1, 1024, 0, ctx->stream>>>(ctx->scan_a, ctx->scan_b, n);
  ++ctx->n_launch;
  k_compact<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, ctx->scan_a, ctx->scan_b, ctx->cf_leaf);
  ++ctx->n_launch;
  SM_CKL("refinement-face leaf list");
  SM_CK(cudaMemcpyAsync(&h[ctx->n_levels + 1], ctx->scan_b + n, sizeof(int32_t), cudaMemcpyDeviceToHost,
                        ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  for (int l = 0; l <= ctx->n_levels; ++l) ctx->leaf_level_off[l] = h[l];
  ctx->n_leaves = h[ctx->n_levels];
  ctx->n_cf_leaves = h[ctx->n_levels + 1];
  ctx->pdl_fence = true;  // level kernels read the new tables before their PDL wait
  return SM_OK;
}

// neighbour tables (nbr, nbr6) of the boxes of level l from the level's
// Morton-sorted range
int sm_build_neighbours(sm_ctx *ctx, int l) {
  const int lo = ctx->level_off[l], hi = ctx->level_off[l + 1];
  const int cnt = (hi - lo) * 26;
  if (cnt == 0) return SM_OK;
  k_neighbours<<<(cnt + 255) / 256, 256, 0, ctx->stream>>>(lo, hi, l, ctx->ijk, ctx->morton, ctx->nbr, ctx->nbr6);
  ++ctx->n_launch;
  SM_CKL("neighbours");
  return SM_OK;
}

extern "C" int sm_build_octree(sm_ctx *ctx, int *n_boxes) {
  SM_RANGE();
  if (!ctx) return SM_EINVAL;
  if (!ctx->arena) return sm_fail(ctx, SM_ESTATE, "no arena bound");
  LevelOffsets lo;
  int n = 0;
  for (int l = 0; l <= ctx->lbase; ++l) {
    lo.off[l] = n;
    n += 1 << (3 * l);
  }
  lo.off[ctx->lbase + 1] = n;
  for (int l = ctx->lbase + 2; l <= SM_MAX_LEVELS; ++l) lo.off[l] = n;
  if (n > ctx->cfg.max_boxes) return sm_fail(ctx, SM_ENOMEM, "max_boxes %d < %d", ctx->cfg.max_boxes, n);
  sm_drop_graphs(ctx);
  k_build_uniform<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, ctx->lbase, lo, ctx->level, ctx->ijk,
                                                            ctx->morton, ctx->parent, ctx->child);
  ++ctx->n_launch;
  SM_CKL("build_uniform");
  for (int l = 0; l <= ctx->lbase; ++l) {
    int cnt = (lo.off[l + 1] - lo.off[l]) * 26;
    k_neighbours<<<(cnt + 255) / 256, 256, 0, ctx->stream>>>(lo.off[l], lo.off[l + 1], l, ctx->ijk,
                                                             ctx->morton, ctx->nbr, ctx->nbr6);
    ++ctx->n_launch;
  }
  SM_CKL("neighbours");
  ctx->n_boxes = n;
  ctx->n_levels = ctx->lbase + 1;
  for (int l = 0; l <= SM_MAX_LEVELS; ++l) ctx->level_off[l] = lo.off[l];
  int st = sm_rebuild_leaves(ctx);
  if (st) return st;
  if (n_boxes) *n_boxes = n;
  return SM_OK;
}

extern "C" int sm_refine_level(sm_ctx *ctx, int level, const int8_t *flags, int *n_new, int *n_dropped) {
  SM_RANGE();
  if (!ctx || !flags) return SM_EINVAL;
  if (!ctx->arena || ctx->n_levels == 0) return sm_fail(ctx, SM_ESTATE, "octree not built");
  if (level != ctx->n_levels - 1 || level >= ctx->lmax)
    return sm_fail(ctx, SM_EINVAL, "refine_level(%d): only the finest level %d below %d", level,
                   ctx->n_levels - 1, ctx->lmax);
  int lo = ctx->level_off[level], n = ctx->level_off[level + 1] - lo;
  SM_CK(cudaMemcpyAsync(ctx->dev_flags, flags, n, cudaMemcpyHostToDevice, ctx->stream));
  SM_CK(cudaMemsetAsync(ctx->dev_count, 0, 4 * sizeof(int32_t), ctx->stream));
  k_refine_accept<<<(n + 255) / 256, 256, 0, ctx->stream>>>(lo, n, ctx->dev_flags, ctx->nbr, ctx->scan_a,
                                                            ctx->dev_count);
  ++ctx->n_launch;
  k_scan<<<1, 1024, 0, ctx->stream>>>(ctx->scan_a, ctx->scan_b, n);
  ++ctx->n_launch;
  SM_CKL("refine accept");
  int32_t h[2];
  SM_CK(cudaMemcpyAsync(&h[0], ctx->scan_b + n, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaMemcpyAsync(&h[1], ctx->dev_count + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  int accepted = h[0];
  if (n_dropped) *n_dropped = h[1];
  if (n_new) *n_new = 8 * accepted;
  if (accepted == 0) return SM_OK;
  int new_lo = ctx->n_boxes;
  sm_drop_graphs(ctx);
  if (new_lo + 8 * accepted > ctx->cfg.max_boxes)
    return sm_fail(ctx, SM_ENOMEM, "max_boxes %d exceeded (%d needed)", ctx->cfg.max_boxes,
                   new_lo + 8 * accepted);
  k_make_children<<<(8 * n + 255) / 256, 256, 0, ctx->stream>>>(lo, n, new_lo, level, ctx->scan_a, ctx->scan_b,
                                                                ctx->level, ctx->ijk, ctx->morton, ctx->parent,
                                                                ctx->child);
  ++ctx->n_launch;
  int hi = new_lo + 8 * accepted;
  int cnt = (hi - new_lo) * 26;
  k_neighbours<<<(cnt + 255) / 256, 256, 0, ctx->stream>>>(new_lo, hi, level + 1, ctx->ijk, ctx->morton,
                                                           ctx->nbr, ctx->nbr6);
  ++ctx->n_launch;
  SM_CKL("make children");
  ctx->n_boxes = hi;
  ctx->n_levels = level + 2;
  for (int l = level + 2; l <= SM_MAX_LEVELS; ++l) ctx->level_off[l] = hi;
  return sm_rebuild_leaves(ctx);
}

extern "C" int sm_get_tables(const sm_ctx *ctx, sm_tables *out) {
  if (!ctx || !out) return SM_EINVAL;
  out->n_boxes = ctx->n_boxes;
  out->n_levels = ctx->n_levels;
  out->n_leaves = ctx->n_leaves;
  for (int l = 0; l <= SM_MAX_LEVELS; ++l) out->level_offset[l] = ctx->level_off[l];
  out->level = ctx->level;
  out->ijk = ctx->ijk;
  out->morton = ctx->morton;
  out->parent = ctx->parent;
  out->child = ctx->child;
  out->nbr = ctx->nbr;
  out->leaf = ctx->leaf;
  return SM_OK;
}

// ---------------------------------------------------------------------------
// fields
// ---------------------------------------------------------------------------
static double *var_ptr(const sm_ctx *ctx, int var) {
  switch (var) {
    case SM_PHI: return ctx->phi;
    case SM_RHS: return ctx->rhs;
    case SM_RES: return ctx->res;
    case SM_NE: return ctx->nbuf[ctx->ncur];
    case SM_NI: return ctx->ibuf[ctx->ncur];
    case SM_EMAG: return ctx->emag;
    case SM_RHO: return ctx->rho;
    default: return nullptr;
  }
}

extern "C" int sm_var_layout(const sm_ctx *ctx, int var, void **dev_ptr, int *ld, int *n_boxes) {
  if (!ctx || !dev_ptr || !ctx->arena) return SM_EINVAL;
  double *p = var_ptr(ctx, var);
  if (!p) return SM_EINVAL;
  *dev_ptr = p;
  if (ld) *ld = CELLS;
  if (n_boxes) *n_boxes = ctx->n_boxes;
  return SM_OK;
}

extern "C" int sm_var_ptr(const sm_ctx *ctx, int var, void **dev_ptr) {
  if (!ctx || !dev_ptr || !ctx->arena) return SM_EINVAL;
  double *p = var_ptr(ctx, var);
  if (!p) return SM_EINVAL;
  *dev_ptr = p;
  return SM_OK;
}

extern "C" int sm_upload(sm_ctx *ctx, int var, const double *host, int n_boxes) {
  if (!ctx || !host || !ctx->arena) return SM_EINVAL;
  double *p = var_ptr(ctx, var);
  if (!p || n_boxes < 0 || n_boxes > ctx->n_boxes)
    return sm_fail(ctx, SM_EINVAL, "upload: bad var %d or n_boxes %d", var, n_boxes);
  SM_CK(cudaMemcpyAsync(p, host, sizeof(double) * CELLS * (size_t)n_boxes, cudaMemcpyHostToDevice,
                        ctx->stream));
  return SM_OK;
}

extern "C" int sm_download(sm_ctx *ctx, int var, double *host, int n_boxes) {
  if (!ctx || !host || !ctx->arena) return SM_EINVAL;
  double *p = var_ptr(ctx, var);
  if (!p || n_boxes < 0 || n_boxes > ctx->n_boxes)
    return sm_fail(ctx, SM_EINVAL, "download: bad var %d or n_boxes %d", var, n_boxes);
  SM_CK(cudaMemcpyAsync(host, p, sizeof(double) * CELLS * (size_t)n_boxes, cudaMemcpyDeviceToHost,
                        ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  return SM_OK;
}

extern "C" int sm_set_table(sm_ctx *ctx, int n, double e_max, const double *mu, const double *diff,
                            const double *alpha) {
  if (!ctx || !mu || !diff || !alpha || n < 2 || n > 4096 || !(e_max > 0.0)) return SM_EINVAL;
  if (!ctx->arena) return sm_fail(ctx, SM_ESTATE, "no arena bound");
  // each table and its slopes t[i+1] - t[i] (the FP64 differences that
  // linear interpolation forms, computed once here)
  std::vector<double> all(6 * 4096, 0.0);
  const double *src[3] = {mu, diff, alpha};
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < n; ++i) {
      all[4096 * k + i] = src[k][i];
      all[4096 * (3 + k) + i] = i + 1 < n ? src[k][i + 1] - src[k][i] : 0.0;
    }
  SM_CK(cudaMemcpyAsync(ctx->tab, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice, ctx->stream));
  // the host arrays may be released right after the call
  SM_CK(cudaStreamSynchronize(ctx->stream));
  ctx->tab_n = n;
  ctx->tab_emax = e_max;
  return SM_OK;
}

// ---------------------------------------------------------------------------
// check of the integer-pipe FP64 <-> FP32 conversions against the hardware
// ---------------------------------------------------------------------------
namespace {

// SplitMix64 output function of counter x (Steele, Lea, Flood 2014)
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_check_cvt(long long n, unsigned long long seed, unsigned long long *__restrict__ count) {
  unsigned long long bad_d = 0, bad_f = 0, bad_x = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long x = splitmix64(seed + (unsigned long long)i);
    const int mode = (int)(i & 3);
    if (mode) {  // exponent near the binary32 range, then fraction tails at the rounding boundary
      const unsigned long long ex = 1023ull - 130ull + (x >> 55) % 261ull;
      x = (x & 0x800fffffffffffffull) | (ex << 52);
      if (mode == 2) x = (x & ~0x1fffffffull) | 0x10000000ull;
      if (mode == 3) {
        const unsigned long long tails[6] = {0x0fffffffull, 0x10000001ull, 0x1fffffffull, 0ull, 1ull, 0x10000000ull};
        x = (x & ~0x1fffffffull) | tails[(x >> 40) % 6];
        if ((x >> 45) & 1) x |= 0x000fffffe0000000ull;  // all kept fraction bits set: carry into the exponent
      }
    }
    const double d = __longlong_as_double((long long)x);
    const float a = cvt_f64_f32_rn(d), b = __double2float_rn(d);
    if (__float_as_uint(a) != __float_as_uint(b) && !(isnan(a) && isnan(b))) ++bad_d;
    const float f = __uint_as_float((unsigned)(x >> 32) ^ (unsigned)x);
    const double c = cvt_f32_f64(f), e = (double)f;
    if (__double_as_longlong(c) != __double_as_longlong(e) && !(isnan(c) && isnan(e))) ++bad_f;
    // fixed point on the grid 2^(E - 1080), E from e to e + 70: reference by
    // exact FP64 scaling, floor and the tie rule
    const unsigned long long z = splitmix64(splitmix64(x));
    int ez = (int)((z >> 52) & 0x7ffull);
    if (ez == 0x7ff) ez = 0x7fe;
    if (mode == 3) ez = 0;  // subnormals and zero
    const unsigned long long bz = (z & 0x800fffffffffffffull) | ((unsigned long long)ez << 52);
    const int E = (ez ? ez : 1) + (int)((z >> 8) % 71ull);
    if (E <= 2046) {
      const double dz = __longlong_as_double((long long)bz), xs = ldexp(dz, 1080 - E);
      const double fl = floor(xs), fr = xs - fl;
      const double ref = (fr > 0.5 || (fr == 0.5 && xs > 0.0)) ? fl + 1.0 : fl;
      if (fix_of_bits(bz, E) != __double2ll_rn(ref)) ++bad_x;
    }
  }
  if (bad_d) atomicAdd(count, bad_d);
  if (bad_f) atomicAdd(count + 1, bad_f);
  if (bad_x) atomicAdd(count + 2, bad_x);
}

}  // namespace

// FP64 pipe throughput probe: FP64_CHAINS independent fused multiply-add
// chains per thread, iters steps each; the sum leaves through *sink only
// when it equals an impossible value, so nothing is optimised away.
constexpr int FP64_CHAINS = 8;
__global__ void __launch_bounds__(256) k_fp64_probe(long long iters, unsigned long long *sink) {
  double x[FP64_CHAINS];
  const double a = 1.0 + 1e-9 * threadIdx.x, b = 1e-7 * blockIdx.x;
#pragma unroll
  for (int c = 0; c < FP64_CHAINS; ++c) x[c] = 0.5 + 0.01 * c;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < FP64_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < FP64_CHAINS; ++c) s += x[c];
  if (s == -1.0) sink[0] = (unsigned long long)__double_as_longlong(s);
}

extern "C" int sm_fp64_probe(long long iters, unsigned long long *d_scratch, double *fma_per_s, double *ms_out,
                             void *stream) {
  if (iters < 1 || !d_scratch || !fma_per_s) return SM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SM_ECUDA;
  const int grid = 8 * sms, block = 256;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return SM_ECUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return SM_ECUDA;
  }
  k_fp64_probe<<<grid, block, 0, st>>>(iters / 8 + 1, d_scratch);  // warm-up
  cudaEventRecord(a, st);
  k_fp64_probe<<<grid, block, 0, st>>>(iters, d_scratch);
  cudaEventRecord(b, st);
  float ms = 0.f;
  const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms > 0.f;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!ok) return SM_ECUDA;
  *fma_per_s = (double)grid * block * FP64_CHAINS * (double)iters / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return SM_OK;
}

extern "C" int sm_check_conversions(long long n, unsigned long long seed, unsigned long long *d_scratch,
                                    unsigned long long *mismatches, void *stream) {
  if (n < 0 || !d_scratch || !mismatches) return SM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_scratch, 0, 3 * sizeof(unsigned long long), st) != cudaSuccess) return SM_ECUDA;
  if (n > 0) k_check_cvt<<<1216, 256, 0, st>>>(n, seed, d_scratch);
  if (cudaGetLastError() != cudaSuccess) return SM_ECUDA;
  if (cudaMemcpyAsync(mismatches, d_scratch, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SM_ECUDA;
  return SM_OK;
}

