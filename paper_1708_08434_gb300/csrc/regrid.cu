// regrid.cu -- refinement criterion (Sec. 2.5, Eq. 8) and regridding of
// the octree: per-box flags from |E| computed on the GPU, a new box set
// under proper nesting (Sec. 2.1.1), field data carried over to the new box
// numbering and prolonged into new boxes.
#include <string.h>

#include <algorithm>
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

static uint64_t h_morton(int i, int j, int k) {
  uint64_t key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= (uint64_t)((i >> b) & 1) << (3 * b);
    key |= (uint64_t)((j >> b) & 1) << (3 * b + 1);
    key |= (uint64_t)((k >> b) & 1) << (3 * b + 2);
  }
  return key;
}

struct Entry {
  int lev, i, j, k, src;
  uint64_t key;
};

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
  if (!ctx || !flags) return SM_EINVAL;
  if (!ctx->arena || ctx->n_levels == 0) return sm_fail(ctx, SM_ESTATE, "octree not built");
  int st;
  // densities of refined boxes = mean of their children, on the old mesh
  if ((st = sm_restrict_pair(ctx, ctx->nbuf[ctx->ncur], ctx->ibuf[ctx->ncur]))) return st;
  const int n = ctx->n_boxes;
  std::vector<int32_t> lev(n), ijk(3 * (size_t)n), par(n), chl(8 * (size_t)n), nbr(26 * (size_t)n);
  std::vector<uint64_t> mort(n);
  SM_CK(cudaMemcpyAsync(lev.data(), ctx->level, 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaMemcpyAsync(ijk.data(), ctx->ijk, 12 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaMemcpyAsync(par.data(), ctx->parent, 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaMemcpyAsync(chl.data(), ctx->child, 32 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaMemcpyAsync(nbr.data(), ctx->nbr, 104 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaMemcpyAsync(mort.data(), ctx->morton, 8 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
  SM_CK(cudaStreamSynchronize(ctx->stream));
  auto leafb = [&](int b) { return chl[8 * (size_t)b] < 0; };
  // refinement: flagged leaves below the maximum level whose 26 neighbour
  // positions of their level hold a box or lie outside the domain
  std::vector<char> ref(n, 0), der(n, 0);
  int nref = 0, nder = 0, ndrop = 0;
  for (int b = 0; b < n; ++b) {
    if (!leafb(b) || flags[b] <= 0 || lev[b] >= ctx->lmax) continue;
    bool ok = true;
    for (int d = 0; d < 26; ++d) ok = ok && nbr[26 * (size_t)b + d] != -2;
    if (ok) ref[b] = 1, ++nref;
    else ++ndrop;
  }
  // derefinement: boxes whose 8 children are leaves flagged -1, unless a
  // non-sibling neighbour of a child has or gets children
  for (int p = 0; p < n; ++p) {
    if (leafb(p)) continue;
    bool ok = true;
    for (int c = 0; c < 8 && ok; ++c) {
      const int ch = chl[8 * (size_t)p + c];
      ok = leafb(ch) && flags[ch] < 0;
    }
    for (int c = 0; c < 8 && ok; ++c) {
      const int ch = chl[8 * (size_t)p + c];
      for (int d = 0; d < 26 && ok; ++d) {
        const int nb = nbr[26 * (size_t)ch + d];
        if (nb >= 0 && par[nb] != p && (!leafb(nb) || ref[nb])) ok = false;
      }
    }
    if (ok) der[p] = 1, ++nder;
  }
  if (n_refined) *n_refined = nref;
  if (n_derefined) *n_derefined = nder;
  if (n_dropped) *n_dropped = ndrop;
  if (nref == 0 && nder == 0) return SM_OK;
  // new box set in (level, Morton) order
  std::vector<Entry> e;
  e.reserve(n + 8 * (size_t)nref);
  for (int b = 0; b < n; ++b) {
    if (par[b] >= 0 && der[par[b]]) continue;
    e.push_back({lev[b], ijk[3 * (size_t)b], ijk[3 * (size_t)b + 1], ijk[3 * (size_t)b + 2], b, mort[b]});
    if (!ref[b])
      continue;
    for (int c = 0; c < 8; ++c) {
      const int ci = 2 * ijk[3 * (size_t)b] + (c & 1), cj = 2 * ijk[3 * (size_t)b + 1] + ((c >> 1) & 1),
                ck = 2 * ijk[3 * (size_t)b + 2] + (c >> 2);
      e.push_back({lev[b] + 1, ci, cj, ck, -1, h_morton(ci, cj, ck)});
    }
  }
  std::sort(e.begin(), e.end(), [](const Entry &a, const Entry &b) {
    return a.lev != b.lev ? a.lev < b.lev : a.key < b.key;
  });
  const int m = (int)e.size();
  if (m > ctx->cfg.max_boxes) return sm_fail(ctx, SM_ENOMEM, "max_boxes %d exceeded (%d needed)", ctx->cfg.max_boxes, m);
  int nlev = 0;
  for (const Entry &x : e) nlev = std::max(nlev, x.lev + 1);
  int off[SM_MAX_LEVELS + 2];
  for (int l = 0, b = 0; l <= SM_MAX_LEVELS + 1; ++l) {
    while (b < m && e[b].lev < l) ++b;
    off[l] = b;
  }
  auto find = [&](int l, uint64_t key) -> int {
    if (l < 0 || l >= nlev) return -1;
    int a = off[l], z = off[l + 1] - 1;
    while (a <= z) {
      const int mid = (a + z) / 2;
      if (e[mid].key == key) return mid;
      if (e[mid].key < key) a = mid + 1;
      else z = mid - 1;
    }
    return -1;
  };
  std::vector<int32_t> nlv(m), nijk(3 * (size_t)m), npar(m), nchl(8 * (size_t)m, -1), src(m), fresh;
  std::vector<uint64_t> nmort(m);
  for (int b = 0; b < m; ++b) {
    nlv[b] = e[b].lev;
    nijk[3 * (size_t)b] = e[b].i;
    nijk[3 * (size_t)b + 1] = e[b].j;
    nijk[3 * (size_t)b + 2] = e[b].k;
    nmort[b] = e[b].key;
    src[b] = e[b].src;
    if (e[b].src < 0) fresh.push_back(b);
    npar[b] = e[b].lev > 0 ? find(e[b].lev - 1, e[b].key >> 3) : -1;
    if (find(e[b].lev + 1, e[b].key << 3) >= 0)
      for (int c = 0; c < 8; ++c) nchl[8 * (size_t)b + c] = find(e[b].lev + 1, (e[b].key << 3) | (uint64_t)c);
  }
  sm_drop_graphs(ctx);
  // fields to the new numbering (new boxes zero), through the scratch array
  // of the previous cycle's potential
  int32_t *dsrc = ctx->scan_b, *dlist = ctx->scan_a;
  SM_CK(cudaMemcpyAsync(dsrc, src.data(), 4 * (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
  double *vars[6] = {ctx->phi, ctx->rhs, ctx->emag, ctx->rho, ctx->nbuf[ctx->ncur], ctx->ibuf[ctx->ncur]};
  for (double *x : vars) {
    k_regrid_gather<<<m, CELLS, 0, ctx->stream>>>(dsrc, x, ctx->old);
    ++ctx->n_launch;
    SM_CK(cudaMemcpyAsync(x, ctx->old, sizeof(double) * CELLS * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  SM_CKL("regrid gather");
  // tables of the new mesh; neighbours and the leaf list on the device
  SM_CK(cudaMemcpyAsync(ctx->level, nlv.data(), 4 * (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
  SM_CK(cudaMemcpyAsync(ctx->ijk, nijk.data(), 12 * (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
  SM_CK(cudaMemcpyAsync(ctx->morton, nmort.data(), 8 * (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
  SM_CK(cudaMemcpyAsync(ctx->parent, npar.data(), 4 * (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
  SM_CK(cudaMemcpyAsync(ctx->child, nchl.data(), 32 * (size_t)m, cudaMemcpyHostToDevice, ctx->stream));
  ctx->n_boxes = m;
  ctx->n_levels = nlev;
  for (int l = 0; l <= SM_MAX_LEVELS; ++l) ctx->level_off[l] = off[l];
  for (int l = 0; l < nlev; ++l)
    if ((st = sm_build_neighbours(ctx, l))) return st;
  if ((st = sm_rebuild_leaves(ctx))) return st;
  // potential and densities of the new boxes from their parents
  if (!fresh.empty()) {
    SM_CK(cudaMemcpyAsync(dlist, fresh.data(), 4 * fresh.size(), cudaMemcpyHostToDevice, ctx->stream));
    k_regrid_prolong<<<(int)fresh.size(), CELLS, 0, ctx->stream>>>(dlist, ctx->parent, ctx->ijk, ctx->nbr6, ctx->bc,
                                                                  ctx->phi, ctx->nbuf[ctx->ncur],
                                                                  ctx->ibuf[ctx->ncur], ctx->dscal + SC_ERR);
    ++ctx->n_launch;
    SM_CKL("regrid prolong");
  }
  SM_CK(cudaStreamSynchronize(ctx->stream));
  return SM_OK;
}
