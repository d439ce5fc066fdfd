// noalloc.cu -- exact Poisson solves on single 8^3 boxes that allocate no
// memory.
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns every byte of device memory (a caching allocator or a
// memory pool it must not bypass), code that runs inside a region where
// allocation is forbidden or would synchronise the device, and embedders
// that only hand over their own input and output buffers.  For them
// sm_box_solve_noalloc solves the 7-point Poisson problem of many single
// boxes with the same eigenbasis method as the level-0 solve of the
// multigrid cycle, keeping its only scratch (one eigenbasis per problem) in
// the file-scope device array below instead of in a context arena.
#include <math.h>
#include <mutex>

#include "sm_internal.cuh"

using namespace sm;

// one eigenbasis per problem: 3 axes x (8x8 vectors + 8 eigenvalues)
#define SMX_BASIS_DOUBLES (3 * 64 + 3 * 8)

// Scratch of every call, on every device that loads the library, held
// until the process exits: SM_NOALLOC_MAX_PROBLEMS x 1728 bytes = 1.77 MB.
static __device__ __align__(256) double g_box_scratch[SM_NOALLOC_MAX_PROBLEMS * SMX_BASIS_DOUBLES];

// device address of g_box_scratch per device ordinal (at most
// SMX_MAX_DEVICES devices).  It is looked up on a device's first call and
// again on every call made outside a stream capture, so a context reset
// (cudaDeviceReset), after which the module is reloaded and the array may
// sit elsewhere, is picked up by the next uncaptured call; a captured call
// uses the address of the last uncaptured one.
#define SMX_MAX_DEVICES 64
static std::mutex g_scratch_mtx;
static double *g_scratch_ptr[SMX_MAX_DEVICES];
static bool g_scratch_ready[SMX_MAX_DEVICES];

static int scratch_address(cudaStream_t stream, double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SM_ECUDA;
  }
  if (dev < 0 || dev >= SMX_MAX_DEVICES) return SM_EINVAL;  // beyond the per-device address table
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return SM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mtx);
  if (!g_scratch_ready[dev] || cs == cudaStreamCaptureStatusNone) {
    if (cs != cudaStreamCaptureStatusNone) return SM_ECUDA;  // first call of the device inside a capture
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_box_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return SM_ECUDA;
    }
    g_scratch_ptr[dev] = (double *)p;
    g_scratch_ready[dev] = true;
  }
  *out = g_scratch_ptr[dev];
  return SM_OK;
}

// One block of 512 threads per problem.  Threads 0..23 write the problem's
// eigenbasis (cosine / sine / quarter-wave sine family per axis, chosen by
// that axis' two boundary types) into its scratch slot; after a block
// barrier every thread reads it back, folds the Dirichlet values into the
// right-hand side, transforms to the eigenbasis, divides by the eigenvalues
// of the 7-point operator and transforms back.
__global__ void __launch_bounds__(512) k_box_solve_noalloc(const double *__restrict__ f, double *__restrict__ phi,
                                                           const int32_t *__restrict__ bc_type,
                                                           const double *__restrict__ bc_val, double h2,
                                                           double *__restrict__ scratch) {
  __shared__ double x[CELLS], y[CELLS], V[3][64], lam[3][8];
  int p = blockIdx.x, t = threadIdx.x;
  double *basis = scratch + (size_t)p * SMX_BASIS_DOUBLES;
  const int32_t *bt = bc_type + 6 * p;
  const double *bv = bc_val + 6 * p;
  if (t < 3 * NC) {
    int a = t / NC, m = t % NC;
    int lo = bt[2 * a] != 0, hi = bt[2 * a + 1] != 0;
    double v[NC], nrm = 0.0;
    for (int i = 0; i < NC; ++i) {
      double s = (i + 0.5) / NC;
      if (!lo && !hi) v[i] = cospi(m * s);
      else if (lo && hi) v[i] = sinpi((m + 1) * s);
      else if (lo) v[i] = sinpi((m + 0.5) * s);
      else v[i] = sinpi((m + 0.5) * (NC - i - 0.5) / NC);
      nrm += v[i] * v[i];
    }
    double th = (!lo && !hi) ? m : ((lo && hi) ? m + 1 : m + 0.5);
    double sn = sinpi(th / (2.0 * NC));
    nrm = rsqrt(nrm);
    for (int i = 0; i < NC; ++i) basis[a * 64 + i * 8 + m] = v[i] * nrm;
    basis[192 + a * 8 + m] = -4.0 * sn * sn;
  }
  __syncthreads();
  if (t < 192) V[t / 64][t % 64] = basis[t];
  if (t < 24) lam[t / 8][t % 8] = basis[192 + t];
  int c[3] = {t & 7, (t >> 3) & 7, t >> 6};
  double r = f[(size_t)p * CELLS + t];
  for (int fc = 0; fc < 6; ++fc) {
    int q = c[fc >> 1] + ((fc & 1) ? 1 : -1);
    if ((q < 0 || q >= NC) && bt[fc]) r -= 2.0 * bv[fc] / h2;
  }
  x[t] = r;
  __syncthreads();
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
  double ev = lam[0][c[0]] + lam[1][c[1]] + lam[2][c[2]];
  // a problem without a Dirichlet face has a zero eigenvalue (the
  // constant mode); that mode is set to zero
  y[t] = ev != 0.0 ? acc * h2 / ev : 0.0;
  __syncthreads();
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
  phi[(size_t)p * CELLS + t] = acc;
}

extern "C" int sm_box_solve_noalloc(double length, int n_problems, const int32_t *bc_type, const double *bc_val,
                                    const double *f, double *phi, void *stream) {
  if (n_problems > SM_NOALLOC_MAX_PROBLEMS) return SM_ENOMEM;  // more than the fixed scratch holds
  if (n_problems < 0 || !(length > 0.0)) return SM_EINVAL;
  if (n_problems > 0 && (!bc_type || !bc_val || !f || !phi)) return SM_EINVAL;
  double *scratch = nullptr;
  int st = scratch_address((cudaStream_t)stream, &scratch);
  if (st) return st;
  if (n_problems == 0) return SM_OK;
  double h = length / NC;
  k_box_solve_noalloc<<<n_problems, 512, 0, (cudaStream_t)stream>>>(f, phi, bc_type, bc_val, h * h, scratch);
  if (cudaGetLastError() != cudaSuccess) return SM_ECUDA;
  return SM_OK;
}
