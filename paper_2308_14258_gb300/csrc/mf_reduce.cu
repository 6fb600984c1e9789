// K5: convergence and residual reductions, accumulated in FP64 in a fixed order.
//
// One pass over the grid accumulates, per block, sum (u - prev)^2 and sum prev^2 over
// every grid point (the relative change of Algorithm 2) and max |r|, sum r^2 of the
// 5-point residual r = u_E + u_W + u_N + u_S - 4u over interior points. Each block owns
// a fixed set of rows and reduces with a fixed shuffle tree; a single-block pass then
// folds the kReduceBlocks partials in a fixed tree, so results do not depend on timing.
#include <math.h>

#include "mf_internal.cuh"

namespace mf {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void warp_reduce(double& a, double& b, double& m, double& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
}

// Error-free sum of two FP32 values (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}

// 5-point residual of FP32 values, E + W + N + S - 4C: the partial sums are exact
// FP32 pairs (TwoSum), so the result is the exact residual rounded about once, with
// an error relative to r itself rather than to |u| (4C is exact in FP32).
__device__ __forceinline__ float residual5(float e, float w, float n, float s, float c) {
  float e1, e2, e3, e4;
  const float s1 = two_sum(e, w, e1);
  const float s2 = two_sum(n, s, e2);
  const float s3 = two_sum(s1, s2, e3);
  const float s4 = two_sum(s3, -4.0f * c, e4);
  return s4 + ((e1 + e2) + (e3 + e4));
}

// Per-point work is FP32 (FP64 throughput is low on this part); a thread's points of a
// row (up to 8 per pass) are folded into FP64 accumulators, so FP64 carries the long sums.
__global__ void __launch_bounds__(kThreads)
reduce_grid_kernel(const float* __restrict__ u, const float* __restrict__ prev, int nx, int ny,
                   double* __restrict__ partial, int residual) {
  double sd = 0.0, sp = 0.0, rmax = 0.0, rsq = 0.0;
  float fd = 0.f, fp = 0.f, fr = 0.f, fmx = 0.f;
  for (int iy = blockIdx.x; iy < ny; iy += gridDim.x) {
    const float* row = u + (size_t)iy * nx;
    const float* prow = prev ? prev + (size_t)iy * nx : nullptr;
    const bool inner_row = residual && iy > 0 && iy < ny - 1;
    // up to 8 points of the row per thread per pass, all loads issued before use; the
    // FP32 partial sums of a pass are folded into FP64
    for (int ix0 = threadIdx.x; ix0 < nx; ix0 += 8 * kThreads) {
      float c[8], pv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int ix = ix0 + k * kThreads;
        c[k] = ix < nx ? row[ix] : 0.f;
        pv[k] = (prow && ix < nx) ? prow[ix] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int ix = ix0 + k * kThreads;
        if (ix >= nx) break;
        if (prow) {
          const float d = c[k] - pv[k];
          fd = fmaf(d, d, fd);
          fp = fmaf(pv[k], pv[k], fp);
        }
        if (inner_row && ix > 0 && ix < nx - 1) {
          const float r = residual5(row[ix + 1], row[ix - 1], row[ix + nx], row[ix - (size_t)nx], c[k]);
          fmx = fmaxf(fmx, fabsf(r));
          fr = fmaf(r, r, fr);
        }
      }
      sd += (double)fd; sp += (double)fp; rsq += (double)fr;
      fd = fp = fr = 0.f;
    }
  }
  sd += (double)fd; sp += (double)fp; rsq += (double)fr;
  rmax = (double)fmx;
  __shared__ double sh[4][kThreads / 32];
  warp_reduce(sd, sp, rmax, rsq);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[0][w] = sd; sh[1][w] = sp; sh[2][w] = rmax; sh[3][w] = rsq; }
  __syncthreads();
  if (w == 0) {
    sd = l < kThreads / 32 ? sh[0][l] : 0.0;
    sp = l < kThreads / 32 ? sh[1][l] : 0.0;
    rmax = l < kThreads / 32 ? sh[2][l] : 0.0;
    rsq = l < kThreads / 32 ? sh[3][l] : 0.0;
    warp_reduce(sd, sp, rmax, rsq);
    if (l == 0) {
      double* o = partial + 4 * (size_t)blockIdx.x;
      o[0] = sd; o[1] = sp; o[2] = rmax; o[3] = rsq;
    }
  }
}

__global__ void __launch_bounds__(kReduceBlocks)
finalize_kernel(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[4][kReduceBlocks / 32];
  const double* p = partial + 4 * (size_t)threadIdx.x;
  double sd = p[0], sp = p[1], rmax = p[2], rsq = p[3];
  warp_reduce(sd, sp, rmax, rsq);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[0][w] = sd; sh[1][w] = sp; sh[2][w] = rmax; sh[3][w] = rsq; }
  __syncthreads();
  if (w == 0) {
    sd = l < kReduceBlocks / 32 ? sh[0][l] : 0.0;
    sp = l < kReduceBlocks / 32 ? sh[1][l] : 0.0;
    rmax = l < kReduceBlocks / 32 ? sh[2][l] : 0.0;
    rsq = l < kReduceBlocks / 32 ? sh[3][l] : 0.0;
    warp_reduce(sd, sp, rmax, rsq);
    if (l == 0) {
      out[0] = sd; out[1] = sp; out[2] = rmax; out[3] = rsq;
      const double num = sqrt(sd), den = sqrt(sp);
      out[4] = den == 0.0 ? (num == 0.0 ? 0.0 : INFINITY) : num / den;
    }
  }
}

}  // namespace

cudaError_t launch_reduce(const float* u, const float* prev, int nx, int ny, double* partial, double* out,
                          cudaStream_t st, bool residual) {
  reduce_grid_kernel<<<kReduceBlocks, kThreads, 0, st>>>(u, prev, nx, ny, partial, residual ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<1, kReduceBlocks, 0, st>>>(partial, out);
  return cudaGetLastError();
}

}  // namespace mf
