// K5: convergence and residual reductions in FP64, in a fixed order.
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

__global__ void __launch_bounds__(kThreads)
reduce_grid_kernel(const float* __restrict__ u, const float* __restrict__ prev, int nx, int ny,
                   double* __restrict__ partial) {
  double sd = 0.0, sp = 0.0, rmax = 0.0, rsq = 0.0;
  for (int iy = blockIdx.x; iy < ny; iy += gridDim.x) {
    const float* row = u + (size_t)iy * nx;
    const bool inner_row = iy > 0 && iy < ny - 1;
    for (int ix = threadIdx.x; ix < nx; ix += kThreads) {
      const float c = row[ix];
      if (prev) {
        const float p = prev[(size_t)iy * nx + ix];
        const double d = (double)c - (double)p;
        sd += d * d;
        sp += (double)p * (double)p;
      }
      if (inner_row && ix > 0 && ix < nx - 1) {
        const double r = (double)row[ix + 1] + (double)row[ix - 1] + (double)row[ix + nx] +
                         (double)row[ix - (size_t)nx] - 4.0 * (double)c;
        rmax = fmax(rmax, fabs(r));
        rsq += r * r;
      }
    }
  }
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
                          cudaStream_t st) {
  reduce_grid_kernel<<<kReduceBlocks, kThreads, 0, st>>>(u, prev, nx, ny, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<1, kReduceBlocks, 0, st>>>(partial, out);
  return cudaGetLastError();
}

}  // namespace mf
