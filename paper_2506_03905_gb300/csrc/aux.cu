// aux.cu -- non-templated reductions: final sum of the FP64 partials and the
// wall-node u_tau statistics (mean per face, largest relative change).
#include "lbm_kernels.cuh"
#include "lbm_launch.h"

namespace lbm {

__global__ void k_reduce_final(const double* partial, int nblocks, double* out) {
  // one thread per value, block order: deterministic
  const int v = threadIdx.x;
  if (v >= RED_VALS) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[b * RED_VALS + v];
  out[v] = s;
}

__global__ void k_wall_stats(const Params p, double* prev, double* out) {
  __shared__ double sh[2][256];
  double acc[2] = {0.0, 0.0};  // [0] sum of u_tau, [1] max relative change
  for (int f = 0; f < 2; ++f) {
    acc[0] = 0.0;
    const int n = p.wall[f] ? p.nwall[f] : 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const double ut = p.utau[f][k];
      const double pv = prev[f * (long long)p.nx * p.nz + k];
      acc[0] += ut;
      if (ut > 0.0) acc[1] = fmax(acc[1], fabs(ut - pv) / ut);
      if (!isfinite(ut)) atomicOr(p.flags, FLAG_NONFINITE);
      prev[f * (long long)p.nx * p.nz + k] = ut;
    }
    sh[0][threadIdx.x] = acc[0];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = n > 0 ? sh[0][0] / n : 0.0;
    __syncthreads();
  }
  sh[1][threadIdx.x] = acc[1];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[2] = sh[1][0];
}

void launch_reduce_final(const double* partial, int nblocks, double* out, cudaStream_t s) {
  k_reduce_final<<<1, 32, 0, s>>>(partial, nblocks, out);
}

void launch_wall_stats(const Params& p, double* prev, double* out, cudaStream_t s) {
  k_wall_stats<<<1, 256, 0, s>>>(p, prev, out);
}

}  // namespace lbm
