// noalloc.cu -- mass and momentum of a population array without any allocation.
//
// Some callers cannot allocate device memory when they need this number:
// host applications that reserve the whole device up front and hand
// libraries fixed buffers, allocators that forbid growth after start-up, or
// loops where cudaMalloc/cudaFree would synchronise the device.  For them,
// lbm_moments_noalloc computes the same FP64 sums as lbm_diagnostics
// (mass = sum of populations, momentum = sum of c_i f_i) from a population
// array the caller owns, keeping its partial sums in a fixed static device
// array instead of context scratch.
//
// The scratch array below is loaded with the library on every GPU that loads
// it and stays there until the process exits.  Its address is looked up once
// per device, on that device's first call (so the first call on a device
// should come before any stream capture), and kept for the life of the
// process: after a cudaDeviceReset the module is loaded again and the kept
// address is stale, so this entry point must not be used on a device after it
// has been reset.  All calls share it: two calls
// whose kernels overlap on the GPU (different streams, or different host
// threads on one device) race on it and must be serialised by the caller.
// Each call writes every partial sum it later reads, so nothing has to be
// cleared between calls.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_ctx.h"
#include "lbm_device.cuh"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 4096;          // partial sums held in the scratch
constexpr long long kNoAllocCellsPerBlock = 4096;  // cells summed by one block
constexpr int kNoAllocVals = 4;                   // mass, momentum x, y, z
constexpr int kMaxDevices = 64;

// 4096 blocks x 4 doubles = 128 KiB of static device memory.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks * kNoAllocVals];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

template <int Q, int ST>
__global__ void __launch_bounds__(kNoAllocThreads)
k_moments_partial(const void* f, int nx, int ny, int nz, int pitch, double* partial) {
  using L = lbm::Lat<Q>;
  using C = lbm::Codec<ST>;
  using T = typename C::T;
  __shared__ double sh[kNoAllocVals][kNoAllocThreads];
  const long long n = (long long)nx * ny * nz;
  const long long ncell = (long long)pitch * ny * nz;
  const long long b0 = blockIdx.x * kNoAllocCellsPerBlock;
  const long long b1 = b0 + kNoAllocCellsPerBlock < n ? b0 + kNoAllocCellsPerBlock : n;
  const T* fs = (const T*)f;
  double acc[kNoAllocVals] = {0.0, 0.0, 0.0, 0.0};
  for (long long k = b0 + threadIdx.x; k < b1; k += kNoAllocThreads) {
    const long long x = k % nx, y = (k / nx) % ny, z = k / ((long long)nx * ny);
    const long long id = (z * ny + y) * pitch + x;
    double m = 1.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double g = (double)C::ld(fs + i * ncell + id);
      m += g;
      jx += L::c(i, 0) * g;
      jy += L::c(i, 1) * g;
      jz += L::c(i, 2) * g;
    }
    acc[0] += m;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
  }
#pragma unroll
  for (int v = 0; v < kNoAllocVals; ++v) sh[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int v = 0; v < kNoAllocVals; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < kNoAllocVals; ++v) partial[blockIdx.x * kNoAllocVals + v] = sh[v][0];
  }
}

__global__ void k_moments_final(const double* partial, int nblocks, double* out) {
  const int v = threadIdx.x;
  if (v >= kNoAllocVals) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[b * kNoAllocVals + v];
  out[v] = s;
}

template <int Q>
void launch_partial(int st, const void* f, int nx, int ny, int nz, int pitch, double* partial,
                    int blocks, cudaStream_t s) {
  switch (st) {
    case LBM_FP32:
      k_moments_partial<Q, lbm::ST_FP32><<<blocks, kNoAllocThreads, 0, s>>>(f, nx, ny, nz, pitch, partial);
      break;
    case LBM_FP16_SHIFTED:
      k_moments_partial<Q, lbm::ST_FP16><<<blocks, kNoAllocThreads, 0, s>>>(f, nx, ny, nz, pitch, partial);
      break;
    case LBM_BF16_SHIFTED:
      k_moments_partial<Q, lbm::ST_BF16><<<blocks, kNoAllocThreads, 0, s>>>(f, nx, ny, nz, pitch, partial);
      break;
    default:
      k_moments_partial<Q, lbm::ST_FP64><<<blocks, kNoAllocThreads, 0, s>>>(f, nx, ny, nz, pitch, partial);
      break;
  }
}

// errors are reported through lbm_last_error(NULL)
lbm_status fail(lbm_status s, const std::string& msg) {
  lbm_ctx_set_error(nullptr, "%s", msg.c_str());
  return s;
}

}  // namespace

extern "C" lbm_status lbm_moments_noalloc(const void* f, int lattice, int storage, int nx, int ny,
                                          int nz, int pitch, double* out, void* stream) {
  if (!f || !out) return fail(LBM_EINVAL, "lbm_moments_noalloc: NULL population or output pointer");
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19)
    return fail(LBM_EINVAL, "lbm_moments_noalloc: lattice must be LBM_D2Q9 or LBM_D3Q19");
  if (storage < LBM_FP32 || storage > LBM_FP64)
    return fail(LBM_EINVAL, "lbm_moments_noalloc: unknown storage");
  if (nx < 1 || ny < 1 || nz < 1 || pitch < nx)
    return fail(LBM_EINVAL, "lbm_moments_noalloc: sizes must be positive and pitch >= nx");
  const long long n = (long long)nx * ny * nz;
  const long long max_cells = (long long)kNoAllocMaxBlocks * kNoAllocCellsPerBlock;
  if (n > max_cells)
    return fail(LBM_EINVAL, "lbm_moments_noalloc: " + std::to_string(n) +
                                " cells exceed the fixed scratch limit of " +
                                std::to_string(max_cells) + " cells");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return fail(LBM_ECUDA, std::string("lbm_moments_noalloc: no usable current device: ") +
                               cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(LBM_EUNSUPPORTED, "lbm_moments_noalloc: device index " + std::to_string(dev) +
                                      " is beyond the " + std::to_string(kMaxDevices) +
                                      " devices this entry point keeps an address for");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      // once per device, with that device current: the device address of the
      // static array (its host-side name is only a stand-in)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(LBM_ECUDA, std::string("lbm_moments_noalloc: cudaGetSymbolAddress failed: ") +
                                   cudaGetErrorString(e));
      g_noalloc_ptr[dev] = (double*)p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  const int blocks = (int)((n + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock);
  cudaStream_t s = (cudaStream_t)stream;
  // an error left pending by an earlier, unrelated call is reported as such, so
  // that the check after the launches sees only this call's launch errors
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(LBM_ECUDA, std::string("lbm_moments_noalloc: a CUDA error was pending before "
                                       "this call: ") + cudaGetErrorString(e));
  if (lattice == LBM_D2Q9) launch_partial<9>(storage, f, nx, ny, nz, pitch, scratch, blocks, s);
  else launch_partial<19>(storage, f, nx, ny, nz, pitch, scratch, blocks, s);
  k_moments_final<<<1, 32, 0, s>>>(scratch, blocks, out);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(LBM_ECUDA, std::string("lbm_moments_noalloc: launch failed: ") + cudaGetErrorString(e));
  return LBM_OK;
}
