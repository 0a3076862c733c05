// lbm_launch.h -- host-side launchers of the step kernels (one set per lattice).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include "lbm_device.cuh"

namespace lbm {
#define LBM_DECLARE_LAUNCHERS(Q)                                                               \
  void launch_bulk_q##Q(int st, const Params& p, int rows, bool pairs, dim3 g, dim3 b,         \
                        cudaStream_t s, int prio);                                             \
  void launch_wall_q##Q(int st, const Params& p, bool regularized, dim3 g, dim3 b,              \
                        cudaStream_t s, int prio);                                             \
  void launch_bulk_tma_q##Q(int st, const Params& p, const CUtensorMap& tm, int zchunk,        \
                            cudaStream_t s);                                                   \
  void launch_init_q##Q(int st, const Params& p, int grid, const double* rho, const double* u, \
                        const double* nt, double rho0, double ucv, double nucv, cudaStream_t s); \
  void launch_fields_q##Q(int st, const Params& p, int grid, double* rho, double* u,          \
                          double* nut, double* nt, double rho0, double vel, double visc,       \
                          cudaStream_t s);                                                     \
  void launch_reduce_q##Q(int st, const Params& p, int blocks, double* partial,              \
                          long long chunk, cudaStream_t s);
LBM_DECLARE_LAUNCHERS(9)
LBM_DECLARE_LAUNCHERS(19)
#undef LBM_DECLARE_LAUNCHERS

void launch_reduce_final(const double* partial, int nblocks, double* out, cudaStream_t s);
// box width of the TMA tile for a storage element size (16-byte aligned start)
inline int tma_box_width(size_t esz) { return 32 + 2 * (int)(16 / esz); }
void launch_wall_stats(const Params& p, double* prev, double* out, cudaStream_t s);
}  // namespace lbm
