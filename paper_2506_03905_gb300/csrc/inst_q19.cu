// Template instantiations of the step kernels for the D3Q19 lattice (all storage types).
#include "lbm_kernels.cuh"
#include "lbm_launch.h"

namespace lbm {

template <int ST>
static void bulk_st(const Params& p, dim3 g, dim3 b, cudaStream_t s) {
  k_bulk<19, ST><<<g, b, 0, s>>>(p);
}
template <int ST>
static void wall_st(const Params& p, dim3 g, dim3 b, cudaStream_t s) {
  k_wall<19, ST><<<g, b, 0, s>>>(p);
}

#define LBM_DISPATCH(FN, ...)                       \
  switch (st) {                                     \
    case ST_FP32: FN<ST_FP32>(__VA_ARGS__); break;  \
    case ST_FP16: FN<ST_FP16>(__VA_ARGS__); break;  \
    case ST_BF16: FN<ST_BF16>(__VA_ARGS__); break;  \
    default: FN<ST_FP64>(__VA_ARGS__); break;       \
  }

void launch_bulk_q19(int st, const Params& p, dim3 g, dim3 b, cudaStream_t s) {
  LBM_DISPATCH(bulk_st, p, g, b, s)
}
void launch_wall_q19(int st, const Params& p, dim3 g, dim3 b, cudaStream_t s) {
  LBM_DISPATCH(wall_st, p, g, b, s)
}

template <int ST>
static void init_st(const Params& p, int grid, const double* rho, const double* u,
                    const double* nt, double rho0, double ucv, double nucv, cudaStream_t s) {
  k_init<19, ST><<<grid, 256, 0, s>>>(p, rho, u, nt, rho0, ucv, nucv);
}
void launch_init_q19(int st, const Params& p, int grid, const double* rho, const double* u,
                     const double* nt, double rho0, double ucv, double nucv, cudaStream_t s) {
  LBM_DISPATCH(init_st, p, grid, rho, u, nt, rho0, ucv, nucv, s)
}

template <int ST>
static void fields_st(const Params& p, int grid, double* rho, double* u, double* nut, double* nt,
                      double rho0, double vel, double visc, cudaStream_t s) {
  k_fields<19, ST><<<grid, 256, 0, s>>>(p, rho, u, nut, nt, rho0, vel, visc);
}
void launch_fields_q19(int st, const Params& p, int grid, double* rho, double* u, double* nut,
                       double* nt, double rho0, double vel, double visc, cudaStream_t s) {
  LBM_DISPATCH(fields_st, p, grid, rho, u, nut, nt, rho0, vel, visc, s)
}

template <int ST>
static void reduce_st(const Params& p, int blocks, double* partial, long long chunk, cudaStream_t s) {
  k_reduce<19, ST><<<blocks, RED_THREADS, 0, s>>>(p, partial, chunk);
}
void launch_reduce_q19(int st, const Params& p, int blocks, double* partial, long long chunk,
                       cudaStream_t s) {
  LBM_DISPATCH(reduce_st, p, blocks, partial, chunk, s)
}

}  // namespace lbm
