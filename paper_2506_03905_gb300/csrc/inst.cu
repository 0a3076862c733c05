// Template instantiations of the step kernels for one lattice (all storage
// types).  The build compiles this file once per lattice with -DLBM_Q=9 and
// -DLBM_Q=19; the launchers it defines are named launch_*_q9 / launch_*_q19.
#ifndef LBM_Q
#error "compile with -DLBM_Q=9 or -DLBM_Q=19"
#endif
#if LBM_Q != 9 && LBM_Q != 19
#error "LBM_Q must be 9 or 19"
#endif
#include "lbm_kernels.cuh"
#include "lbm_launch.h"

#define LBM_QCAT2(a, b) a##_q##b
#define LBM_QCAT(a, b) LBM_QCAT2(a, b)
#define LBM_QNAME(fn) LBM_QCAT(fn, LBM_Q)

namespace lbm {

// Launch with an explicit priority attribute (prio != 0), which a captured
// graph kernel node keeps; the wall branch of a step uses the highest priority
// so that it runs beside the inner-row grid instead of after it.
template <typename... A>
static void launch_prio(void (*k)(A...), dim3 g, dim3 b, cudaStream_t s, int prio, A... args) {
  if (prio == 0) {
    k<<<g, b, 0, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, args...);
}

// Inner rows with TMA staging: block 32 x 8, grid over x tiles, y tiles of the
// rows 1..ny-2 and chunks of zchunk planes; two stages of Q boxes in dynamic
// shared memory.
template <int ST>
static void bulk_tma_st(const Params& p, const CUtensorMap& tm, int zchunk, cudaStream_t s) {
  using TT = TmaTile<LBM_Q, ST>;
  const int smem = TT::SMEM_BYTES;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_bulk_tma<LBM_Q, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr_set = true;
  }
  dim3 g((p.nx + 31) / 32, (p.ny - 2 + TT::BH - 1) / TT::BH, (p.nz + zchunk - 1) / zchunk);
  dim3 b(32, TT::BH, 1);
  k_bulk_tma<LBM_Q, ST><<<g, b, smem, s>>>(p, tm, zchunk);
}

template <int ST>
static void bulk_st(const Params& p, int rows, bool pairs, dim3 g, dim3 b, cudaStream_t s, int prio) {
  // the face logic is needed unless every cell of the launch has periodic or
  // in-lattice neighbours: the inner rows (whose x-face columns of a
  // non-periodic x axis go to a separate ROWS_XEDGE launch), or every row of
  // a lattice periodic in x and y
  // (pairs: two cells per thread, and the launch shape of lbm_ctx_bulk_launch_dims
  // covers pairs of cells along x)
  const int rs = rows & ROWS_MASK;
  const bool fast = rs == ROWS_INNER || (rs == ROWS_ALL && p.px && p.py);
  if (fast && pairs) {
    if (p.collision == 0) launch_prio(k_bulk2<LBM_Q, ST, COLL_BGK>, g, b, s, prio, p, rows);
    else launch_prio(k_bulk2<LBM_Q, ST, COLL_REG>, g, b, s, prio, p, rows);
  }
  else if (fast) launch_prio(k_bulk<LBM_Q, ST, false>, g, b, s, prio, p, rows);
  else launch_prio(k_bulk<LBM_Q, ST, true>, g, b, s, prio, p, rows);
}
template <int ST>
static void wall_st(const Params& p, bool regularized, dim3 g, dim3 b, cudaStream_t s, int prio) {
  if (regularized && p.collision == 0) launch_prio(k_wall<LBM_Q, ST, WALLS_REG, COLL_BGK>, g, b, s, prio, p);
  else if (regularized) launch_prio(k_wall<LBM_Q, ST, WALLS_REG, COLL_REG>, g, b, s, prio, p);
  else launch_prio(k_wall<LBM_Q, ST, WALLS_BB>, g, b, s, prio, p);
}

#define LBM_DISPATCH(FN, ...)                       \
  switch (st) {                                     \
    case ST_FP32: FN<ST_FP32>(__VA_ARGS__); break;  \
    case ST_FP16: FN<ST_FP16>(__VA_ARGS__); break;  \
    case ST_BF16: FN<ST_BF16>(__VA_ARGS__); break;  \
    default: FN<ST_FP64>(__VA_ARGS__); break;       \
  }

void LBM_QNAME(launch_bulk)(int st, const Params& p, int rows, bool pairs, dim3 g, dim3 b,
                           cudaStream_t s, int prio) {
  LBM_DISPATCH(bulk_st, p, rows, pairs, g, b, s, prio)
}
void LBM_QNAME(launch_bulk_tma)(int st, const Params& p, const CUtensorMap& tm, int zchunk, cudaStream_t s) {
  LBM_DISPATCH(bulk_tma_st, p, tm, zchunk, s)
}
void LBM_QNAME(launch_wall)(int st, const Params& p, bool regularized, dim3 g, dim3 b, cudaStream_t s,
                           int prio) {
  LBM_DISPATCH(wall_st, p, regularized, g, b, s, prio)
}

template <int ST>
static void init_st(const Params& p, int grid, const double* rho, const double* u,
                    const double* nt, double rho0, double ucv, double nucv, cudaStream_t s) {
  k_init<LBM_Q, ST><<<grid, 256, 0, s>>>(p, rho, u, nt, rho0, ucv, nucv);
}
void LBM_QNAME(launch_init)(int st, const Params& p, int grid, const double* rho, const double* u,
                     const double* nt, double rho0, double ucv, double nucv, cudaStream_t s) {
  LBM_DISPATCH(init_st, p, grid, rho, u, nt, rho0, ucv, nucv, s)
}

template <int ST>
static void fields_st(const Params& p, int grid, double* rho, double* u, double* nut, double* nt,
                      double rho0, double vel, double visc, cudaStream_t s) {
  k_fields<LBM_Q, ST><<<grid, 256, 0, s>>>(p, rho, u, nut, nt, rho0, vel, visc);
}
void LBM_QNAME(launch_fields)(int st, const Params& p, int grid, double* rho, double* u, double* nut,
                       double* nt, double rho0, double vel, double visc, cudaStream_t s) {
  LBM_DISPATCH(fields_st, p, grid, rho, u, nut, nt, rho0, vel, visc, s)
}

template <int ST>
static void reduce_st(const Params& p, int blocks, double* partial, long long chunk, cudaStream_t s) {
  k_reduce<LBM_Q, ST><<<blocks, RED_THREADS, 0, s>>>(p, partial, chunk);
}
void LBM_QNAME(launch_reduce)(int st, const Params& p, int blocks, double* partial, long long chunk,
                       cudaStream_t s) {
  LBM_DISPATCH(reduce_st, p, blocks, partial, chunk, s)
}

}  // namespace lbm
