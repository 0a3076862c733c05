// lbm_ctx.h -- the context object behind the opaque lbm_ctx handle.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"

struct lbm_ctx {
  lbm_config cfg;
  lbm_bc bc[6];
  int Q = 0, st = 0;
  size_t esz = 4, rsz = 4;         // storage / compute element size
  int nx = 0, ny = 0, nz = 0, pitch = 0;
  long long ncell = 0;             // padded cells (pitch * ny * nz)
  long long ncells = 0;            // cells (nx * ny * nz)
  double dt = 0, ucv = 0, nucv = 0, nu_lb = 0;
  double F_lb[3] = {0, 0, 0};
  cudaStream_t stream = nullptr;   // caller's stream
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side_stream = nullptr;  // wall pre-pass branch of a step
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int prio_hi = 0;                     // greatest stream priority of the device
  int sms = 152;                       // streaming multiprocessors of the device
  void* f[2] = {nullptr, nullptr};
  void* v[2] = {nullptr, nullptr};   // SA-field records (u_x, u_y, u_z, nu_tilde) per cell
  double* utau[2] = {nullptr, nullptr};
  void* uw[2] = {nullptr, nullptr};
  void* rhow[2] = {nullptr, nullptr};
  void* invd2 = nullptr;   // 1 / d^2 of the SA model per (y, x), compute type, [y * pitch + x]
  double* utau_prev = nullptr;
  unsigned* flags = nullptr;
  unsigned last_flags = 0;
  unsigned newton_count = 0;        // flags[1] at the last check
  double* partial = nullptr;       // FP64 reduction scratch: red_blocks * RED_VALS
  int red_blocks = 0;
  long long red_chunk = 0;
  double* red_out = nullptr;
  double* staging = nullptr;       // device staging of host transfers (doubles)
  size_t staging_count = 0;
  int cur = 0;                     // buffer holding the current state
  bool ready = false;
  bool finalized = false;
  long long steps_done = 0;
  unsigned long long launches = 0;   // kernels launched (graph replays included)
  unsigned long long graph_launches[2] = {0, 0};   // kernels in each captured graph
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  bool gvalid[2] = {false, false};
  lbm::Params base;
  CUtensorMap tmap[2];                 // population buffer k as a 4-D tensor [q][z][y][x]
  bool tma_ok = false;                 // inner rows use the TMA-staged kernel
#ifndef LBM_TMA_ZCHUNK
#define LBM_TMA_ZCHUNK 8
#endif
  int tma_zchunk = LBM_TMA_ZCHUNK;     // z planes marched by one block
  long long wait_limit = 1LL << 24;    // polls of a bounded device-side wait (Params::wait_limit)
  std::string err;
  std::vector<void*> allocs;
};

void lbm_ctx_set_error(lbm_ctx* c, const char* fmt, ...);
lbm_status lbm_ctx_finalize(lbm_ctx* c);
lbm::Params lbm_ctx_params(const lbm_ctx* c, int src);
// returns the row-set argument of the launch (rows, with ROWS_ZY for the swapped block order)
int lbm_ctx_bulk_launch_dims(const lbm_ctx* c, int rows, dim3* g, dim3* b);
bool lbm_ctx_bulk_pairs(const lbm_ctx* c, int rows);
