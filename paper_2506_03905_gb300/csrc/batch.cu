// batch.cu -- batched sweeps: many independent lattices advanced by one
// persistent, cooperative kernel launch (see include/lbm.h).
//
// Work is split into items: phase A items are chunks of wall nodes of one y
// face of one instance, phase B items are ranges of cells of one instance.
// Every warp of the persistent grid walks the item lists with a stride of the
// number of warps in the grid; a grid barrier separates phase A (wall pre-pass of every
// instance) from phase B (bulk update of every instance) and one step from
// the next.  The barrier is an atomic counter with a generation number; its
// spin is bounded (about a second), after which it records LBM_ETIMEOUT and
// every CTA leaves the kernel.  The launch is cooperative, so all CTAs are
// resident and the barrier cannot wait on a CTA that never starts.
//
// Each instance keeps its own configuration, faces and buffers (the Params of
// its context for both buffer parities); only the storage type has to be the
// same for all instances of a batch.  The instances' buffer parities live in
// device memory and are advanced by the kernel, so a captured launch can be
// replayed without host updates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_ctx.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

struct BatchInst {
  Params p[2];   // p[k]: step reading buffer k
  int Q;
  int cur;       // buffer the next step reads (advanced by the kernel)
  int nx, ny, nz;
};

struct WorkItem {
  int inst;
  int face;      // phase A: 0 = ymin, 1 = ymax
  int begin, end;
};

struct GridBar {
  unsigned count;
  unsigned gen;
  unsigned err;
  unsigned pad;
};

constexpr long long kSpinLimit = 1LL << 24;   // x ~64 ns sleep: about one second

// Grid-wide barrier of a cooperative launch; returns false once any CTA gave up.
__device__ bool grid_sync(GridBar* bar) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bar->gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long it = 0;
      while (*vgen == g) {
        if (++it > kSpinLimit) {
          atomicOr(&bar->err, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_sh = ok && (atomicAdd(&bar->err, 0u) == 0u);
  }
  __syncthreads();
  return ok_sh != 0;
}

// Work items are taken by warps: each warp copies the parameters of its
// item's instance from global memory into its own shared-memory slot (read
// through a reference to global memory every field would be a load, repeated
// after each population store, which may alias it as far as the compiler
// knows).  Warp-private slots need only warp-level synchronisation, so a slow
// item holds up no other warp of the CTA.
constexpr int kMaxWarps = 8;   // blocks of at most 256 threads

__device__ __forceinline__ void warp_load_params(Params* dst, const Params* src, int* q_dst,
                                                 const int* q_src, int lane) {
  static_assert(sizeof(Params) % sizeof(int) == 0, "Params is copied as ints");
  __syncwarp();      // the warp is done with its previous item's copy
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int k = lane; k < (int)(sizeof(Params) / sizeof(int)); k += 32) d[k] = s[k];
  if (lane == 0) *q_dst = *q_src;
  __syncwarp();
}

// Minimum resident blocks per SM requested from the compiler for k_batch (its
// register budget; 0 leaves the choice to the compiler).  Three blocks of 256
// (<= 80 registers, a few spilled) measured fastest on GB300 for the 96-instance
// sweep.
#ifndef LBM_BATCH_MINB
#define LBM_BATCH_MINB 3
#endif
#if LBM_BATCH_MINB > 0
#define LBM_BATCH_BOUNDS __launch_bounds__(256, LBM_BATCH_MINB)
#else
#define LBM_BATCH_BOUNDS __launch_bounds__(256)
#endif

template <int ST>
__global__ void LBM_BATCH_BOUNDS k_batch(BatchInst* inst, int ninst, const WorkItem* itemsA,
                               int nA, const WorkItem* itemsB, int nB, GridBar* bar, int nsteps) {
  __shared__ Params sp[kMaxWarps];
  __shared__ int sq[kMaxWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib, nw = gridDim.x * (blockDim.x >> 5);
  for (int step = 0; step < nsteps; ++step) {
    // phase A: wall pre-pass of every instance (items of 32 wall nodes)
    for (int it = gw; it < nA; it += nw) {
      const WorkItem w = itemsA[it];
      const BatchInst& b = inst[w.inst];
      warp_load_params(&sp[wib], &b.p[(b.cur + step) & 1], &sq[wib], &b.Q, lane);
      const Params& p = sp[wib];
      const int Q = sq[wib];
      for (int node = w.begin + lane; node < w.end; node += 32) {
        if (Q == 19) wall_node<19, ST>(p, w.face, node);
        else wall_node<9, ST>(p, w.face, node);
      }
    }
    if (!grid_sync(bar)) return;
    // phase B: bulk update of every cell of every instance
    for (int it = gw; it < nB; it += nw) {
      const WorkItem w = itemsB[it];
      const BatchInst& b = inst[w.inst];
      warp_load_params(&sp[wib], &b.p[(b.cur + step) & 1], &sq[wib], &b.Q, lane);
      const Params& p = sp[wib];
      const int Q = sq[wib], nx = p.nx, nxy = p.nx * p.ny;
      for (int c = w.begin + lane; c < w.end; c += 32) {
        const int z = c / nxy, r = c - z * nxy;
        const int y = r / nx, x = r - y * nx;
        if (Q == 19) bulk_cell<19, ST, true>(p, x, y, z);
        else bulk_cell<9, ST, true>(p, x, y, z);
      }
    }
    if (!grid_sync(bar)) return;
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < ninst; i += blockDim.x) inst[i].cur = (inst[i].cur + nsteps) & 1;
  }
}

using BatchKernel = void (*)(BatchInst*, int, const WorkItem*, int, const WorkItem*, int, GridBar*,
                             int);

BatchKernel batch_kernel(int st) {
  switch (st) {
    case ST_FP32: return k_batch<ST_FP32>;
    case ST_FP16: return k_batch<ST_FP16>;
    case ST_BF16: return k_batch<ST_BF16>;
    default: return k_batch<ST_FP64>;
  }
}

std::string g_batch_err;

}  // namespace

struct lbm_batch {
  std::vector<lbm_ctx*> ctxs;
  int st = 0;
  cudaStream_t stream = nullptr;
  BatchInst* d_inst = nullptr;
  GridBar* d_bar = nullptr;
  WorkItem* d_itemsA = nullptr;
  int nA = 0;
  WorkItem* d_itemsB = nullptr;
  int nB = 0;
  int threads = 256;
  int tile = 256;         // cells per phase-B item (one warp each)
  int grid = 0;
  bool tuned = false;
  bool launched = false;  // a launch may still be running: check its barrier flag first
  bool use_graph = true;  // false if capturing the cooperative launch was refused
  cudaGraphExec_t gexec = nullptr;
  int g_nsteps = -1;
  std::vector<int> dev_cur;  // buffer parity of each instance as the device holds it
  std::string err;
};

#define BATCH_TRY(b, expr)                                                   \
  do {                                                                       \
    cudaError_t e_ = (expr);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      (b)->err = std::string(#expr " failed: ") + cudaGetErrorString(e_);    \
      return LBM_ECUDA;                                                      \
    }                                                                        \
  } while (0)

// Instances in work-item order: D3Q19 first, then D2Q9, so that the warps of
// an SM mostly run one lattice's code at a time (instruction-cache locality).
static std::vector<int> instance_order(const lbm_batch* b) {
  std::vector<int> order;
  for (int q : {19, 9})
    for (int i = 0; i < (int)b->ctxs.size(); ++i)
      if (b->ctxs[i]->Q == q) order.push_back(i);
  return order;
}

// Phase B items: ranges of `tile` cells of one instance, each advanced by one warp.
static lbm_status build_items_B(lbm_batch* b, int tile) {
  std::vector<WorkItem> items;
  for (int i : instance_order(b)) {
    const lbm_ctx* c = b->ctxs[i];
    const int n = (int)c->ncells;
    for (int a = 0; a < n; a += tile) items.push_back({i, 0, a, std::min(n, a + tile)});
  }
  if (b->d_itemsB) cudaFree(b->d_itemsB);
  b->d_itemsB = nullptr;
  b->nB = (int)items.size();
  BATCH_TRY(b, cudaMalloc(&b->d_itemsB, std::max<size_t>(1, items.size()) * sizeof(WorkItem)));
  BATCH_TRY(b, cudaMemcpy(b->d_itemsB, items.data(), items.size() * sizeof(WorkItem),
                          cudaMemcpyHostToDevice));
  b->tile = tile;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return LBM_OK;
}

// Phase A items: chunks of one warp of wall nodes of one face of one instance.
static lbm_status build_items_A(lbm_batch* b, int chunk) {
  std::vector<WorkItem> items;
  for (int i : instance_order(b)) {
    const lbm_ctx* c = b->ctxs[i];
    for (int f = 0; f < 2; ++f) {
      if (!c->base.wall[f]) continue;
      const int nw = c->base.nwall[f];
      for (int a = 0; a < nw; a += chunk) items.push_back({i, f, a, std::min(nw, a + chunk)});
    }
  }
  if (b->d_itemsA) cudaFree(b->d_itemsA);
  b->d_itemsA = nullptr;
  b->nA = (int)items.size();
  BATCH_TRY(b, cudaMalloc(&b->d_itemsA, std::max<size_t>(1, items.size()) * sizeof(WorkItem)));
  BATCH_TRY(b, cudaMemcpy(b->d_itemsA, items.data(), items.size() * sizeof(WorkItem),
                          cudaMemcpyHostToDevice));
  return LBM_OK;
}

static lbm_status set_threads(lbm_batch* b, int threads) {
  int dev = 0, sms = 0, per_sm = 0;
  BATCH_TRY(b, cudaGetDevice(&dev));
  BATCH_TRY(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BATCH_TRY(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(b->st), threads, 0));
  if (per_sm < 1) {
    b->err = "the batch kernel does not fit on an SM with this block size";
    return LBM_EUNSUPPORTED;
  }
  b->threads = threads;
  b->grid = sms * per_sm;
  lbm_status s = build_items_A(b, 32);
  if (s != LBM_OK) return s;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return LBM_OK;
}

// Enqueue one cooperative launch advancing every instance by nsteps.
static lbm_status launch(lbm_batch* b, int nsteps, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid, 1, 1);
  cfg.blockDim = dim3(b->threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BATCH_TRY(b, cudaLaunchKernelEx(&cfg, batch_kernel(b->st), b->d_inst, (int)b->ctxs.size(),
                                  (const WorkItem*)b->d_itemsA, b->nA,
                                  (const WorkItem*)b->d_itemsB, b->nB, b->d_bar, nsteps));
  return LBM_OK;
}

static lbm_status check_bar(lbm_batch* b) {
  GridBar h;
  BATCH_TRY(b, cudaMemcpyAsync(&h, b->d_bar, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  if (h.err) {
    b->err = "grid barrier of the batch kernel timed out";
    return LBM_ETIMEOUT;
  }
  return LBM_OK;
}

static void advance_host_parity(lbm_batch* b, int nsteps) {
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    lbm_ctx* c = b->ctxs[i];
    c->cur = (c->cur + nsteps) & 1;
    c->steps_done += nsteps;
    b->dev_cur[i] = (b->dev_cur[i] + nsteps) & 1;
  }
}

// A context stepped on its own (lbm_step) since the last batch launch has a
// different buffer parity than the device copy: upload the current ones.
static lbm_status sync_parity(lbm_batch* b) {
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    if (b->ctxs[i]->cur == b->dev_cur[i]) continue;
    const int cur = b->ctxs[i]->cur;
    BATCH_TRY(b, cudaMemcpyAsync(&b->d_inst[i].cur, &cur, sizeof(int), cudaMemcpyHostToDevice,
                                 b->stream));
    BATCH_TRY(b, cudaStreamSynchronize(b->stream));
    b->dev_cur[i] = cur;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, lbm_batch** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!ctxs || n < 1) {
    g_batch_err = "lbm_batch_create: need at least one context";
    return LBM_EINVAL;
  }
  lbm_batch* b = new lbm_batch();
  for (int i = 0; i < n; ++i) {
    lbm_ctx* c = ctxs[i];
    if (!c || !c->ready) {
      delete b;
      g_batch_err = "lbm_batch_create: every context must hold a state (lbm_set_fields)";
      return LBM_EINVAL;
    }
    lbm_status s = lbm_ctx_finalize(c);
    if (s != LBM_OK) {
      delete b;
      g_batch_err = "lbm_batch_create: context " + std::to_string(i) + ": " + c->err;
      return s;
    }
    if (i > 0 && c->st != ctxs[0]->st) {
      delete b;
      g_batch_err = "lbm_batch_create: all instances must share one storage type";
      return LBM_EINVAL;
    }
    b->ctxs.push_back(c);
  }
  b->st = ctxs[0]->st;
  b->stream = ctxs[0]->stream;
  for (int i = 0; i < n; ++i) b->dev_cur.push_back(ctxs[i]->cur);
  std::vector<BatchInst> hi(n);
  for (int i = 0; i < n; ++i) {
    const lbm_ctx* c = ctxs[i];
    std::memset(&hi[i], 0, sizeof(BatchInst));
    hi[i].p[0] = lbm_ctx_params(c, 0);
    hi[i].p[1] = lbm_ctx_params(c, 1);
    hi[i].Q = c->Q;
    hi[i].cur = c->cur;
    hi[i].nx = c->nx;
    hi[i].ny = c->ny;
    hi[i].nz = c->nz;
  }
  lbm_status st = LBM_OK;
  if (cudaMalloc(&b->d_inst, n * sizeof(BatchInst)) != cudaSuccess ||
      cudaMalloc(&b->d_bar, sizeof(GridBar)) != cudaSuccess) {
    g_batch_err = "lbm_batch_create: device allocation failed";
    lbm_batch_destroy(b);
    return LBM_ENOMEM;
  }
  // the contexts' pending work (state set-up) must be complete before the batch
  // reads their parameters on another order of launches
  for (lbm_ctx* c : b->ctxs) cudaStreamSynchronize(c->stream);
  if (cudaMemcpy(b->d_inst, hi.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_bar, 0, sizeof(GridBar)) != cudaSuccess) {
    g_batch_err = "lbm_batch_create: upload failed";
    lbm_batch_destroy(b);
    return LBM_ECUDA;
  }
  st = set_threads(b, 256);
  if (st == LBM_OK) st = build_items_B(b, 256);
  if (st != LBM_OK) {
    g_batch_err = b->err;
    lbm_batch_destroy(b);
    return st;
  }
  *out = b;
  return LBM_OK;
}

// Candidate block sizes and tile sizes are timed on the live state (each trial
// advances every instance by its steps) and the fastest pair is kept.
extern "C" lbm_status lbm_batch_tune(lbm_batch* b, int best[2]) {
  if (!b) return LBM_EINVAL;
  {
    lbm_status s0 = sync_parity(b);
    if (s0 != LBM_OK) return s0;
  }
  const int threads_c[2] = {128, 256};
  const int tiles_c[3] = {64, 256, 1024};   // cells per warp item
  float best_ms = 1e30f;
  int bt = b->threads, btile = b->tile;
  cudaEvent_t e0, e1;
  BATCH_TRY(b, cudaEventCreate(&e0));
  BATCH_TRY(b, cudaEventCreate(&e1));
  const int trial = 3;
  for (int t : threads_c) {
    lbm_status s = set_threads(b, t);
    if (s != LBM_OK) continue;
    for (int k : tiles_c) {
      s = build_items_B(b, k);
      if (s != LBM_OK) return s;
      s = launch(b, 1, b->stream);   // warm-up
      if (s != LBM_OK) return s;
      advance_host_parity(b, 1);
      BATCH_TRY(b, cudaEventRecord(e0, b->stream));
      s = launch(b, trial, b->stream);
      if (s != LBM_OK) return s;
      advance_host_parity(b, trial);
      BATCH_TRY(b, cudaEventRecord(e1, b->stream));
      BATCH_TRY(b, cudaEventSynchronize(e1));
      float ms = 0.f;
      BATCH_TRY(b, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        bt = t;
        btile = k;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lbm_status s = set_threads(b, bt);
  if (s == LBM_OK) s = build_items_B(b, btile);
  if (s != LBM_OK) return s;
  b->tuned = true;
  if (best) {
    best[0] = bt;
    best[1] = btile;
  }
  return check_bar(b);
}

extern "C" lbm_status lbm_batch_step(lbm_batch* b, int nsteps) {
  if (!b || nsteps < 0) return LBM_EINVAL;
  if (nsteps == 0) return LBM_OK;
  lbm_status s;
  if (b->launched) {
    // a barrier timeout of the previous launch is reported here
    s = check_bar(b);
    if (s != LBM_OK) return s;
  }
  s = sync_parity(b);
  if (s != LBM_OK) return s;
  if (!b->tuned) {
    s = lbm_batch_tune(b, nullptr);
    if (s != LBM_OK) return s;
  }
  if (!b->use_graph) {
    s = launch(b, nsteps, b->stream);
    if (s != LBM_OK) return s;
    advance_host_parity(b, nsteps);
    b->launched = true;
    return LBM_OK;
  }
  // one persistent launch per call, replayed from a graph while nsteps repeats
  if (!b->gexec || b->g_nsteps != nsteps) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    cudaStream_t cap;
    BATCH_TRY(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      s = launch(b, nsteps, cap);
      e = cudaStreamEndCapture(cap, &g);
      if (s == LBM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || !b->gexec) {
      // the cooperative launch could not be captured: launch it directly
      cudaGetLastError();
      b->use_graph = false;
      s = launch(b, nsteps, b->stream);
      if (s != LBM_OK) return s;
      advance_host_parity(b, nsteps);
      b->launched = true;
      return LBM_OK;
    }
    b->g_nsteps = nsteps;
  }
  BATCH_TRY(b, cudaGraphLaunch(b->gexec, b->stream));
  advance_host_parity(b, nsteps);
  b->launched = true;
  return LBM_OK;
}

extern "C" void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->d_bar) cudaFree(b->d_bar);
  if (b->d_itemsA) cudaFree(b->d_itemsA);
  if (b->d_itemsB) cudaFree(b->d_itemsB);
  delete b;
}

extern "C" const char* lbm_batch_last_error(const lbm_batch* b) {
  return b ? b->err.c_str() : g_batch_err.c_str();
}
