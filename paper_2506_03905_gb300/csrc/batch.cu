// batch.cu -- batched sweeps: many independent lattices advanced by one
// persistent, cooperative kernel launch (see include/lbm.h).
//
// Work is split into items, each taken by one warp: chunks of 32 wall nodes
// of one y face of one instance (the wall pre-pass, kind A), ranges of cells
// of the rows without wall nodes of one instance (kind B, or kind I when all
// of them have in-lattice or periodic neighbours and take the face-free path),
// and ranges of cells of the wall rows of one instance (kind W, which read what
// the instance's A items of the same step wrote).  The D3Q19 and the D2Q9
// instances form two groups, each advanced by its own kernel (one velocity set
// per kernel keeps the code a warp may jump to small); the two launches run one
// after the other.  The items of one step of a group are listed as
//   A items of every instance, then for each instance its B / I and W items,
// and the steps of a launch follow one another.  Warps take items in that
// order from one atomic ticket counter, so every item a warp may wait on has an
// earlier ticket and is held by a running warp: no deadlock, and no grid-wide
// barrier.  The dependencies are per instance and counted per instance:
//   A(n, k) and B(n, k) need every item of step n-1 of instance k finished,
//   W(n, k) needs every A item of step n of instance k finished,
// which is what lets a warp start on one instance's next step while another
// instance is still finishing its current one.  Every wait is bounded: after
// spin_limit polls (about a second) the warp records a failure, and every warp
// leaves at its next ticket or wait; the host reports LBM_ETIMEOUT.
//
// Each instance keeps its own configuration, faces and buffers (the Params of
// its context for both buffer parities); only the storage type has to be the
// same for all instances of a batch.  The instances' buffer parities live in
// device memory and are advanced by the warp that finishes an instance's last
// item of the launch, so a captured launch can be replayed without host
// updates.  The counters are cleared by a memset captured with the launch.
//
// A second mode (lbm_batch_set_mode, or the autotuner's choice) advances the
// same items by ordinary launches, per step and group one kernel per item
// kind over every instance (k_multi_a, k_multi_cells), with the wall branch on
// a second stream; see "Multi-instance launches" below.
//
// This translation unit reads, within one launch, data that other warps wrote
// earlier in the same launch; it defines LBM_COHERENT_LOADS so that those
// loads are plain global loads, ordered by the fences around the counters.
#define LBM_COHERENT_LOADS 1

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
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
  int items;     // work items of one step
  int itemsA;    // wall pre-pass items of one step
};

// Item kinds.  KIND_A: a chunk of wall nodes (the wall pre-pass).  KIND_I:
// cells whose six neighbours are all in the lattice or periodic (the
// face-free path).  KIND_B: other cells that do not read the wall pre-pass
// (the x-face columns of a non-periodic x axis, the face rows of a lattice
// without walls).  KIND_W: the two wall rows, which read what the instance's
// A items of the same step wrote.
enum { KIND_A = 0, KIND_B = 1, KIND_W = 2, KIND_I = 3 };

// A cell item covers entries [begin, end) of a box of cells: columns
// xa + k xs (k < ncol), rows ya + j ys (j < nrow), every z plane, x fastest.
struct WorkItem {
  int inst;
  int kind;      // KIND_A / KIND_B / KIND_I / KIND_W
  int face;      // KIND_A: 0 = ymin, 1 = ymax
  int begin, end;   // wall nodes (A) or entries of the box (B, I, W)
  int xa, xs, ncol, ya, ys, nrow;
  int nz;        // planes of the box (entries: columns fastest, then planes, then rows)
};

// Control block of one launch of a lattice group, cleared before it: the ticket
// counter and the failure flag.  The per-instance counts of finished items and
// finished A items follow the two groups' blocks.
struct BatchCtl {
  unsigned long long next;
  unsigned err;
  unsigned pad;
};

constexpr int kCtlSlots = 4;    // control copies of launches in flight
constexpr long long kSpinLimit = 1LL << 24;   // x ~64 ns sleep: about one second

// Lane 0 waits until *ctr >= target; false if the wait gave up or another warp
// already failed.  spin_limit == 0 is the test setting: every wait that would
// have to poll at all gives up at once.
// Counter reads and increments with acquire / release semantics at GPU scope
// (instead of full fences around plain accesses).  The warp's other lanes are
// ordered with lane 0's accesses by __syncwarp.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned add_release(unsigned* p, unsigned a) {
  unsigned old;
  asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(a) : "memory");
  return old;
}

__device__ __forceinline__ bool wait_count(const unsigned* ctr, unsigned target, BatchCtl* ctl,
                                           long long spin_limit, int lane) {
  int ok = 1;
  if (lane == 0 && target > 0) {
    volatile const unsigned* verr = &ctl->err;
    long long it = 0;
    while (ld_acquire(ctr) < target) {   // acquire: the producers' writes are visible after it
      if (*verr) {
        ok = 0;
        break;
      }
      if (++it > spin_limit) {
        atomicOr(&ctl->err, 1u);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

// Work items are taken by warps: each warp copies the parameters of its
// item's instance from global memory into its own shared-memory slot (read
// through a reference to global memory every field would be a load, repeated
// after each population store, which may alias it as far as the compiler
// knows).  Warp-private slots need only warp-level synchronisation, so a slow
// item holds up no other warp of the CTA.
constexpr int kMaxWarps = 8;   // blocks of at most 256 threads

__device__ __forceinline__ void warp_load_params(Params* dst, const Params* src, int lane) {
  static_assert(sizeof(Params) % sizeof(int) == 0, "Params is copied as ints");
  __syncwarp();      // the warp is done with its previous item's copy
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int k = lane; k < (int)(sizeof(Params) / sizeof(int)); k += 32) d[k] = s[k];
  __syncwarp();
}

// Minimum resident blocks per SM requested from the compiler for k_batch (its
// register budget; 0 leaves the choice to the compiler).  Two blocks of 256
// (<= 128 registers) measured fastest on GB300 for the 96-instance sweep
// (FP32 21.1k MLUPS; 3 blocks / 80 registers 19.8k, 4 / 64 17.1k, 1 / 208
// 21.0k, the compiler's choice 20.0k).  Two cells per lane iteration with both
// cells' loads issued first measured slower (19.5k).
#ifndef LBM_BATCH_MINB
#define LBM_BATCH_MINB 2
#endif
#if LBM_BATCH_MINB > 0
#define LBM_BATCH_BOUNDS __launch_bounds__(256, LBM_BATCH_MINB)
#else
#define LBM_BATCH_BOUNDS __launch_bounds__(256)
#endif

// The entries c0, c0 + 32, c0 + 64, ... of a cell item's box (ncol columns of
// stride xs from xa, then the nz planes, then nrow rows of stride ys from ya)
// as cell coordinates: one division set for the first entry, then carries.
// Planes before rows: a cell's z neighbours are a row's length away in the
// entry order and its y neighbours ncol * nz entries away, instead of a whole
// plane (the re-reads then stay in L2 on large plates).
struct BoxWalk {
  int col, row, z;
  int dcol, dz;   // 32 entries = dz planes and dcol columns
  __device__ __forceinline__ BoxWalk(const WorkItem& w, int c0) {
    const int per_row = w.ncol * w.nz;
    row = c0 / per_row;
    const int r = c0 - row * per_row;
    z = r / w.ncol;
    col = r - z * w.ncol;
    dz = 32 / w.ncol;
    dcol = 32 - dz * w.ncol;
  }
  __device__ __forceinline__ int x(const WorkItem& w) const { return w.xa + col * w.xs; }
  __device__ __forceinline__ int y(const WorkItem& w) const { return w.ya + row * w.ys; }
  __device__ __forceinline__ void next(const WorkItem& w) {
    col += dcol;
    if (col >= w.ncol) {
      col -= w.ncol;
      ++z;
    }
    z += dz;
    while (z >= w.nz) {
      z -= w.nz;
      ++row;
    }
  }
};

// One kernel per lattice: the code a warp may run holds one velocity set only
// (instruction-fetch stalls dominated a kernel holding both), and the two
// launches of a batch step one after the other, each over its own instances.
template <int ST, int Q>
__global__ void LBM_BATCH_BOUNDS k_batch(BatchInst* inst, const WorkItem* items, int nitems,
                                         BatchCtl* ctl, unsigned* done, unsigned* done_a,
                                         int nsteps, long long spin_limit) {
  __shared__ Params sp[kMaxWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned long long total = (unsigned long long)nsteps * (unsigned long long)nitems;
  volatile const unsigned* verr = &ctl->err;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = *verr ? total : atomicAdd(&ctl->next, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) break;
    const int step = (int)(t / (unsigned long long)nitems);
    const WorkItem w = items[(int)(t - (unsigned long long)step * nitems)];
    BatchInst& b = inst[w.inst];
    const unsigned per = (unsigned)b.items, per_a = (unsigned)b.itemsA;
    // dependencies of this item (every counted item has an earlier ticket)
    const bool ok = w.kind == KIND_W
                        ? wait_count(&done_a[w.inst], spin_limit == 0 ? ~0u : (step + 1) * per_a, ctl,
                                     spin_limit, lane)
                        : wait_count(&done[w.inst],
                                     step == 0 ? 0u : (spin_limit == 0 ? ~0u : step * per), ctl,
                                     spin_limit, lane);
    if (!ok) break;
    warp_load_params(&sp[wib], &b.p[(b.cur + step) & 1], lane);
    const Params& p = sp[wib];
    if (w.kind == KIND_A) {
      for (int node = w.begin + lane; node < w.end; node += 32) wall_node<Q, ST>(p, w.face, node);
    } else {
      BoxWalk at(w, w.begin + lane);
      if (w.kind == KIND_I) {
        for (int c = w.begin + lane; c < w.end; c += 32, at.next(w))
          bulk_interior<Q, ST>(p, at.x(w), at.y(w), at.z);
      } else {
        for (int c = w.begin + lane; c < w.end; c += 32, at.next(w))
          bulk_cell<Q, ST, true>(p, at.x(w), at.y(w), at.z);
      }
    }
    __syncwarp();
    if (lane == 0) {
      // release: this item's writes (all lanes, ordered by the __syncwarp) before its count
      if (w.kind == KIND_A) add_release(&done_a[w.inst], 1u);
      const unsigned d = add_release(&done[w.inst], 1u) + 1u;
      // the instance's last item of this launch: no other item of it remains
      if (d == (unsigned)nsteps * per) b.cur = (b.cur + nsteps) & 1;
    }
  }
}

using BatchKernel = void (*)(BatchInst*, const WorkItem*, int, BatchCtl*, unsigned*, unsigned*, int,
                             long long);

template <int Q> BatchKernel batch_kernel_q(int st) {
  switch (st) {
    case ST_FP32: return k_batch<ST_FP32, Q>;
    case ST_FP16: return k_batch<ST_FP16, Q>;
    case ST_BF16: return k_batch<ST_BF16, Q>;
    default: return k_batch<ST_FP64, Q>;
  }
}
BatchKernel batch_kernel(int st, int q) { return q == 19 ? batch_kernel_q<19>(st) : batch_kernel_q<9>(st); }

// ---------------------------------------------------------------------------
// Multi-instance launches (mode 1).  Per step and lattice group three kernels
// run over the items of every instance, one CTA per item: the wall pre-pass
// (A items of kMultiNodes nodes) followed by the wall rows and x-face columns
// (W and B items) on a second stream, and the face-free cells (I items) on
// the batch's stream beside them; the branches join before the next step.
// The launches are direct (not captured: see step_multi).
// Kernel boundaries order the steps, so there are no device-side waits, and
// each kernel has the register budget of its own work.
// ---------------------------------------------------------------------------
#ifndef LBM_MULTI_CELLS
#define LBM_MULTI_CELLS 128
#endif
constexpr int kMultiCells = LBM_MULTI_CELLS;   // cells per B / I / W item, one per thread
constexpr int kMultiNodes = 128;   // wall nodes per A item, one per thread
enum { MK_A = 0, MK_I = 1, MK_BW = 2 };

// The instance's parameters for the item's step, copied to shared memory by the CTA.
__device__ __forceinline__ const Params& cta_params(Params* sp, const BatchInst& b, int step) {
  static_assert(sizeof(Params) % sizeof(int) == 0, "Params is copied as ints");
  const int* s = reinterpret_cast<const int*>(&b.p[(b.cur + step) & 1]);
  int* d = reinterpret_cast<int*>(sp);
  for (int k = threadIdx.x; k < (int)(sizeof(Params) / sizeof(int)); k += blockDim.x) d[k] = s[k];
  __syncthreads();
  return *sp;
}

template <int ST, int Q>
__global__ void __launch_bounds__(kMultiNodes, 8) k_multi_a(const BatchInst* inst, const WorkItem* items,
                                                            int step) {
  __shared__ Params sp;
  const WorkItem w = items[blockIdx.x];
  const Params& p = cta_params(&sp, inst[w.inst], step);
  const int node = w.begin + threadIdx.x;
  if (node < w.end) wall_node<Q, ST>(p, w.face, node);
}

template <int ST, int Q, bool FACE_FREE>
__device__ __forceinline__ void multi_cells(Params* sp, const BatchInst* inst, const WorkItem* items,
                                            int step) {
  const WorkItem w = items[blockIdx.x];
  const Params& p = cta_params(sp, inst[w.inst], step);
  const int c = w.begin + threadIdx.x;
  if (c >= w.end) return;
  const BoxWalk at(w, c);
  if (FACE_FREE) bulk_interior<Q, ST>(p, at.x(w), at.y(w), at.z);
  else bulk_cell<Q, ST, true>(p, at.x(w), at.y(w), at.z);
}

// The cell kernels at the compiler's register choice (FP32, FP64: 72-92
// registers for D3Q19) and, for 16-bit storage, at 64 registers (8 blocks per
// SM): on the 96-instance sweep FP16 27.1k -> 28.4k MLUPS, while 64 registers
// made FP32 slower (27.1k -> 26.5k).
template <int ST, int Q, bool FACE_FREE>
__global__ void __launch_bounds__(kMultiCells) k_multi_cells(const BatchInst* inst,
                                                             const WorkItem* items, int step) {
  __shared__ Params sp;
  multi_cells<ST, Q, FACE_FREE>(&sp, inst, items, step);
}
template <int ST, int Q, bool FACE_FREE>
__global__ void __launch_bounds__(kMultiCells, 1024 / kMultiCells)
    k_multi_cells64(const BatchInst* inst, const WorkItem* items, int step) {
  __shared__ Params sp;
  multi_cells<ST, Q, FACE_FREE>(&sp, inst, items, step);
}

// Buffer parities of every instance advanced by the steps of a launch sequence.
__global__ void k_multi_advance(BatchInst* inst, int n, int nsteps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) inst[k].cur = (inst[k].cur + nsteps) & 1;
}

using MultiKernel = void (*)(const BatchInst*, const WorkItem*, int);
template <int Q, int ST> MultiKernel multi_kernel_st(int kind) {
  if (kind == MK_A) return k_multi_a<ST, Q>;
  if constexpr (ST == ST_FP16 || ST == ST_BF16)
    return kind == MK_I ? k_multi_cells64<ST, Q, true> : k_multi_cells64<ST, Q, false>;
  else
    return kind == MK_I ? k_multi_cells<ST, Q, true> : k_multi_cells<ST, Q, false>;
}
template <int Q> MultiKernel multi_kernel_q(int st, int kind) {
  switch (st) {
    case ST_FP32: return multi_kernel_st<Q, ST_FP32>(kind);
    case ST_FP16: return multi_kernel_st<Q, ST_FP16>(kind);
    case ST_BF16: return multi_kernel_st<Q, ST_BF16>(kind);
    default: return multi_kernel_st<Q, ST_FP64>(kind);
  }
}
MultiKernel multi_kernel(int st, int q, int kind) {
  return q == 19 ? multi_kernel_q<19>(st, kind) : multi_kernel_q<9>(st, kind);
}

std::string g_batch_err;

}  // namespace

struct lbm_batch {
  std::vector<lbm_ctx*> ctxs;
  int st = 0;
  cudaStream_t stream = nullptr;
  BatchInst* d_inst = nullptr;
  std::vector<BatchInst> h_inst;
  // lattice groups: 0 = D3Q19 instances, 1 = D2Q9 instances, each advanced by
  // its own kernel; the items of group g are d_items[item_off[g] ...]
  WorkItem* d_items = nullptr;
  int nitems[2] = {0, 0};        // items of one step per group
  int item_off[2] = {0, 0};
  void* d_ctl = nullptr;         // BatchCtl per group, then done[n], done_a[n]
  size_t ctl_bytes = 0;
  int threads = 256;
  int tile = 256;                // cells per B / I / W item (one warp each)
  int grid[2] = {0, 0};
  bool tuned = false;
  bool use_graph = true;         // false if capturing the cooperative launch was refused
  cudaGraphExec_t gexec = nullptr;
  int g_nsteps = -1;
  std::vector<int> dev_cur;      // buffer parity of each instance as the device holds it
  long long spin_limit = kSpinLimit;   // polls before a warp gives up at a wait
  // pinned copies of the groups' control blocks, one pair per launch in flight
  // (a ring of kCtlSlots): a later launch cannot overwrite the copy of an
  // earlier one before the host has read it
  BatchCtl* h_ctl = nullptr;
  cudaEvent_t ev_ctl[kCtlSlots] = {};
  bool ctl_pending[kCtlSlots] = {};   // the slot's copy has not been inspected yet
  int ctl_next = 0;                   // slot of the next launch's copy (the oldest one)
  bool ctl_failed = false;            // an inspected copy showed a wait that gave up
  // mode 1 (multi-instance launches): items per group and kind (MK_A, MK_I, MK_BW)
  int mode = 0;                  // 0: persistent ticketed kernel, 1: multi-instance launches
  int forced_mode = -1;          // lbm_batch_set_mode; -1: the autotuner's choice
  WorkItem* d_mitems = nullptr;
  int moff[2][3] = {{0, 0, 0}, {0, 0, 0}};
  int mn[2][3] = {{0, 0, 0}, {0, 0, 0}};
  cudaStream_t side = nullptr;   // wall branch of a multi-instance step
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int prio_hi = 0;
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

static void drop_graph(lbm_batch* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
}

static int group_q(int g) { return g == 0 ? 19 : 9; }

// The items of one step of a lattice group: wall-node chunks of 32 of every
// instance first, then per instance its ranges of `tile` cells: the face-free
// box (rows 1..ny-2, or every row of a y-periodic lattice without walls, times
// the columns 1..nx-2, or every column of an x-periodic one), the x-face
// columns of those rows, and the two face rows (wall rows after the wall
// pre-pass, KIND_W, or the face rows of a lattice without walls, KIND_B).
static void push_box(std::vector<WorkItem>& items, int inst, int kind, int tile, int nz, int xa,
                     int xs, int ncol, int ya, int ys, int nrow) {
  const int n = ncol * nrow * nz;
  for (int a = 0; a < n; a += tile)
    items.push_back({inst, kind, 0, a, std::min(n, a + tile), xa, xs, ncol, ya, ys, nrow, nz});
}

static void group_items(const lbm_batch* b, int g, int tile, std::vector<WorkItem>& items,
                        std::vector<int>& per_a, int achunk = 32) {
  std::vector<int> order;
  for (int i = 0; i < (int)b->ctxs.size(); ++i)
    if (b->ctxs[i]->Q == group_q(g)) order.push_back(i);
  for (int i : order) {
    const lbm_ctx* c = b->ctxs[i];
    for (int f = 0; f < 2; ++f) {
      if (!c->base.wall[f]) continue;
      const int nw = c->base.nwall[f];
      for (int a = 0; a < nw; a += achunk) {
        items.push_back({i, KIND_A, f, a, std::min(nw, a + achunk), 0, 0, 0, 0, 0, 0, 0});
        ++per_a[i];
      }
    }
  }
  for (int i : order) {
    const lbm_ctx* c = b->ctxs[i];
    const bool walls = per_a[i] > 0;
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    const bool px = c->base.px, py = c->base.py && !walls;
    // face-free rows and columns
    const int ya = py ? 0 : 1, nrow = py ? ny : std::max(0, ny - 2);
    const int xa = px ? 0 : 1, ncol = px ? nx : std::max(0, nx - 2);
    if (ncol > 0 && nrow > 0) push_box(items, i, KIND_I, tile, nz, xa, 1, ncol, ya, 1, nrow);
    if (!px && nrow > 0)     // x-face columns 0 and nx - 1 of those rows
      push_box(items, i, KIND_B, tile, nz, 0, nx - 1, nx > 1 ? 2 : 1, ya, 1, nrow);
    if (!py)                 // face rows 0 and ny - 1
      push_box(items, i, walls ? KIND_W : KIND_B, tile, nz, 0, 1, nx, 0, ny - 1, ny > 1 ? 2 : 1);
  }
}

static lbm_status build_items(lbm_batch* b, int tile) {
  std::vector<WorkItem> items;
  std::vector<int> per(b->ctxs.size(), 0), per_a(b->ctxs.size(), 0);
  for (int g = 0; g < 2; ++g) {
    b->item_off[g] = (int)items.size();
    group_items(b, g, tile, items, per_a);
    b->nitems[g] = (int)items.size() - b->item_off[g];
  }
  for (const WorkItem& w : items) ++per[w.inst];
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  BATCH_TRY(b, cudaMalloc(&b->d_items, std::max<size_t>(1, items.size()) * sizeof(WorkItem)));
  BATCH_TRY(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem),
                          cudaMemcpyHostToDevice));
  // per-instance item counts, written into the two adjacent int fields of each
  // device instance record (its parity is left as the device holds it); no
  // launch is in flight when the items are rebuilt
  std::vector<int> counts(2 * b->ctxs.size());
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    counts[2 * i] = per[i];
    counts[2 * i + 1] = per_a[i];
  }
  static_assert(offsetof(BatchInst, itemsA) == offsetof(BatchInst, items) + sizeof(int),
                "items and itemsA are adjacent");
  BATCH_TRY(b, cudaMemcpy2DAsync((char*)b->d_inst + offsetof(BatchInst, items), sizeof(BatchInst),
                                 counts.data(), 2 * sizeof(int), 2 * sizeof(int), b->ctxs.size(),
                                 cudaMemcpyHostToDevice, b->stream));
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  b->tile = tile;
  drop_graph(b);
  return LBM_OK;
}

// The items of the multi-instance mode, per group split by kernel: A, I, then
// B and W (one CTA each).
static lbm_status build_multi_items(lbm_batch* b) {
  std::vector<WorkItem> all, items;
  std::vector<int> per_a(b->ctxs.size(), 0);
  for (int g = 0; g < 2; ++g) {
    all.clear();
    group_items(b, g, kMultiCells, all, per_a, kMultiNodes);
    for (int kind = 0; kind < 3; ++kind) {
      b->moff[g][kind] = (int)items.size();
      for (const WorkItem& w : all) {
        const int k = w.kind == KIND_A ? MK_A : (w.kind == KIND_I ? MK_I : MK_BW);
        if (k == kind) items.push_back(w);
      }
      b->mn[g][kind] = (int)items.size() - b->moff[g][kind];
    }
  }
  if (b->d_mitems) cudaFree(b->d_mitems);
  b->d_mitems = nullptr;
  BATCH_TRY(b, cudaMalloc(&b->d_mitems, std::max<size_t>(1, items.size()) * sizeof(WorkItem)));
  BATCH_TRY(b, cudaMemcpy(b->d_mitems, items.data(), items.size() * sizeof(WorkItem),
                          cudaMemcpyHostToDevice));
  return LBM_OK;
}

static cudaError_t launch_multi_kernel(lbm_batch* b, int g, int kind, int step, cudaStream_t s, int prio) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->mn[g][kind], 1, 1);
  cfg.blockDim = dim3(kind == MK_A ? kMultiNodes : kMultiCells, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = prio != 0 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, multi_kernel(b->st, group_q(g), kind), (const BatchInst*)b->d_inst,
                            (const WorkItem*)b->d_mitems + b->moff[g][kind], step);
}

// Enqueue nsteps multi-instance steps on s: per step the wall branch (A, then
// B / W items) on the side stream at the highest priority beside the I items,
// joined before the next step; then the parities advance.
static lbm_status launch_multi(lbm_batch* b, int nsteps, cudaStream_t s) {
  for (int step = 0; step < nsteps; ++step) {
    BATCH_TRY(b, cudaEventRecord(b->ev_fork, s));
    BATCH_TRY(b, cudaStreamWaitEvent(b->side, b->ev_fork, 0));
    for (int g = 0; g < 2; ++g)
      if (b->mn[g][MK_A] > 0) BATCH_TRY(b, launch_multi_kernel(b, g, MK_A, step, b->side, b->prio_hi));
    for (int g = 0; g < 2; ++g)
      if (b->mn[g][MK_BW] > 0) BATCH_TRY(b, launch_multi_kernel(b, g, MK_BW, step, b->side, b->prio_hi));
    for (int g = 0; g < 2; ++g)   // launched after the wall branch: measured faster than before it
      if (b->mn[g][MK_I] > 0) BATCH_TRY(b, launch_multi_kernel(b, g, MK_I, step, s, 0));
    BATCH_TRY(b, cudaEventRecord(b->ev_join, b->side));
    BATCH_TRY(b, cudaStreamWaitEvent(s, b->ev_join, 0));
  }
  const int n = (int)b->ctxs.size();
  k_multi_advance<<<(n + 255) / 256, 256, 0, s>>>(b->d_inst, n, nsteps);
  BATCH_TRY(b, cudaGetLastError());
  return LBM_OK;
}

static void advance_host_parity(lbm_batch* b, int nsteps);

// Multi-instance steps, launched directly: the wall branch's stream priority
// is honoured only by direct launches (captured 32-step chunks replayed from a
// graph: 26.1k against 27.1k MLUPS on the 96-instance FP32 sweep).
static lbm_status step_multi(lbm_batch* b, int nsteps) {
  lbm_status s = launch_multi(b, nsteps, b->stream);
  if (s != LBM_OK) return s;
  advance_host_parity(b, nsteps);
  return LBM_OK;
}

static lbm_status set_threads(lbm_batch* b, int threads) {
  int dev = 0, sms = 0;
  BATCH_TRY(b, cudaGetDevice(&dev));
  BATCH_TRY(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  for (int g = 0; g < 2; ++g) {
    int per_sm = 0;
    BATCH_TRY(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(b->st, group_q(g)),
                                                               threads, 0));
    if (per_sm < 1) {
      b->err = "the batch kernel does not fit on an SM with this block size";
      return LBM_EUNSUPPORTED;
    }
    b->grid[g] = sms * per_sm;
  }
  b->threads = threads;
  drop_graph(b);
  return LBM_OK;
}

// Enqueue the control-block reset and one cooperative launch advancing every
// instance by nsteps.
// Enqueue the control-block reset and, per lattice group with instances, one
// cooperative launch advancing them by nsteps (the groups one after the other).
static lbm_status launch(lbm_batch* b, int nsteps, cudaStream_t s) {
  BATCH_TRY(b, cudaMemsetAsync(b->d_ctl, 0, b->ctl_bytes, s));
  BatchCtl* ctl = (BatchCtl*)b->d_ctl;
  unsigned* done = (unsigned*)((char*)b->d_ctl + 2 * sizeof(BatchCtl));
  unsigned* done_a = done + b->ctxs.size();
  for (int g = 0; g < 2; ++g) {
    if (b->nitems[g] == 0) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid[g], 1, 1);
    cfg.blockDim = dim3(b->threads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BATCH_TRY(b, cudaLaunchKernelEx(&cfg, batch_kernel(b->st, group_q(g)), b->d_inst,
                                    (const WorkItem*)b->d_items + b->item_off[g], b->nitems[g],
                                    ctl + g, done, done_a, nsteps, b->spin_limit));
  }
  return LBM_OK;
}

// After a launch on b->stream: copy the control block to pinned host memory
// behind it, to be inspected later without blocking the host.
static void inspect_ctl(lbm_batch* b, int slot) {
  BatchCtl* h = b->h_ctl + 2 * slot;
  b->ctl_pending[slot] = false;
  if (h[0].err || h[1].err) b->ctl_failed = true;
  h[0].err = h[1].err = 0;
}

static lbm_status queue_ctl_copy(lbm_batch* b) {
  const int slot = b->ctl_next;
  if (b->ctl_pending[slot]) {
    // kCtlSlots launches in flight: the oldest one's copy is read before its
    // slot is reused (this call then waits for that launch)
    BATCH_TRY(b, cudaEventSynchronize(b->ev_ctl[slot]));
    inspect_ctl(b, slot);
  }
  BATCH_TRY(b, cudaMemcpyAsync(b->h_ctl + 2 * slot, b->d_ctl, 2 * sizeof(BatchCtl),
                               cudaMemcpyDeviceToHost, b->stream));
  BATCH_TRY(b, cudaEventRecord(b->ev_ctl[slot], b->stream));
  b->ctl_pending[slot] = true;
  b->ctl_next = (slot + 1) % kCtlSlots;
  return LBM_OK;
}

// Inspect the control copy of the last launch.  blocking = false: if that
// launch has not finished yet, report nothing now (a later call will).  After
// a reported timeout the instances' states are not valid; the device parities
// are re-sent before the next launch.
static lbm_status poll_ctl(lbm_batch* b, bool blocking) {
  // the slots in launch order, oldest first (all copies are on b->stream, so a
  // copy is complete only if every older one is)
  for (int k = 0; k < kCtlSlots; ++k) {
    const int slot = (b->ctl_next + k) % kCtlSlots;
    if (!b->ctl_pending[slot]) continue;
    if (blocking) {
      BATCH_TRY(b, cudaEventSynchronize(b->ev_ctl[slot]));
    } else {
      const cudaError_t q = cudaEventQuery(b->ev_ctl[slot]);
      if (q == cudaErrorNotReady) break;
      BATCH_TRY(b, q);
    }
    inspect_ctl(b, slot);
  }
  if (b->ctl_failed) {
    b->ctl_failed = false;
    for (int& d : b->dev_cur) d = -1;
    b->err = "a bounded wait of the batch kernel gave up; the instances' states are not valid";
    return LBM_ETIMEOUT;
  }
  return LBM_OK;
}

static void advance_host_parity(lbm_batch* b, int nsteps) {
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    lbm_ctx* c = b->ctxs[i];
    c->cur = (c->cur + nsteps) & 1;
    c->steps_done += nsteps;
    if (b->dev_cur[i] >= 0) b->dev_cur[i] = (b->dev_cur[i] + nsteps) & 1;
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

// One launch of nsteps on b->stream (directly), with its control copy.
static lbm_status launch_tracked(lbm_batch* b, int nsteps) {
  lbm_status s = launch(b, nsteps, b->stream);
  if (s != LBM_OK) return s;
  advance_host_parity(b, nsteps);
  return queue_ctl_copy(b);
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
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) {
        delete b;
        g_batch_err = "lbm_batch_create: a context appears twice";
        return LBM_EINVAL;
      }
    b->ctxs.push_back(c);
  }
  b->st = ctxs[0]->st;
  b->stream = ctxs[0]->stream;
  for (int i = 0; i < n; ++i) b->dev_cur.push_back(ctxs[i]->cur);
  b->h_inst.resize(n);
  for (int i = 0; i < n; ++i) {
    const lbm_ctx* c = ctxs[i];
    std::memset(&b->h_inst[i], 0, sizeof(BatchInst));
    b->h_inst[i].p[0] = lbm_ctx_params(c, 0);
    b->h_inst[i].p[1] = lbm_ctx_params(c, 1);
    b->h_inst[i].Q = c->Q;
    b->h_inst[i].cur = c->cur;
  }
  b->ctl_bytes = 2 * sizeof(BatchCtl) + 2 * (size_t)n * sizeof(unsigned);
  {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) hi = 0;
    b->prio_hi = hi;
  }
  if (cudaMalloc(&b->d_inst, n * sizeof(BatchInst)) != cudaSuccess ||
      cudaMalloc(&b->d_ctl, b->ctl_bytes) != cudaSuccess ||
      cudaMallocHost(&b->h_ctl, 2 * kCtlSlots * sizeof(BatchCtl)) != cudaSuccess ||
      cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, b->prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    g_batch_err = "lbm_batch_create: device allocation failed";
    lbm_batch_destroy(b);
    return LBM_ENOMEM;
  }
  for (cudaEvent_t& e : b->ev_ctl) {
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      e = nullptr;
      g_batch_err = "lbm_batch_create: event creation failed";
      lbm_batch_destroy(b);
      return LBM_ENOMEM;
    }
  }
  std::memset(b->h_ctl, 0, 2 * kCtlSlots * sizeof(BatchCtl));
  // the contexts' pending work (state set-up) must be complete before the batch
  // reads their parameters on another order of launches
  for (lbm_ctx* c : b->ctxs) cudaStreamSynchronize(c->stream);
  if (cudaMemcpy(b->d_inst, b->h_inst.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(b->d_ctl, 0, b->ctl_bytes) != cudaSuccess) {
    g_batch_err = "lbm_batch_create: upload failed";
    lbm_batch_destroy(b);
    return LBM_ECUDA;
  }
  lbm_status st = set_threads(b, 256);
  if (st == LBM_OK) st = build_items(b, 256);
  if (st == LBM_OK) st = build_multi_items(b);
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
  lbm_status s = poll_ctl(b, true);
  if (s != LBM_OK) return s;
  s = sync_parity(b);
  if (s != LBM_OK) return s;
  const int threads_c[2] = {128, 256};
  const int tiles_c[3] = {64, 256, 1024};   // cells per warp item
  float best_ms = 1e30f;
  int bt = b->threads, btile = b->tile;
  cudaEvent_t e0, e1;
  BATCH_TRY(b, cudaEventCreate(&e0));
  BATCH_TRY(b, cudaEventCreate(&e1));
  const int trial = 3;
  for (int t : threads_c) {
    s = set_threads(b, t);
    if (s != LBM_OK) continue;
    for (int k : tiles_c) {
      s = build_items(b, k);
      if (s == LBM_OK) s = launch_tracked(b, 1);   // warm-up
      if (s != LBM_OK) break;
      BATCH_TRY(b, cudaEventRecord(e0, b->stream));
      s = launch_tracked(b, trial);
      if (s != LBM_OK) break;
      BATCH_TRY(b, cudaEventRecord(e1, b->stream));
      BATCH_TRY(b, cudaEventSynchronize(e1));
      s = poll_ctl(b, true);
      if (s != LBM_OK) break;
      float ms = 0.f;
      BATCH_TRY(b, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        bt = t;
        btile = k;
      }
    }
    if (s != LBM_OK && s != LBM_EUNSUPPORTED) break;
  }
  if (s != LBM_OK && s != LBM_EUNSUPPORTED) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
  }
  // the multi-instance launches, timed the same way (uncaptured)
  float multi_ms = 1e30f;
  s = launch_multi(b, 1, b->stream);
  if (s == LBM_OK) {
    advance_host_parity(b, 1);
    BATCH_TRY(b, cudaEventRecord(e0, b->stream));
    s = launch_multi(b, trial, b->stream);
  }
  if (s == LBM_OK) {
    advance_host_parity(b, trial);
    BATCH_TRY(b, cudaEventRecord(e1, b->stream));
    BATCH_TRY(b, cudaEventSynchronize(e1));
    BATCH_TRY(b, cudaEventElapsedTime(&multi_ms, e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != LBM_OK) return s;
  b->mode = b->forced_mode >= 0 ? b->forced_mode : (multi_ms < best_ms ? 1 : 0);
  s = set_threads(b, bt);
  if (s == LBM_OK) s = build_items(b, btile);
  if (s != LBM_OK) return s;
  b->tuned = true;
  if (best) {
    best[0] = bt;
    best[1] = btile;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_step(lbm_batch* b, int nsteps) {
  if (!b || nsteps < 0) return LBM_EINVAL;
  if (nsteps == 0) return LBM_OK;
  // a timeout of an earlier launch that has finished is reported here
  lbm_status s = poll_ctl(b, false);
  if (s != LBM_OK) return s;
  s = sync_parity(b);
  if (s != LBM_OK) return s;
  if (!b->tuned) {
    s = lbm_batch_tune(b, nullptr);
    if (s != LBM_OK) return s;
  }
  if (b->mode == 1) return step_multi(b, nsteps);
  if (!b->use_graph) return launch_tracked(b, nsteps);
  // one persistent launch per call, replayed from a graph while nsteps repeats
  if (!b->gexec || b->g_nsteps != nsteps) {
    drop_graph(b);
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
    if (e != cudaSuccess || s != LBM_OK || !b->gexec) {
      // the cooperative launch could not be captured: launch it directly
      cudaGetLastError();
      drop_graph(b);
      b->use_graph = false;
      return launch_tracked(b, nsteps);
    }
    b->g_nsteps = nsteps;
  }
  BATCH_TRY(b, cudaGraphLaunch(b->gexec, b->stream));
  advance_host_parity(b, nsteps);
  return queue_ctl_copy(b);
}

extern "C" lbm_status lbm_batch_wait(lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  lbm_status s = poll_ctl(b, true);
  if (s != LBM_OK) return s;
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_set_wait_limit(lbm_batch* b, long long polls) {
  if (!b || polls < 0) return LBM_EINVAL;
  b->spin_limit = polls > 0 ? polls : 0;
  drop_graph(b);   // the limit is a launch argument of the captured kernel
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_info(const lbm_batch* b, int out[5]) {
  if (!b || !out) return LBM_EINVAL;
  const bool multi = b->mode == 1;
  out[0] = multi ? kMultiCells : b->threads;
  out[1] = multi ? kMultiCells : b->tile;
  out[2] = !multi && b->use_graph ? 1 : 0;
  out[3] = multi ? b->mn[0][0] + b->mn[0][1] + b->mn[0][2] + b->mn[1][0] + b->mn[1][1] + b->mn[1][2]
                 : b->nitems[0] + b->nitems[1];
  out[4] = b->mode;
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_set_mode(lbm_batch* b, int mode) {
  if (!b || mode < -1 || mode > 1) return LBM_EINVAL;
  lbm_status s = poll_ctl(b, true);
  if (s != LBM_OK) return s;
  b->forced_mode = mode;
  if (mode >= 0) b->mode = mode;
  return LBM_OK;
}

extern "C" void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->d_ctl) cudaFree(b->d_ctl);
  if (b->d_items) cudaFree(b->d_items);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  for (cudaEvent_t& e : b->ev_ctl)
    if (e) cudaEventDestroy(e);
  if (b->d_mitems) cudaFree(b->d_mitems);
  if (b->side) {
    cudaStreamSynchronize(b->side);
    cudaStreamDestroy(b->side);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  delete b;
}

extern "C" const char* lbm_batch_last_error(const lbm_batch* b) {
  return b ? b->err.c_str() : g_batch_err.c_str();
}
