// api.cu -- host implementation of the C ABI declared in include/lbm.h.
//
// A context owns the double-buffered population, velocity and nu_tilde fields,
// the per-wall-node state of both y faces and the FP64 reduction scratch.  A
// step is two launches on the context stream: the wall pre-pass (k_wall) and
// the fused bulk kernel (k_bulk).  With walls a step is three launches issued
// directly: the wall pre-pass and then the two wall rows on a high-priority
// side stream, the inner rows on the context stream.  Without walls a step is
// one bulk launch, and pairs of steps are captured once per buffer parity into
// CUDA graphs and replayed by lbm_step.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_ctx.h"
#include "lbm_launch.h"

using namespace lbm;

static std::string g_static_error;

void lbm_ctx_set_error(lbm_ctx* c, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_static_error = buf;
}

#define CUDA_TRY(ctx, expr)                                                            \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      lbm_ctx_set_error(ctx, "%s failed: %s", #expr, cudaGetErrorString(e_));          \
      return LBM_ECUDA;                                                                \
    }                                                                                  \
  } while (0)

static void* dalloc(lbm_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* ptr = nullptr;
  if (c->cfg.alloc) {
    ptr = c->cfg.alloc(bytes, c->cfg.alloc_user);
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    ptr = nullptr;
  }
  if (ptr) c->allocs.push_back(ptr);
  return ptr;
}

// Device staging for host-side field transfers: allocated once (largest
// request so far) through the context allocator and kept until destroy.
static double* host_staging(lbm_ctx* c, size_t count) {
  if (c->staging_count >= count) return c->staging;
  if (c->staging) {
    if (c->cfg.free) c->cfg.free(c->staging, c->cfg.alloc_user);
    else if (!c->cfg.alloc) cudaFree(c->staging);
    c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), (void*)c->staging), c->allocs.end());
    c->staging = nullptr;
    c->staging_count = 0;
  }
  c->staging = (double*)dalloc(c, count * sizeof(double));
  if (c->staging) c->staging_count = count;
  return c->staging;
}

static size_t storage_bytes(int st) {
  switch (st) {
    case LBM_FP32: return 4;
    case LBM_FP16_SHIFTED:
    case LBM_BF16_SHIFTED: return 2;
    default: return 8;
  }
}

static int to_dev_storage(int st) {
  switch (st) {
    case LBM_FP32: return ST_FP32;
    case LBM_FP16_SHIFTED: return ST_FP16;
    case LBM_BF16_SHIFTED: return ST_BF16;
    default: return ST_FP64;
  }
}

// The wall pre-pass branch runs at the highest stream priority, so that its
// blocks are dispatched as soon as resources free up instead of queueing
// behind the whole inner-row grid.
static bool side_stream_create(cudaStream_t* s, int* prio_hi) {
  int lo = 0, hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) hi = 0;
  *prio_hi = hi;
  return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, hi) == cudaSuccess;
}

extern "C" const char* lbm_last_error(const lbm_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_static_error.c_str();
}

extern "C" lbm_status lbm_create(const lbm_config* cfg, lbm_ctx** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!cfg) {
    lbm_ctx_set_error(nullptr, "cfg is NULL");
    return LBM_EINVAL;
  }
  const lbm_config& k = *cfg;
  if (k.lattice != LBM_D2Q9 && k.lattice != LBM_D3Q19) {
    lbm_ctx_set_error(nullptr, "lattice must be LBM_D2Q9 or LBM_D3Q19");
    return LBM_EINVAL;
  }
  if (k.nx < 1 || k.ny < 1 || k.nz < 1 || (k.lattice == LBM_D2Q9 && k.nz != 1)) {
    lbm_ctx_set_error(nullptr, "bad sizes (D2Q9 needs nz == 1)");
    return LBM_EINVAL;
  }
  if ((long long)k.nx * k.ny * k.nz > (1LL << 31)) {
    lbm_ctx_set_error(nullptr, "lattice larger than 2^31 cells");
    return LBM_EINVAL;
  }
  if (!(k.dx > 0) || !(k.nu > 0) || !(k.rho0 > 0) || !(k.u_ref > 0) || !(k.mach > 0)) {
    lbm_ctx_set_error(nullptr, "dx, nu, rho0, u_ref and mach must be positive");
    return LBM_EINVAL;
  }
  if (k.collision != LBM_BGK && k.collision != LBM_REGULARIZED) {
    lbm_ctx_set_error(nullptr, "unknown collision");
    return LBM_EINVAL;
  }
  if (k.storage < LBM_FP32 || k.storage > LBM_FP64) {
    lbm_ctx_set_error(nullptr, "unknown storage");
    return LBM_EINVAL;
  }
  if (k.turbulence != LBM_SA && k.turbulence != LBM_LAMINAR) {
    lbm_ctx_set_error(nullptr, "unknown turbulence model");
    return LBM_EINVAL;
  }
  if (k.wall_law != LBM_LAW_SA_ANALYTIC && k.wall_law != LBM_LAW_LOG) {
    lbm_ctx_set_error(nullptr, "unknown wall law");
    return LBM_EINVAL;
  }
  if (!(std::fabs(k.u_shift * k.mach / (std::sqrt(3.0) * k.u_ref)) < 0.5)) {
    lbm_ctx_set_error(nullptr, "u_shift must be finite and well below the lattice speed");
    return LBM_EINVAL;
  }
  if (k.staging != 0 && k.staging != 1) {
    lbm_ctx_set_error(nullptr, "staging must be 0 (direct loads) or 1 (TMA tiles)");
    return LBM_EINVAL;
  }
  if (k.wall_law == LBM_LAW_LOG && !(k.kappa > 0)) {
    lbm_ctx_set_error(nullptr, "log law needs kappa > 0");
    return LBM_EINVAL;
  }
  lbm_ctx* c = new lbm_ctx();
  c->cfg = k;
  c->Q = k.lattice;
  c->st = to_dev_storage(k.storage);
  c->esz = storage_bytes(k.storage);
  c->rsz = k.storage == LBM_FP64 ? 8 : 4;
  c->nx = k.nx;
  c->ny = k.ny;
  c->nz = k.nz;
  c->pitch = (k.nx + 7) / 8 * 8;
  c->ncell = (long long)c->pitch * k.ny * k.nz;
  c->ncells = (long long)k.nx * k.ny * k.nz;
  if ((long long)c->Q * c->ncell >= (1LL << 31)) {
    lbm_ctx_set_error(nullptr, "Q * padded cells must stay below 2^31 (32-bit indexing)");
    delete c;
    return LBM_EUNSUPPORTED;
  }
  // acoustic scaling (Section 4.1.1): dt = M dx / (sqrt(3) U_ref)
  c->dt = k.mach * k.dx / (std::sqrt(3.0) * k.u_ref);
  c->ucv = c->dt / k.dx;
  c->nucv = c->dt / (k.dx * k.dx);
  c->nu_lb = k.nu * c->nucv;
  for (int a = 0; a < 3; ++a) c->F_lb[a] = k.force[a] * c->dt * c->dt / k.dx;
  if (!(c->nu_lb > 0.0) || !(0.5 + 3.0 * c->nu_lb > 0.5)) {
    lbm_ctx_set_error(nullptr, "tau0 = 1/2 + 3 nu_lb is not above 1/2 (nu_lb = %g)", c->nu_lb);
    delete c;
    return LBM_EINVAL;
  }
  for (int f = 0; f < 6; ++f) {
    std::memset(&c->bc[f], 0, sizeof(lbm_bc));
    c->bc[f].kind = LBM_BC_PERIODIC;
    c->bc[f].beta = 0.28;
    c->bc[f].ref_node = 2;
    c->bc[f].x_start = -INFINITY;
    c->bc[f].nut_ratio_in = 3.0;
    c->bc[f].d_w = 0.5;
  }
  c->stream = (cudaStream_t)k.stream;
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      !side_stream_create(&c->side_stream, &c->prio_hi) ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    lbm_ctx_set_error(nullptr, "cannot create capture stream: %s",
                      cudaGetErrorString(cudaGetLastError()));
    delete c;
    return LBM_ECUDA;
  }
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      c->sms = sms;
  }
  bool ok = true;
  for (int b = 0; b < 2; ++b) {
    c->f[b] = dalloc(c, (size_t)c->Q * c->ncell * c->esz);
    c->v[b] = dalloc(c, (size_t)4 * c->ncell * c->rsz);
    const size_t nodes = (size_t)k.nx * k.nz;
    c->utau[b] = (double*)dalloc(c, nodes * sizeof(double));
    c->uw[b] = dalloc(c, 3 * nodes * c->rsz);
    c->rhow[b] = dalloc(c, nodes * c->rsz);
    ok = ok && c->f[b] && c->v[b] && c->utau[b] && c->uw[b] && c->rhow[b];
  }
  c->utau_prev = (double*)dalloc(c, 2 * (size_t)k.nx * k.nz * sizeof(double));
  c->invd2 = dalloc(c, (size_t)c->pitch * k.ny * c->rsz);
  ok = ok && c->invd2;
  c->flags = (unsigned*)dalloc(c, sizeof(unsigned) * 4);
  c->red_blocks = 2 * 152;
  c->red_chunk = (c->ncells + c->red_blocks - 1) / c->red_blocks;
  c->partial = (double*)dalloc(c, (size_t)c->red_blocks * RED_VALS * sizeof(double));
  c->red_out = (double*)dalloc(c, 16 * sizeof(double));
  ok = ok && c->utau_prev && c->flags && c->partial && c->red_out;
  if (!ok) {
    lbm_destroy(c);
    lbm_ctx_set_error(nullptr, "device allocation failed");
    return LBM_ENOMEM;
  }
  *out = c;
  return LBM_OK;
}

extern "C" lbm_status lbm_set_bc(lbm_ctx* c, int face, const lbm_bc* bc) {
  if (!c || !bc) return LBM_EINVAL;
  if (face < LBM_XMIN || face > LBM_ZMAX) {
    lbm_ctx_set_error(c, "face %d out of range", face);
    return LBM_EINVAL;
  }
  const int kd = bc->kind;
  if (kd < LBM_BC_PERIODIC || kd > LBM_BC_WALL_CAI_DEGRIGNY) {
    lbm_ctx_set_error(c, "unknown boundary kind %d", kd);
    return LBM_EINVAL;
  }
  const bool xf = face <= LBM_XMAX, yf = face == LBM_YMIN || face == LBM_YMAX;
  const bool wall = kd == LBM_BC_WALL_SLIP_BB || kd == LBM_BC_WALL_HRFD ||
                    kd == LBM_BC_WALL_CAI_DEGRIGNY;
  if (face >= LBM_ZMIN && kd != LBM_BC_PERIODIC) {
    lbm_ctx_set_error(c, "z faces must be periodic");
    return LBM_EUNSUPPORTED;
  }
  if (xf && kd != LBM_BC_PERIODIC && kd != LBM_BC_INLET_ZOUHE && kd != LBM_BC_OUTLET_ZEROGRAD) {
    lbm_ctx_set_error(c, "x faces take periodic, inlet or outlet conditions");
    return LBM_EINVAL;
  }
  if ((kd == LBM_BC_INLET_ZOUHE && face != LBM_XMIN) ||
      (kd == LBM_BC_OUTLET_ZEROGRAD && face != LBM_XMAX)) {
    lbm_ctx_set_error(c, "inlet only on xmin, outlet only on xmax");
    return LBM_EINVAL;
  }
  if (yf && (kd == LBM_BC_INLET_ZOUHE || kd == LBM_BC_OUTLET_ZEROGRAD)) {
    lbm_ctx_set_error(c, "y faces take periodic, wall, symmetry or free-stream conditions");
    return LBM_EINVAL;
  }
  if (wall && !(bc->ref_node == 1 || bc->ref_node == 2)) {
    lbm_ctx_set_error(c, "ref_node must be 1 (B) or 2 (F)");
    return LBM_EINVAL;
  }
  if ((kd == LBM_BC_WALL_HRFD || kd == LBM_BC_WALL_CAI_DEGRIGNY) && bc->ref_node != 2) {
    lbm_ctx_set_error(c, "regularized walls take their reference velocity at F (ref_node = 2)");
    return LBM_EINVAL;
  }
  if (kd == LBM_BC_WALL_HRFD && !(bc->beta >= 0.0 && bc->beta <= 1.0)) {
    lbm_ctx_set_error(c, "beta must lie in [0, 1]");
    return LBM_EINVAL;
  }
  const double d_w = bc->d_w == 0.0 ? 0.5 : bc->d_w;
  if (wall && !(d_w > 0.0 && d_w <= 1.0)) {
    lbm_ctx_set_error(c, "d_w must lie in (0, 1]");
    return LBM_EINVAL;
  }
  if (bc->interp < LBM_IBB_NONE || bc->interp > LBM_IBB_YU ||
      (bc->interp != LBM_IBB_NONE && kd != LBM_BC_WALL_SLIP_BB)) {
    lbm_ctx_set_error(c, "interp is LBM_IBB_NONE, _BOUZIDI or _YU, on bounce-back walls only");
    return LBM_EINVAL;
  }
  if (kd == LBM_BC_WALL_SLIP_BB && bc->interp == LBM_IBB_NONE && d_w != 0.5) {
    lbm_ctx_set_error(c, "half-way bounce-back needs d_w = 1/2 (use an interpolated rule)");
    return LBM_EINVAL;
  }
  c->bc[face] = *bc;
  c->bc[face].d_w = d_w;
  c->finalized = false;
  c->gvalid[0] = c->gvalid[1] = false;
  return LBM_OK;
}

static void build_tensor_maps(lbm_ctx* c);

// Weights (a_o, a_F, a_i, a_K) of a face's bounce-back rule in deviation form,
// h_i(B, t+1) = a_o h*_opp(B) + a_F h*_opp(B + c_i) + a_i h*_i(B) + a_K K, for
// the incoming direction i, K = 6 w_i (rho_w c_i.u_w - c_ix U) (the moving-wall
// term plus the change of reference equilibrium from opp(i) to i).  Every rule
// is affine with weights summing to one, so the reference equilibria enter only
// through K.  q is the link fraction d_w.
//   Eq. 31 (half-way): h*_opp(B) + K.
//   Eq. 36, q >= 1/2: (h*_opp(B) + K) / 2q + (1 - 1/2q) h*_i(B)   [h*_i(B) = h_i(F, t+1)]
//   Eq. 36, q <  1/2: 2q h*_opp(B) + (1 - 2q) h*_opp(F) + K       [F = B + c_i]
//   Eq. 37: the wall-point value W = q h*_opp(B) + (1 - q) h*_opp(F) + K (the
//     streamed population interpolated to the wall and bounced back), then
//     W + r (h*_i(B) - W) with r = q / (1 + q).
static void ibb_weights(int interp, double q, double a[4]) {
  a[0] = 1.0;
  a[1] = 0.0;
  a[2] = 0.0;
  a[3] = 1.0;
  if (interp == LBM_IBB_BOUZIDI && q >= 0.5) {
    a[0] = a[3] = 1.0 / (2.0 * q);
    a[2] = 1.0 - 1.0 / (2.0 * q);
  } else if (interp == LBM_IBB_BOUZIDI) {
    a[0] = 2.0 * q;
    a[1] = 1.0 - 2.0 * q;
  } else if (interp == LBM_IBB_YU) {
    const double r = q / (1.0 + q);
    a[0] = q * (1.0 - r);
    a[1] = (1.0 - q) * (1.0 - r);
    a[2] = r;
    a[3] = 1.0 - r;
  }
}

// Validate the face combination and build the kernel parameters.
lbm_status lbm_ctx_finalize(lbm_ctx* c) {
  if (c->finalized) return LBM_OK;
  const lbm_config& k = c->cfg;
  for (int ax = 0; ax < 3; ++ax) {
    const bool a = c->bc[2 * ax].kind == LBM_BC_PERIODIC, b = c->bc[2 * ax + 1].kind == LBM_BC_PERIODIC;
    if (a != b) {
      lbm_ctx_set_error(c, "periodic faces must come in pairs (axis %d)", ax);
      return LBM_EINVAL;
    }
  }
  Params& p = c->base;
  std::memset(&p, 0, sizeof(p));
  p.nx = c->nx;
  p.ny = c->ny;
  p.nz = c->nz;
  p.pitch = c->pitch;
  p.ncell = c->ncell;
  p.collision = k.collision;
  p.turbulent = k.turbulence == LBM_SA;
  p.wall_law = k.wall_law;
  p.law_kappa = k.kappa;
  p.law_B = k.B;
  p.nu = c->nu_lb;
  for (int a = 0; a < 3; ++a) p.F[a] = c->F_lb[a];
  p.has_force = (p.F[0] != 0.0 || p.F[1] != 0.0 || p.F[2] != 0.0);
  p.Ush = k.u_shift * c->ucv;
  for (int i = 0; i < c->Q; ++i) {
    // 3 w_i c_i . F, in the kernels' direction order
    double cF = 0.0, w = 0.0;
    for (int a = 0; a < 3; ++a)
      cF += (c->Q == 9 ? Lat<9>::c(i, a) : Lat<19>::c(i, a)) * p.F[a];
    w = c->Q == 9 ? Lat<9>::w(i) : Lat<19>::w(i);
    p.guoA[i] = 3.0 * w * cF;
  }
  for (int f = 0; f < 6; ++f) p.kind[f] = c->bc[f].kind;
  p.px = c->bc[LBM_XMIN].kind == LBM_BC_PERIODIC;
  p.py = c->bc[LBM_YMIN].kind == LBM_BC_PERIODIC;
  int nhrfd = 0;
  for (int fi = 0; fi < 2; ++fi) {
    const lbm_bc& b = c->bc[LBM_YMIN + fi];
    const bool wall = b.kind == LBM_BC_WALL_SLIP_BB || b.kind == LBM_BC_WALL_HRFD ||
                      b.kind == LBM_BC_WALL_CAI_DEGRIGNY;
    p.wall[fi] = 0;
    if (!wall) continue;
    int x0 = 0;
    while (x0 < c->nx && !(k.origin[0] + (x0 + 0.5) * k.dx >= b.x_start)) ++x0;
    p.xw0[fi] = x0;
    p.xs_lb[fi] = std::isfinite(b.x_start) ? (b.x_start - k.origin[0]) / k.dx : -1e30;
    p.beta[fi] = b.beta;
    p.ref_node[fi] = b.ref_node;
    p.d_w[fi] = b.d_w;
    p.interp[fi] = b.kind == LBM_BC_WALL_SLIP_BB ? b.interp : LBM_IBB_NONE;
    ibb_weights(p.interp[fi], b.d_w, p.ibb[fi]);
    p.nwall[fi] = (c->nx - x0) * c->nz;
    if (p.nwall[fi] > 0) p.wall[fi] = b.kind;
    if (b.kind == LBM_BC_WALL_HRFD || b.kind == LBM_BC_WALL_CAI_DEGRIGNY) ++nhrfd;
    if (c->ny < 3) {
      lbm_ctx_set_error(c, "walls need ny >= 3 (nodes B, F, FF)");
      return LBM_EINVAL;
    }
    if (p.wall[fi] && x0 == 0 && c->bc[LBM_XMIN].kind == LBM_BC_INLET_ZOUHE) {
      lbm_ctx_set_error(c, "a wall may not start at the inlet column");
      return LBM_EINVAL;
    }
  }
  if (nhrfd == 2 && c->ny < 6) {
    lbm_ctx_set_error(c, "two regularized walls need ny >= 6");
    return LBM_EINVAL;
  }
  const int pf[4] = {LBM_XMIN, LBM_XMAX, LBM_YMIN, LBM_YMAX};
  for (int j = 0; j < 4; ++j) {
    const lbm_bc& b = c->bc[pf[j]];
    for (int a = 0; a < 3; ++a) p.u_face[j][a] = b.u_in[a] * c->ucv;
    p.nt_face[j] = b.nut_ratio_in * c->nu_lb;
  }
  if (c->bc[LBM_XMIN].kind == LBM_BC_INLET_ZOUHE && !(p.u_face[0][0] < 1.0)) {
    lbm_ctx_set_error(c, "inlet velocity must be below one lattice speed");
    return LBM_EINVAL;
  }
  for (int b = 0; b < 2; ++b) {
    p.utau[b] = c->utau[b];
    p.uw[b] = c->uw[b];
    p.rhow[b] = c->rhow[b];
  }
  p.flags = c->flags;
  p.wait_limit = c->wait_limit;
  // 1 / d^2 of the SA model per (y, x): distance to the nearest wall face (the
  // line d_w below row 0 / above row ny - 1), measured to the leading-edge
  // point for columns upstream of a wall's x_start; 0 without walls
  {
    std::vector<double> tab((size_t)c->pitch * c->ny, 0.0);
    for (int y = 0; y < c->ny; ++y)
      for (int x = 0; x < c->nx; ++x) {
        double d2 = INFINITY;
        for (int f = 0; f < 2; ++f) {
          if (!p.wall[f]) continue;
          const double dy = f == 0 ? y + p.d_w[f] : (c->ny - 1 - y) + p.d_w[f];
          double e = dy * dy;
          if (x < p.xw0[f]) {
            const double dxl = (x + 0.5) - p.xs_lb[f];
            e += dxl * dxl;
          }
          d2 = std::min(d2, e);
        }
        tab[(size_t)y * c->pitch + x] = std::isfinite(d2) ? 1.0 / d2 : 0.0;
      }
    // on the context stream, complete before the host copy goes out of scope
    std::vector<float> tf;
    const void* src = tab.data();
    size_t bytes = tab.size() * sizeof(double);
    if (c->rsz != sizeof(double)) {
      tf.assign(tab.begin(), tab.end());
      src = tf.data();
      bytes = tf.size() * sizeof(float);
    }
    cudaError_t e = cudaMemcpyAsync(c->invd2, src, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      lbm_ctx_set_error(c, "wall-distance table upload failed: %s", cudaGetErrorString(e));
      return LBM_ECUDA;
    }
  }
  p.invd2 = c->invd2;
  build_tensor_maps(c);
  // float copies of the lattice parameters for the FP32 kernels
  p.nu_f = (float)p.nu;
  p.inv_nu = 1.0 / p.nu;
  p.inv_nu_f = (float)p.inv_nu;
  p.Ush_f = (float)p.Ush;
  for (int a = 0; a < 3; ++a) p.F_f[a] = (float)p.F[a];
  for (int i = 0; i < 19; ++i) p.guoA_f[i] = (float)p.guoA[i];
  for (int f = 0; f < 2; ++f) {
    p.xs_lb_f[f] = (float)p.xs_lb[f];
    p.d_w_f[f] = (float)(p.wall[f] ? p.d_w[f] : 0.5);
    for (int k = 0; k < 4; ++k) p.ibb_f[f][k] = (float)p.ibb[f][k];
  }
  for (int j = 0; j < 4; ++j) {
    p.nt_face_f[j] = (float)p.nt_face[j];
    for (int a = 0; a < 3; ++a) p.u_face_f[j][a] = (float)p.u_face[j][a];
  }
  c->finalized = true;
  c->gvalid[0] = c->gvalid[1] = false;
  return LBM_OK;
}

Params lbm_ctx_params(const lbm_ctx* c, int src) {
  Params p = c->base;
  p.f_src = c->f[src];
  p.f_dst = c->f[1 - src];
  p.v_src = c->v[src];
  p.v_dst = c->v[1 - src];
  return p;
}

// Tensor maps of both population buffers for the TMA-staged inner-row kernel:
// 4-D [q][z][y][x], box (32 + 2 * 16/esz) x 8 x 1 x 1.  Built only when the
// alignment rules of tiled bulk copies hold: 16-byte base address and strides;
// the box width and the x start x0 - 16/esz (x0 a multiple of 32) are 16-byte
// multiples by construction.
static void build_tensor_maps(lbm_ctx* c) {
  c->tma_ok = false;
  if (c->cfg.staging != 1) return;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  if (!encode || c->ny < 3) return;
  CUtensorMapDataType dt;
  switch (c->st) {
    case ST_FP32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case ST_FP16: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    case ST_BF16: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    default: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
  }
  const cuuint64_t esz = c->esz;
  const cuuint64_t dims[4] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)c->nz, (cuuint64_t)c->Q};
  const cuuint64_t strides[3] = {(cuuint64_t)c->pitch * esz, (cuuint64_t)c->pitch * c->ny * esz,
                                 (cuuint64_t)c->ncell * esz};
  const cuuint32_t box[4] = {(cuuint32_t)tma_box_width(c->esz), 8, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if ((box[0] * esz) % 16 || strides[0] % 16 || strides[1] % 16 || strides[2] % 16) return;
  for (int b = 0; b < 2; ++b) {
    if (((uintptr_t)c->f[b]) % 16) return;
    CUresult r = encode(&c->tmap[b], dt, 4, c->f[b], dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;
  }
  c->tma_ok = true;
}

// The face-free row sets (the inner rows, every row of a lattice periodic in x
// and y) of x-periodic BGK lattices run two cells per thread (k_bulk2).  On the
// 2048x512x8 plate (regularized collision, inlet and outlet columns) the pair
// kernel measured slower than one cell per thread (FP32 28.2k vs 29.6k MLUPS,
// FP16 30.9k vs 32.6k); on the BGK channel faster in FP16 (33.5k vs 31.3k)
// and equal in FP32.
// Which face-free row sets run two cells per thread: LBM_BULK_PAIRS 1, those of
// lattices periodic in x with BGK collision; 2, every one.
bool lbm_ctx_bulk_pairs(const lbm_ctx* c, int rows) {
  const bool fast = rows == ROWS_INNER || (rows == ROWS_ALL && c->base.px && c->base.py);
  if (LBM_BULK_PAIRS >= 2) return fast;
  return LBM_BULK_PAIRS && fast && c->base.px && c->base.collision == 0;
}

// Launch shape of k_bulk for a row set (ROWS_ALL / ROWS_INNER / ROWS_WALL).
// The face-free row sets (the inner rows, every row of a lattice periodic in x
// and y) run two cells per thread along x.
int lbm_ctx_bulk_launch_dims(const lbm_ctx* c, int rows, dim3* g, dim3* b) {
  const bool pairs = lbm_ctx_bulk_pairs(c, rows);
  const int nxt = pairs ? (c->nx + 1) / 2 : c->nx;   // threads along x
  int bx = 32;
  while (bx > 1 && bx / 2 >= nxt) bx /= 2;
  const int nrows = rows == ROWS_ALL ? c->ny : (rows == ROWS_WALL ? 2 : c->ny - 2);
  int by = LBM_BULK_THREADS / bx;
  if (rows == ROWS_WALL) by = 2;
  if (rows == ROWS_XEDGE) {   // columns 0 and nx-1: 2 x (LBM_BULK_THREADS / 2) cells per block
    const int h = LBM_BULK_THREADS / 2;
    *b = dim3(2, h, 1);
    *g = dim3(1, (nrows + h - 1) / h, c->nz);
    return rows;
  }
  *b = dim3(bx, by, 1);
  *g = dim3((nxt + bx - 1) / bx, (nrows + by - 1) / by, c->nz);
  // Block order.  Blocks are dispatched x fastest, then grid y, then grid z;
  // a cell re-reads the planes z +/- 1 and the rows y +/- 1 of its own launch.
  // With the planes in grid z a plane is re-read nx * ny cells later; with the
  // planes in grid y (ROWS_ZY) a row band is re-read nx * by * nz cells later.
  // The shorter distance keeps the re-reads in L2 (the 2048x512x8 plate: a
  // plane is 1 M cells, 80 MB of populations, read again after ~2 planes).
  if ((rows == ROWS_INNER || rows == ROWS_ALL) && (long long)by * c->nz < (long long)nrows &&
      c->nz <= 65535 && g->y <= 65535u) {
    *g = dim3(g->x, c->nz, g->y);
    return rows | ROWS_ZY;
  }
  return rows;
}

// Bounce-back wall passes take LBM_WALL_BLOCKS_PER_SM blocks of 128 threads per
// SM at most, shared between the wall faces, and their blocks stride over the
// nodes: the FP64 Newton bounds them, a few warps per SM keep that pipe busy,
// and the registers they leave free stay with the inner rows running beside
// them (on the 256x128x128 channel, 0.1304 ms per step against 0.1318 ms with
// one thread per node).  Regularized passes, bound by the latency of their
// gathers, keep one thread per node (capped to 1 and 2 blocks per SM their
// step took 0.224 and 0.168 ms against 0.151 ms).
#ifndef LBM_WALL_BLOCKS_PER_SM
#define LBM_WALL_BLOCKS_PER_SM 2
#endif

// One launch per wall class present (bounce-back, regularized): each kernel
// holds one scheme's code and leaves the other class's face alone.
static void launch_wall(lbm_ctx* c, const Params& p, cudaStream_t s, int prio = 0) {
  for (int cls = 0; cls < 2; ++cls) {
    const bool regularized = cls == 1;
    int maxw = 0, faces = 0;
    for (int f = 0; f < 2; ++f)
      if (p.wall[f] && (p.wall[f] != BC_WALL_BB) == regularized) {
        maxw = std::max(maxw, p.nwall[f]);
        ++faces;
      }
    if (faces == 0) continue;
    int gx = (maxw + 127) / 128;
    if (!regularized) gx = std::min(gx, std::max(1, c->sms * LBM_WALL_BLOCKS_PER_SM / faces));
    dim3 g(gx, 2, 1), b(128, 1, 1);
    if (c->Q == 9) launch_wall_q9(c->st, p, regularized, g, b, s, prio);
    else launch_wall_q19(c->st, p, regularized, g, b, s, prio);
    ++c->launches;
  }
}

static void launch_bulk(lbm_ctx* c, const Params& p, int rows, cudaStream_t s, int prio = 0) {
  if (rows == ROWS_INNER && c->tma_ok) {
    const int src = p.f_src == c->f[0] ? 0 : 1;
    if (c->Q == 9) launch_bulk_tma_q9(c->st, p, c->tmap[src], c->tma_zchunk, s);
    else launch_bulk_tma_q19(c->st, p, c->tmap[src], c->tma_zchunk, s);
    ++c->launches;
    if (!p.px) launch_bulk(c, p, ROWS_XEDGE, s, prio);   // inlet / outlet columns
    return;
  }
  dim3 g, b;
  const int rarg = lbm_ctx_bulk_launch_dims(c, rows, &g, &b);
  const bool pairs = lbm_ctx_bulk_pairs(c, rows);
  if (c->Q == 9) launch_bulk_q9(c->st, p, rarg, pairs, g, b, s, prio);
  else launch_bulk_q19(c->st, p, rarg, pairs, g, b, s, prio);
  ++c->launches;
  if (rows == ROWS_INNER && !p.px) launch_bulk(c, p, ROWS_XEDGE, s, prio);   // inlet / outlet columns
}

// Every row of a lattice without walls.  Periodic in x and y: one launch of
// the face-free kernel; otherwise the inner rows take the face-free kernel and
// only the face rows and columns the general one.
static void launch_all_rows(lbm_ctx* c, const Params& p, cudaStream_t s) {
  if ((p.px && p.py) || c->ny < 3) {
    launch_bulk(c, p, ROWS_ALL, s);
    return;
  }
  launch_bulk(c, p, ROWS_INNER, s);
  launch_bulk(c, p, ROWS_WALL, s);
}

// Whether the wall rows hold cells the wall pass does not step itself (it steps
// regularized wall nodes): bounce-back nodes, a face without a wall, or the
// columns upstream of a wall's leading edge.
static bool wall_rows_needed(const Params& p) {
  for (int f = 0; f < 2; ++f)
    if (!(p.wall[f] && p.wall[f] != BC_WALL_BB && p.xw0[f] == 0)) return true;
  return false;
}

// One step.  With walls, only the two wall rows depend on the wall pre-pass:
// the inner rows run on `s` while the side stream runs the wall pre-pass and
// then the wall rows (fork / join through events, also inside graph capture).
static void launch_step(lbm_ctx* c, int src, cudaStream_t s) {
  const Params p = lbm_ctx_params(c, src);
  if (!(p.wall[0] || p.wall[1])) {
    launch_all_rows(c, p, s);
    return;
  }
  cudaEventRecord(c->ev_fork, s);
  cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0);
  launch_wall(c, p, c->side_stream, c->prio_hi);
  if (wall_rows_needed(p)) launch_bulk(c, p, ROWS_WALL, c->side_stream, c->prio_hi);
  cudaEventRecord(c->ev_join, c->side_stream);
  launch_bulk(c, p, ROWS_INNER, s);
  cudaStreamWaitEvent(s, c->ev_join, 0);
}

extern "C" lbm_status lbm_set_fields(lbm_ctx* c, const double* rho, const double* u,
                                     const double* nu_tilde, int on_device) {
  if (!c || !rho || !u || !nu_tilde) return LBM_EINVAL;
  lbm_status s = lbm_ctx_finalize(c);
  if (s != LBM_OK) return s;
  const long long n = c->ncells;
  const double *drho = rho, *du = u, *dnt = nu_tilde;
  double* staging = nullptr;
  if (!on_device) {
    staging = host_staging(c, 5 * (size_t)n);
    if (!staging) {
      lbm_ctx_set_error(c, "staging allocation failed");
      return LBM_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(staging, rho, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(staging + n, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(staging + 4 * n, nu_tilde, n * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream);
    if (e != cudaSuccess) {
      lbm_ctx_set_error(c, "upload failed: %s", cudaGetErrorString(e));
      return LBM_ECUDA;
    }
    drho = staging;
    du = staging + n;
    dnt = staging + 4 * n;
  }
  Params p = lbm_ctx_params(c, 1 - c->cur);  // writes into buffer `cur`
  const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
  if (c->Q == 9)
    launch_init_q9(c->st, p, grid, drho, du, dnt, c->cfg.rho0, c->ucv, c->nucv, c->stream);
  else
    launch_init_q19(c->st, p, grid, drho, du, dnt, c->cfg.rho0, c->ucv, c->nucv, c->stream);
  ++c->launches;
  for (int b = 0; b < 2; ++b)
    CUDA_TRY(c, cudaMemsetAsync(c->utau[b], 0, (size_t)c->nx * c->nz * sizeof(double), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->utau_prev, 0, 2 * (size_t)c->nx * c->nz * sizeof(double), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->flags, 0, sizeof(unsigned) * 4, c->stream));
  CUDA_TRY(c, cudaGetLastError());
  if (staging) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->ready = true;
  return LBM_OK;
}

static lbm_status ensure_graph(lbm_ctx* c, int parity) {
  if (c->gvalid[parity]) return LBM_OK;
  if (c->gexec[parity]) {
    cudaGraphExecDestroy(c->gexec[parity]);
    c->gexec[parity] = nullptr;
  }
  CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  // kernels recorded into the graph are counted when it is replayed
  const unsigned long long before = c->launches;
  launch_step(c, parity, c->cap_stream);
  launch_step(c, 1 - parity, c->cap_stream);
  c->graph_launches[parity] = c->launches - before;
  c->launches = before;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != cudaSuccess) {
    lbm_ctx_set_error(c, "graph capture failed: %s", cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  e = cudaGraphInstantiate(&c->gexec[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    lbm_ctx_set_error(c, "graph instantiate failed: %s", cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  c->gvalid[parity] = true;
  return LBM_OK;
}

// Lattices with walls and at least this many cells launch their steps directly
// (see lbm_step).
constexpr long long kDirectWallCells = 1LL << 21;

extern "C" lbm_status lbm_step(lbm_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return LBM_EINVAL;
  if (!c->ready) {
    lbm_ctx_set_error(c, "lbm_set_fields (or lbm_set_state) must come first");
    return LBM_EINVAL;
  }
  lbm_status s = lbm_ctx_finalize(c);
  if (s != LBM_OK) return s;
  int left = nsteps;
  // Large lattices with walls launch each step directly: the wall pre-pass
  // branch only overlaps the inner rows when its stream priority is honoured,
  // which replayed graphs did not do on GB300 (measured 0.38 ms vs 0.21 ms per
  // step on the 256x128x128 channel).  Smaller lattices, whose steps are bound
  // by launch latency rather than by the overlap, and wall-free lattices replay
  // captured graphs of two steps.
  const bool walls = c->base.wall[0] || c->base.wall[1];
  if (walls && c->ncells >= kDirectWallCells) {
    for (; left > 0; --left) {
      launch_step(c, c->cur, c->stream);
      c->cur ^= 1;
    }
    CUDA_TRY(c, cudaGetLastError());
  }
  if (left >= 2) {
    s = ensure_graph(c, c->cur);
    if (s != LBM_OK) return s;
    while (left >= 2) {
      CUDA_TRY(c, cudaGraphLaunch(c->gexec[c->cur], c->stream));
      c->launches += c->graph_launches[c->cur];
      left -= 2;
    }
  }
  if (left == 1) {
    launch_step(c, c->cur, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    c->cur ^= 1;
  }
  c->steps_done += nsteps;
  return LBM_OK;
}

extern "C" lbm_status lbm_step_timed(lbm_ctx* c, int nsteps, float kernel_ms[3]) {
  if (!c || nsteps < 0 || !kernel_ms) return LBM_EINVAL;
  if (!c->ready) {
    lbm_ctx_set_error(c, "lbm_set_fields (or lbm_set_state) must come first");
    return LBM_EINVAL;
  }
  lbm_status s = lbm_ctx_finalize(c);
  if (s != LBM_OK) return s;
  std::vector<cudaEvent_t> ev(4 * (size_t)nsteps);
  for (auto& e : ev) CUDA_TRY(c, cudaEventCreate(&e));
  for (int k = 0; k < nsteps; ++k) {
    // the kernels of lbm_step, one after the other so that each one's duration
    // is measurable: wall pre-pass, then bulk (inner rows, then wall rows)
    const Params p = lbm_ctx_params(c, c->cur);
    const bool walls = p.wall[0] || p.wall[1];
    cudaEvent_t* e = &ev[4 * (size_t)k];
    CUDA_TRY(c, cudaEventRecord(e[0], c->stream));
    if (walls) launch_wall(c, p, c->stream);
    CUDA_TRY(c, cudaEventRecord(e[1], c->stream));
    if (walls) {
      launch_bulk(c, p, ROWS_INNER, c->stream);
      CUDA_TRY(c, cudaEventRecord(e[2], c->stream));
      if (wall_rows_needed(p)) launch_bulk(c, p, ROWS_WALL, c->stream);
    } else {
      launch_all_rows(c, p, c->stream);
      CUDA_TRY(c, cudaEventRecord(e[2], c->stream));
    }
    CUDA_TRY(c, cudaEventRecord(e[3], c->stream));
    c->cur ^= 1;
  }
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  float wall = 0.f, bulk = 0.f, inner = 0.f;
  for (int k = 0; k < nsteps; ++k) {
    const cudaEvent_t* e = &ev[4 * (size_t)k];
    float a = 0.f, b = 0.f, d = 0.f;
    cudaEventElapsedTime(&a, e[0], e[1]);
    cudaEventElapsedTime(&b, e[1], e[3]);
    cudaEventElapsedTime(&d, e[1], e[2]);
    wall += a;
    bulk += b;
    inner += d;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  kernel_ms[0] = bulk;
  kernel_ms[1] = wall;
  kernel_ms[2] = inner;
  c->steps_done += nsteps;
  return LBM_OK;
}

static lbm_status check_flags(lbm_ctx* c) {
  unsigned h[4] = {0, 0, 0, 0};
  CUDA_TRY(c, cudaMemcpyAsync(h, c->flags, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->last_flags = h[0];
  c->newton_count = h[1];
  if (h[0] & FLAG_TMA_TIMEOUT) {
    lbm_ctx_set_error(c, "a bounded wait for a tiled load expired; the state is not valid");
    return LBM_ETIMEOUT;
  }
  if (h[0] & FLAG_NONFINITE) {
    lbm_ctx_set_error(c, "non-finite value in the state");
    return LBM_ENONFINITE;
  }
  if (h[0] & FLAG_NEWTON) {
    lbm_ctx_set_error(c, "the u_tau Newton iteration reached its limit at %u wall-node updates",
                      h[1]);
    return LBM_ENEWTON;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_fields(lbm_ctx* c, unsigned mask, void* const* dst, int dst_on_device) {
  if (!c || (mask && !dst)) return LBM_EINVAL;
  if (!c->ready) {
    lbm_ctx_set_error(c, "no state yet");
    return LBM_EINVAL;
  }
  if (mask & ~0xFFu) {
    lbm_ctx_set_error(c, "unknown field bits in mask");
    return LBM_EINVAL;
  }
  const long long n = c->ncells;
  const Params p = lbm_ctx_params(c, c->cur);
  const double vel = c->cfg.dx / c->dt, visc = c->cfg.dx * c->cfg.dx / c->dt;
  const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
  int slot = 0;
  double* tmp = nullptr;
  for (int bit = 0; bit < 4; ++bit) {
    if (!(mask & (1u << bit))) continue;
    const size_t count = (bit == 1 ? 3 : 1) * (size_t)n;
    double* out = (double*)dst[slot++];
    if (!out) return LBM_EINVAL;
    double* target = out;
    if (!dst_on_device) {
      if (!tmp) tmp = host_staging(c, 3 * (size_t)n);
      if (!tmp) {
        lbm_ctx_set_error(c, "staging allocation failed");
        return LBM_ENOMEM;
      }
      target = tmp;
    }
    double* a[4] = {nullptr, nullptr, nullptr, nullptr};
    a[bit] = target;
    if (c->Q == 9)
      launch_fields_q9(c->st, p, grid, a[0], a[1], a[2], a[3], c->cfg.rho0, vel, visc, c->stream);
    else
      launch_fields_q19(c->st, p, grid, a[0], a[1], a[2], a[3], c->cfg.rho0, vel, visc, c->stream);
    ++c->launches;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dst_on_device)
      e = cudaMemcpyAsync(out, tmp, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      lbm_ctx_set_error(c, "field export failed: %s", cudaGetErrorString(e));
      return LBM_ECUDA;
    }
  }
  // wall-node arrays: u_tau and C_f = 2 (u_tau / U_ref)^2 on the (z, x) grid of each y face
  if (mask & 0xF0u) {
    const size_t nodes = (size_t)c->nx * c->nz;
    std::vector<double> ut(nodes), full(nodes);
    for (int bit = 4; bit < 8; ++bit) {
      if (!(mask & (1u << bit))) continue;
      const int fi = (bit - 4) & 1;
      const bool cf = bit >= 6;
      std::fill(full.begin(), full.end(), 0.0);
      if (c->base.wall[fi]) {
        const int nw = c->base.nwall[fi];
        CUDA_TRY(c, cudaMemcpyAsync(ut.data(), c->utau[fi], nw * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        const int x0 = c->base.xw0[fi], nwx = c->nx - x0;
        for (int m = 0; m < nw; ++m) {
          const int z = m / nwx, x = x0 + m % nwx;
          const double v = ut[m] * vel;
          full[(size_t)z * c->nx + x] = cf ? 2.0 * (v / c->cfg.u_ref) * (v / c->cfg.u_ref) : v;
        }
      }
      double* out = (double*)dst[slot++];
      if (!out) return LBM_EINVAL;
      if (dst_on_device)
        CUDA_TRY(c, cudaMemcpyAsync(out, full.data(), nodes * sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream));
      else
        std::memcpy(out, full.data(), nodes * sizeof(double));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
  }
  return check_flags(c);
}

extern "C" lbm_status lbm_diagnostics(lbm_ctx* c, lbm_diag* out) {
  if (!c || !out) return LBM_EINVAL;
  if (!c->ready) {
    lbm_ctx_set_error(c, "no state yet");
    return LBM_EINVAL;
  }
  const Params p = lbm_ctx_params(c, c->cur);
  if (c->Q == 9) launch_reduce_q9(c->st, p, c->red_blocks, c->partial, c->red_chunk, c->stream);
  else launch_reduce_q19(c->st, p, c->red_blocks, c->partial, c->red_chunk, c->stream);
  launch_reduce_final(c->partial, c->red_blocks, c->red_out, c->stream);
  launch_wall_stats(p, c->utau_prev, c->red_out + 8, c->stream);
  c->launches += 3;
  CUDA_TRY(c, cudaGetLastError());
  double h[16];
  CUDA_TRY(c, cudaMemcpyAsync(h, c->red_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  lbm_status s = check_flags(c);
  const double vel = c->cfg.dx / c->dt;
  out->mass = h[0];
  // populations are stored relative to f^eq(1, U x): each cell carries U more x-momentum
  out->momentum[0] = h[1] + c->base.Ush * (double)c->ncells;
  out->momentum[1] = h[2];
  out->momentum[2] = h[3];
  out->mean_u_tau[0] = h[8] * vel;
  out->mean_u_tau[1] = h[9] * vel;
  out->max_rel_du_tau = h[10];
  out->nonfinite = (c->last_flags & FLAG_NONFINITE) ? 1 : 0;
  out->newton_failures = (int)std::min<unsigned>(c->newton_count, 0x7fffffffu);
  // non-finite values and Newton failures are reported in *out, not as errors
  return (s == LBM_ENONFINITE || s == LBM_ENEWTON) ? LBM_OK : s;
}

extern "C" lbm_status lbm_run_to_convergence(lbm_ctx* c, double tol, int check_every,
                                             long long max_steps, long long* steps_done,
                                             double* residual) {
  if (!c || !(tol > 0.0) || check_every < 1 || max_steps < 0 || !steps_done || !residual)
    return LBM_EINVAL;
  if (!c->ready) {
    lbm_ctx_set_error(c, "lbm_set_fields (or lbm_set_state) must come first");
    return LBM_EINVAL;
  }
  lbm_status s = lbm_ctx_finalize(c);
  if (s != LBM_OK) return s;
  if (!(c->base.wall[0] || c->base.wall[1])) {
    lbm_ctx_set_error(c, "the convergence test needs a wall (it watches u_tau)");
    return LBM_EINVAL;
  }
  *steps_done = 0;
  *residual = INFINITY;
  // the u_tau of the starting state is the first reference
  launch_wall_stats(lbm_ctx_params(c, c->cur), c->utau_prev, c->red_out + 8, c->stream);
  ++c->launches;
  long long done = 0;
  double res = INFINITY;
  while (done < max_steps) {
    const int n = (int)std::min<long long>(check_every, max_steps - done);
    s = lbm_step(c, n);
    if (s != LBM_OK) return s;
    done += n;
    launch_wall_stats(lbm_ctx_params(c, c->cur), c->utau_prev, c->red_out + 8, c->stream);
    ++c->launches;
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(&res, c->red_out + 10, sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    s = check_flags(c);   // synchronises the stream
    *steps_done = done;
    *residual = res;
    if (s != LBM_OK) return s;
    if (res < tol) break;
  }
  return LBM_OK;
}

extern "C" size_t lbm_state_bytes(const lbm_ctx* c) {
  if (!c) return 0;
  return (size_t)c->Q * c->ncell * c->esz + (size_t)4 * c->ncell * c->rsz +
         2 * (size_t)c->nx * c->nz * sizeof(double);
}

extern "C" lbm_status lbm_get_state(lbm_ctx* c, void* dst) {
  if (!c || !dst) return LBM_EINVAL;
  if (!c->ready) {
    lbm_ctx_set_error(c, "no state yet");
    return LBM_EINVAL;
  }
  char* o = (char*)dst;
  const size_t fb = (size_t)c->Q * c->ncell * c->esz, vb = 4 * (size_t)c->ncell * c->rsz,
               wb = (size_t)c->nx * c->nz * sizeof(double);
  CUDA_TRY(c, cudaMemcpyAsync(o, c->f[c->cur], fb, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(o + fb, c->v[c->cur], vb, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(o + fb + vb, c->utau[0], wb, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(o + fb + vb + wb, c->utau[1], wb, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

extern "C" lbm_status lbm_set_state(lbm_ctx* c, const void* src) {
  if (!c || !src) return LBM_EINVAL;
  lbm_status s = lbm_ctx_finalize(c);
  if (s != LBM_OK) return s;
  const char* o = (const char*)src;
  const size_t fb = (size_t)c->Q * c->ncell * c->esz, vb = 4 * (size_t)c->ncell * c->rsz,
               wb = (size_t)c->nx * c->nz * sizeof(double);
  CUDA_TRY(c, cudaMemcpyAsync(c->f[c->cur], o, fb, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->v[c->cur], o + fb, vb, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->utau[0], o + fb + vb, wb, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->utau[1], o + fb + vb + wb, wb, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->flags, 0, sizeof(unsigned) * 4, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->ready = true;
  return LBM_OK;
}

extern "C" lbm_status lbm_lattice_params(const lbm_ctx* c, double out[6]) {
  if (!c || !out) return LBM_EINVAL;
  out[0] = c->dt;
  out[1] = c->nu_lb;
  out[2] = 0.5 + 3.0 * c->nu_lb;
  out[3] = c->F_lb[0];
  out[4] = c->F_lb[1];
  out[5] = c->F_lb[2];
  return LBM_OK;
}

extern "C" void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (int p = 0; p < 2; ++p)
    if (c->gexec[p]) cudaGraphExecDestroy(c->gexec[p]);
  for (void* ptr : c->allocs) {
    if (c->cfg.free) c->cfg.free(ptr, c->cfg.alloc_user);
    else if (!c->cfg.alloc) cudaFree(ptr);
  }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

extern "C" unsigned long long lbm_kernel_launches(const lbm_ctx* c) {
  return c ? c->launches : 0ULL;
}

extern "C" long long lbm_steps_done(const lbm_ctx* c) { return c ? c->steps_done : -1; }

extern "C" lbm_status lbm_set_wait_limit(lbm_ctx* c, long long polls) {
  if (!c || polls < 0) return LBM_EINVAL;
  c->wait_limit = polls;
  c->finalized = false;   // the limit is a kernel parameter: rebuild them (and the graphs)
  c->gvalid[0] = c->gvalid[1] = false;
  return LBM_OK;
}
