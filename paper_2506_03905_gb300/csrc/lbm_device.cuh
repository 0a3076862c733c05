// lbm_device.cuh -- device-side building blocks of the LBM-RANS step.
//
// Lattice units throughout (dx = dt = 1, c_s^2 = 1/3).  Populations are stored
// as deviations h_i = f_i - E_i from the equilibrium at rest density and a
// constant reference velocity U along x, E_i = f_i^eq(1, U x) (U = 0 gives
// h_i = f_i - w_i).  All arithmetic runs on these small deviations in the
// compute type R (float, or double for the FP64 mode): a force or viscous
// increment per step is then many ulps of the stored value instead of a few.
//
// Memory layout (structure of arrays, x fastest, rows padded to `pitch`):
//   f[q][z][y][x]  -> f[q * ncell + (z*ny + y)*pitch + x]
//   v[z][y][x][4] -> v[4 * ((z*ny + y)*pitch + x) + k]: per cell the record
//                    (u_x, u_y, u_z, nu_tilde) of the previous step, so that the
//                    SA stencil reads a neighbour with one vector load
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

// Loads of the population and SA-field buffers.  The step kernels read buffers
// that no thread of the same launch writes, so they mark their pointers
// __restrict__ and read the records through the read-only path.  A persistent
// kernel that advances several steps in one launch (the batch) reads data other
// CTAs wrote earlier in the same launch: its translation unit defines
// LBM_COHERENT_LOADS, which turns both off, so that every such load is a plain
// global load ordered by the kernel's own fences.
#ifdef LBM_COHERENT_LOADS
#define LBM_RESTRICT
#define LBM_LDG(p) (*(p))
#else
#define LBM_RESTRICT __restrict__
#define LBM_LDG(p) __ldg(p)
#endif

namespace lbm {

enum BcKind {
  BC_PERIODIC = 0, BC_WALL_BB = 1, BC_WALL_HRFD = 2, BC_SYMMETRY = 3,
  BC_INLET = 4, BC_OUTLET = 5, BC_FREESTREAM = 6, BC_WALL_CAI = 7
};
enum { XMIN = 0, XMAX = 1, YMIN = 2, YMAX = 3 };
enum { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2, ST_FP64 = 3 };
// collision operator of a kernel instantiation (Params::collision: 0 BGK, 1 regularized)
enum { COLL_ANY = -1, COLL_BGK = 0, COLL_REG = 1 };
// flags[0]: failure bits; flags[1]: wall-node updates whose Newton iteration
// reached its limit (count); flags[2..3] unused
enum { FLAG_NONFINITE = 1u, FLAG_NEWTON = 2u, FLAG_TMA_TIMEOUT = 4u };
// k_bulk row sets: ROWS_ALL every row; ROWS_INNER rows 1..ny-2 (independent of
// the wall pre-pass, so they run concurrently with it) without the x-face
// columns of a non-periodic x axis; ROWS_WALL rows 0, ny-1.  ROWS_XEDGE:
// columns 0 and nx-1 of rows 1..ny-2 (the x-face cells of a non-periodic x
// axis, which both inner-row kernels leave out).
enum { ROWS_ALL = 0, ROWS_INNER = 1, ROWS_WALL = 2, ROWS_XEDGE = 3 };
// Flag on a row set: the launch grid holds the z planes in y and the row tiles
// in z, so that consecutive blocks step through z before y (the blocks that
// re-read a plane's neighbours then run close together; see
// lbm_ctx_bulk_launch_dims).
enum { ROWS_ZY = 16, ROWS_MASK = 15 };
// threads per k_bulk block (x fastest: 32 x 2 cells for nx >= 32)
#ifndef LBM_BULK_THREADS
#define LBM_BULK_THREADS 64
#endif
// 1: the face-free rows run two cells per thread (k_bulk2); 0: one (k_bulk)
#ifndef LBM_BULK_PAIRS
#define LBM_BULK_PAIRS 1
#endif
constexpr int RED_THREADS = 256;   // FP64 reduction block size
constexpr int RED_VALS = 4;        // mass, momentum x/y/z

// --------------------------------------------------------------------------
// Velocity sets.  D2Q9: rest, 4 axis, 4 diagonal.  D3Q19: rest, 6 axis, 12
// edge diagonals.  Directions 2k-1 and 2k are opposite (k >= 1).
// --------------------------------------------------------------------------
template <int Q> struct Lat;

template <> struct Lat<9> {
  static constexpr int Q = 9, D = 2;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                             {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  // index of the direction with c_y negated
  __host__ __device__ static constexpr int my(int i) {
    constexpr int t[9] = {0, 1, 2, 4, 3, 7, 8, 5, 6};
    return t[i];
  }
};

template <> struct Lat<19> {
  static constexpr int Q = 19, D = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int my(int i) {
    constexpr int t[19] = {0, 1, 2, 4, 3, 5, 6, 9, 10, 7, 8, 11, 12, 13, 14, 18, 17, 16, 15};
    return t[i];
  }
};

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// --------------------------------------------------------------------------
// Storage codecs: shifted deviation g = f - w in the storage type.
// FP16 values are kept multiplied by 2^12 so that deviations down to ~1e-8
// stay in the normal range (|g| < 16 is always representable).
// --------------------------------------------------------------------------
template <int ST> struct Codec;
// ld / st convert between storage and deviations in the compute type; the
// raw forms leave the storage scale kScale in (stored value = kScale x h),
// for the interior path, whose collision takes the scale into its constants.
template <> struct Codec<ST_FP32> {
  using T = float;
  static constexpr int kScale = 1;
  __device__ static __forceinline__ float ld(const T* p) { return *p; }
  __device__ static __forceinline__ void st(T* p, float v) { *p = v; }
  __device__ static __forceinline__ float ld_raw(const T* p) { return *p; }
  __device__ static __forceinline__ void st_raw(T* p, float v) { *p = v; }
  // two neighbouring elements p[0], p[1] (p 2-element aligned) in one access
  __device__ static __forceinline__ void ld2_raw(const T* p, float* a, float* b) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    *a = v.x;
    *b = v.y;
  }
  __device__ static __forceinline__ void st2_raw(T* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  }
  // a pair of raw values as loaded (P2), read from p[0], p[1] in one access or
  // from two addresses, and its two values in the compute type
  using P2 = float2;
  __device__ static __forceinline__ P2 ld_pair(const T* p) { return *reinterpret_cast<const float2*>(p); }
  __device__ static __forceinline__ P2 pair(const T* a, const T* b) { return make_float2(*a, *b); }
  __device__ static __forceinline__ float lo(P2 v) { return v.x; }
  __device__ static __forceinline__ float hi(P2 v) { return v.y; }
  __device__ static __forceinline__ float2 both(P2 v) { return v; }
};
template <> struct Codec<ST_FP64> {
  using T = double;
  static constexpr int kScale = 1;
  __device__ static __forceinline__ double ld(const T* p) { return *p; }
  __device__ static __forceinline__ void st(T* p, double v) { *p = v; }
  __device__ static __forceinline__ double ld_raw(const T* p) { return *p; }
  __device__ static __forceinline__ void st_raw(T* p, double v) { *p = v; }
  __device__ static __forceinline__ void ld2_raw(const T* p, double* a, double* b) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    *a = v.x;
    *b = v.y;
  }
  __device__ static __forceinline__ void st2_raw(T* p, double a, double b) {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
  }
  using P2 = double2;
  __device__ static __forceinline__ P2 ld_pair(const T* p) { return *reinterpret_cast<const double2*>(p); }
  __device__ static __forceinline__ P2 pair(const T* a, const T* b) { return make_double2(*a, *b); }
  __device__ static __forceinline__ double lo(P2 v) { return v.x; }
  __device__ static __forceinline__ double hi(P2 v) { return v.y; }
};
template <> struct Codec<ST_FP16> {
  using T = __half;
  static constexpr int kScale = 4096;   // 2^12: deviations of O(1e-4) keep 11 bits in FP16
  __device__ static __forceinline__ float ld(const T* p) { return __half2float(*p) * (1.0f / 4096.0f); }
  __device__ static __forceinline__ void st(T* p, float v) { *p = __float2half_rn(v * 4096.0f); }
  __device__ static __forceinline__ float ld_raw(const T* p) { return __half2float(*p); }
  __device__ static __forceinline__ void st_raw(T* p, float v) { *p = __float2half_rn(v); }
  __device__ static __forceinline__ void ld2_raw(const T* p, float* a, float* b) {
    const __half2 v = *reinterpret_cast<const __half2*>(p);
    *a = __low2float(v);
    *b = __high2float(v);
  }
  __device__ static __forceinline__ void st2_raw(T* p, float a, float b) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);   // one packed conversion
  }
  // a pair stays in one 32-bit register until it is converted
  using P2 = __half2;
  __device__ static __forceinline__ P2 ld_pair(const T* p) { return *reinterpret_cast<const __half2*>(p); }
  __device__ static __forceinline__ P2 pair(const T* a, const T* b) { return __halves2half2(*a, *b); }
  __device__ static __forceinline__ float lo(P2 v) { return __low2float(v); }
  __device__ static __forceinline__ float hi(P2 v) { return __high2float(v); }
  __device__ static __forceinline__ float2 both(P2 v) { return __half22float2(v); }
};
template <> struct Codec<ST_BF16> {
  using T = __nv_bfloat16;
  static constexpr int kScale = 1;
  __device__ static __forceinline__ float ld(const T* p) { return __bfloat162float(*p); }
  __device__ static __forceinline__ void st(T* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ static __forceinline__ float ld_raw(const T* p) { return __bfloat162float(*p); }
  __device__ static __forceinline__ void st_raw(T* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ static __forceinline__ void ld2_raw(const T* p, float* a, float* b) {
    const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
    *a = __low2float(v);
    *b = __high2float(v);
  }
  __device__ static __forceinline__ void st2_raw(T* p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
  }
  using P2 = __nv_bfloat162;
  __device__ static __forceinline__ P2 ld_pair(const T* p) {
    return *reinterpret_cast<const __nv_bfloat162*>(p);
  }
  __device__ static __forceinline__ P2 pair(const T* a, const T* b) { return __halves2bfloat162(*a, *b); }
  __device__ static __forceinline__ float lo(P2 v) { return __low2float(v); }
  __device__ static __forceinline__ float hi(P2 v) { return __high2float(v); }
  __device__ static __forceinline__ float2 both(P2 v) { return __bfloat1622float2(v); }
};
template <int ST> struct Compute { using R = float; };
template <> struct Compute<ST_FP64> { using R = double; };

// Arithmetic helpers: FP32 uses the fast hardware reciprocal-based divide and
// power (a few ulp, far below the 1e-5 parity tolerance); FP64 stays exact.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
// fused multiply-add in the compute type
__device__ __forceinline__ float fmaf_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaf_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float pow_sixth(float x) { return __powf(x, 1.0f / 6.0f); }
__device__ __forceinline__ double pow_sixth(double x) { return pow(x, 1.0 / 6.0); }
// square root of a non-negative value: x * rsqrt(x) (2 ulp) in FP32, exact in FP64
__device__ __forceinline__ float nn_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ double nn_sqrt(double x) { return sqrt(x); }

// --------------------------------------------------------------------------
// Two FP32 lanes in one value: cell A in .x, cell B in .y.  Sums, products and
// fused multiply-adds issue as one packed instruction for both lanes (add /
// mul / fma on .f32x2, sm_100 and later); each lane is rounded exactly as the
// scalar instruction rounds it.  Divisions, square roots and powers have no
// packed form and run per lane.  The two-cells-per-thread kernels compute on
// this type, which halves their issued FP32 arithmetic.
// --------------------------------------------------------------------------
struct f2 {
  float2 v;
  f2() = default;
  __device__ __forceinline__ f2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit f2(float2 a) : v(a) {}
  __device__ __forceinline__ explicit f2(double a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ explicit f2(int a) : v(make_float2((float)a, (float)a)) {}
};
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.v.x, -a.v.y); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2& operator*=(f2& a, f2 b) { return a = a * b; }
__device__ __forceinline__ f2 fmaf_r(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
// a / b: one approximate reciprocal per lane, the product packed
__device__ __forceinline__ f2 fdiv(f2 a, f2 b) {
  return a * f2(__fdividef(1.0f, b.v.x), __fdividef(1.0f, b.v.y));
}
__device__ __forceinline__ f2 pow_sixth(f2 x) { return f2(pow_sixth(x.v.x), pow_sixth(x.v.y)); }
__device__ __forceinline__ f2 nn_sqrt(f2 x) {
  const f2 r(x.v.x > 0.0f ? rsqrtf(x.v.x) : 0.0f, x.v.y > 0.0f ? rsqrtf(x.v.y) : 0.0f);
  return x * r;
}

// Per-lane comparisons and selections of the compute types (float, double, f2).
// sel_pos(c, a, b) = c > 0 ? a : b; pos_part(x) = x > 0 ? x : 0;
// min_lt(q, r) = q < r ? q : r; all_ge(a, b): a >= b in every lane;
// sel_ge(a, b, x, y) = a >= b ? x : y; any_pos(x): x > 0 in some lane.
template <class R> __device__ __forceinline__ R sel_pos(R c, R a, R b) { return c > (R)0 ? a : b; }
template <class R> __device__ __forceinline__ R pos_part(R x) { return x > (R)0 ? x : (R)0; }
template <class R> __device__ __forceinline__ R min_lt(R q, R r) { return q < r ? q : r; }
template <class R> __device__ __forceinline__ bool all_ge(R a, R b) { return a >= b; }
template <class R> __device__ __forceinline__ R sel_ge(R a, R b, R x, R y) { return a >= b ? x : y; }
template <class R> __device__ __forceinline__ bool any_pos(R x) { return x > (R)0; }
template <> __device__ __forceinline__ f2 sel_pos(f2 c, f2 a, f2 b) {
  return f2(c.v.x > 0.0f ? a.v.x : b.v.x, c.v.y > 0.0f ? a.v.y : b.v.y);
}
template <> __device__ __forceinline__ f2 pos_part(f2 x) {
  return f2(x.v.x > 0.0f ? x.v.x : 0.0f, x.v.y > 0.0f ? x.v.y : 0.0f);
}
template <> __device__ __forceinline__ f2 min_lt(f2 q, f2 r) {
  return f2(q.v.x < r.v.x ? q.v.x : r.v.x, q.v.y < r.v.y ? q.v.y : r.v.y);
}
template <> __device__ __forceinline__ bool all_ge(f2 a, f2 b) { return a.v.x >= b.v.x && a.v.y >= b.v.y; }
template <> __device__ __forceinline__ f2 sel_ge(f2 a, f2 b, f2 x, f2 y) {
  return f2(a.v.x >= b.v.x ? x.v.x : y.v.x, a.v.y >= b.v.y ? x.v.y : y.v.y);
}
template <> __device__ __forceinline__ bool any_pos(f2 x) { return x.v.x > 0.0f || x.v.y > 0.0f; }

// --------------------------------------------------------------------------
// Kernel parameters (lattice units), passed by value.
// --------------------------------------------------------------------------
struct Params {
  int nx, ny, nz, pitch;
  long long ncell;             // pitch * ny * nz: stride between directions / components
  int collision;               // 0 BGK, 1 regularized
  int turbulent;               // 1: SA active
  int wall_law;                // 0 Eq. 16, 1 log law
  int has_force;
  double nu;                   // molecular viscosity (lattice)
  double inv_nu;               // 1 / nu
  double F[3];                 // body force density (lattice)
  double guoA[19];             // 3 w_i c_i.F per direction (Guo forcing coefficient)
  double Ush;                  // reference velocity U (x) of the stored deviations
  // float copies for the FP32 kernels: converting a double per thread would run
  // on the FP64 pipe, which on GB300 has 1/64 of the FP32 rate
  float nu_f, inv_nu_f, F_f[3], guoA_f[19], Ush_f, xs_lb_f[2], u_face_f[4][3], nt_face_f[4], d_w_f[2],
      ibb_f[2][4];
  double law_kappa, law_B;
  int kind[6];                 // face kinds
  int px, py;                  // x / y periodic
  // y faces, index 0 = ymin, 1 = ymax
  int wall[2];                 // 0 or BC_WALL_BB / BC_WALL_HRFD
  int xw0[2];                  // first wall column (columns before it are symmetry)
  double xs_lb[2];             // leading edge position in lattice units from the x face
  double beta[2];
  int ref_node[2];
  double d_w[2];               // wall-to-boundary-node distance / Delta (1/2: half-way)
  int interp[2];               // bounce-back walls: 0 half-way, 1 Bouzidi, 2 Yu
  // bounce-back rule of each y face as affine weights (a_o, a_F, a_i, a_K) of
  //   h_i(B) = a_o h*_opp(B) + a_F h*_opp(B + c_i) + a_i h*_i(B) + a_K K,
  //   K = 6 w_i (rho_w c_i.u_w - c_ix U)
  // for an incoming direction i (Eq. 31: 1, 0, 0, 1; Eqs. 36-37: ibb_weights)
  double ibb[2][4];
  int nwall[2];                // (nx - xw0) * nz wall nodes
  double u_face[4][3];         // prescribed velocity of xmin, xmax, ymin, ymax
  double nt_face[4];           // prescribed nu_tilde of xmin, xmax, ymin, ymax
  // state
  const void* f_src;
  void* f_dst;
  const void* v_src;           // SA-field records (u_x, u_y, u_z, nu_tilde), compute type
  void* v_dst;
  double* utau[2];             // per wall node, FP64 (also the Newton warm start)
  void* uw[2];                 // BB: slip velocity (3 per node), compute type
  void* rhow[2];               // BB: wall density, compute type
  const void* invd2;           // 1 / d^2 (wall distance of the SA model), compute type, [y][x]
  unsigned* flags;
  long long wait_limit;        // polls of a bounded device-side wait before it gives up
};

// Parameter in the compute type: the float copy for FP32, the double for FP64.
template <class R> __device__ __forceinline__ R psel(double d, float f);
template <> __device__ __forceinline__ float psel<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double psel<double>(double d, float) { return d; }
template <> __device__ __forceinline__ f2 psel<f2>(double, float f) { return f2(f); }

// SA-field record of a cell: the velocity and nu_tilde, stored together (16 B
// in FP32, 32 B in FP64).  ld_rec reads a record of the source buffer with one
// vector load (through the read-only path unless LBM_COHERENT_LOADS); st_rec
// writes one with vector stores.
template <class R> struct Rec {
  R x, y, z, n;   // u_x, u_y, u_z, nu_tilde
};
template <class I> __device__ __forceinline__ Rec<float> ld_rec(const float* v, I id) {
  const float4 a = LBM_LDG(reinterpret_cast<const float4*>(v) + id);
  return {a.x, a.y, a.z, a.w};
}
template <class I> __device__ __forceinline__ Rec<double> ld_rec(const double* v, I id) {
  const double2* q = reinterpret_cast<const double2*>(v) + 2 * id;
  const double2 a = LBM_LDG(q), b = LBM_LDG(q + 1);
  return {a.x, a.y, b.x, b.y};
}
template <class I>
__device__ __forceinline__ void st_rec(float* v, I id, float x, float y, float z, float n) {
  reinterpret_cast<float4*>(v)[id] = make_float4(x, y, z, n);
}
template <class I>
__device__ __forceinline__ void st_rec(double* v, I id, double x, double y, double z, double n) {
  double2* q = reinterpret_cast<double2*>(v) + 2 * id;
  q[0] = make_double2(x, y);
  q[1] = make_double2(z, n);
}

__device__ __forceinline__ long long cidx(const Params& p, int x, int y, int z) {
  return ((long long)z * p.ny + y) * p.pitch + x;
}

// --------------------------------------------------------------------------
// Spalart-Allmaras model (Section 2.2, Eqs. 10-14) and its stencil.
// --------------------------------------------------------------------------
struct SAConst {
  static constexpr double cb1 = 0.1355, cb2 = 0.622, sigma = 2.0 / 3.0, kappa = 0.41;
  static constexpr double cw2 = 0.3, cw3 = 2.0, cv1 = 7.1, rlim = 10.0;
  static constexpr double cv2lim = 0.7, cv3lim = 0.9;
};

// nu_t = nu_tilde f_v1(nu_tilde / nu) (Eq. 10); inv_nu = 1 / nu
template <class R> __device__ __forceinline__ R sa_nut(R nt, R inv_nu) {
  const R chi = nt * inv_nu;
  const R c3 = chi * chi * chi;
  return nt * fdiv(c3, c3 + (R)(SAConst::cv1 * SAConst::cv1 * SAConst::cv1));
}

// P - D of Eq. 12 with S~ (Eq. 13, kept positive by the ICCFD7 limiter) and r, f_w (Eq. 14)
template <class R> __device__ __forceinline__ R sa_source(R nt, R S, R inv_nu, R inv_d2) {
  constexpr double k2 = SAConst::kappa * SAConst::kappa;
  const R cw1 = (R)(SAConst::cb1 / k2 + (1.0 + SAConst::cb2) / SAConst::sigma);
  const R chi = nt * inv_nu;
  const R c3 = chi * chi * chi;
  const R fv1 = fdiv(c3, c3 + (R)(SAConst::cv1 * SAConst::cv1 * SAConst::cv1));
  const R fv2 = (R)1 - fdiv(chi, (R)1 + chi * fv1);
  const R inv_kd2 = inv_d2 * (R)(1.0 / k2);
  const R sbar = nt * fv2 * inv_kd2;
  const R lim = -(R)SAConst::cv2lim * S;
  R st = S + sbar;
  if (!all_ge(sbar, lim))
    st = sel_ge(sbar, lim, st,
                S + fdiv(S * ((R)(SAConst::cv2lim * SAConst::cv2lim) * S + (R)SAConst::cv3lim * sbar),
                         (R)(SAConst::cv3lim - 2.0 * SAConst::cv2lim) * S - sbar));
  R r = (R)SAConst::rlim;
  if (any_pos(st)) r = sel_pos(st, min_lt(fdiv(nt * inv_kd2, st), r), r);
  const R r2 = r * r, r6 = r2 * r2 * r2;
  const R g = r + (R)SAConst::cw2 * (r6 - r);
  const R g2 = g * g, g6 = g2 * g2 * g2;
  const R cw36 = (R)64;  // c_w3^6
  const R fw = g * pow_sixth(fdiv((R)65, g6 + cw36));   // (1 + c_w3^6) / (g^6 + c_w3^6)
  return (R)SAConst::cb1 * st * nt - cw1 * fw * nt * nt * inv_d2;
}

// Neighbour nu_tilde and velocity with the face ghost rules of the SA stencil:
// periodic wrap; symmetry and wall faces mirror (normal velocity negated);
// inlet and free-stream faces the prescribed state; outlet zero gradient.
template <class R> struct Nb {
  R nt;
  R u[3];
};

template <class R>
__device__ __forceinline__ Nb<R> load_nb(const Params& p, const R* LBM_RESTRICT v, int x, int y,
                                         int z) {
  const Rec<R> r = ld_rec(v, cidx(p, x, y, z));
  Nb<R> n;
  n.nt = r.n;
  n.u[0] = r.x;
  n.u[1] = r.y;
  n.u[2] = r.z;
  return n;
}

template <class R>
__device__ Nb<R> neighbour(const Params& p, const R* LBM_RESTRICT v, int x, int y, int z,
                           int axis, int s) {
  if (axis == 0) {
    int xn = x + s;
    if (xn >= 0 && xn < p.nx) return load_nb<R>(p, v, xn, y, z);
    if (p.px) return load_nb<R>(p, v, xn < 0 ? xn + p.nx : xn - p.nx, y, z);
    const int f = xn < 0 ? XMIN : XMAX;
    const int k = p.kind[f];
    if (k == BC_OUTLET) return load_nb<R>(p, v, x, y, z);
    Nb<R> n;  // inlet (and any prescribed face)
    n.nt = psel<R>(p.nt_face[f], p.nt_face_f[f]);
    n.u[0] = psel<R>(p.u_face[f][0], p.u_face_f[f][0]);
    n.u[1] = psel<R>(p.u_face[f][1], p.u_face_f[f][1]);
    n.u[2] = psel<R>(p.u_face[f][2], p.u_face_f[f][2]);
    return n;
  }
  if (axis == 1) {
    int yn = y + s;
    if (yn >= 0 && yn < p.ny) return load_nb<R>(p, v, x, yn, z);
    if (p.py) return load_nb<R>(p, v, x, yn < 0 ? yn + p.ny : yn - p.ny, z);
    const int f = yn < 0 ? YMIN : YMAX;
    const int k = p.kind[f];
    if (k == BC_FREESTREAM) {
      Nb<R> n;
      n.nt = psel<R>(p.nt_face[f], p.nt_face_f[f]);
      n.u[0] = psel<R>(p.u_face[f][0], p.u_face_f[f][0]);
      n.u[1] = psel<R>(p.u_face[f][1], p.u_face_f[f][1]);
      n.u[2] = psel<R>(p.u_face[f][2], p.u_face_f[f][2]);
      return n;
    }
    Nb<R> n = load_nb<R>(p, v, x, y, z);  // mirror
    n.u[1] = -n.u[1];
    return n;
  }
  int zn = z + s;
  zn = zn < 0 ? zn + p.nz : (zn >= p.nz ? zn - p.nz : zn);
  return load_nb<R>(p, v, x, y, zn);
}

// 1 / d^2 with d the distance from the cell centre to the nearest wall (0
// without walls): a wall face is the line d_w below the first (above the
// last) row, a wall with a leading edge at x_start the half-line x >= x_start,
// and upstream cells measure to its edge point.  The context tabulates it per
// (y, x) when its faces are set (lbm_ctx_finalize); the kernels read the table.
template <class R> __device__ __forceinline__ R inv_wall_dist2(const Params& p, int x, int y) {
  return __ldg((const R*)p.invd2 + (y * p.pitch + x));
}

// Explicit Euler update of Eq. 11 at one cell, clipped at zero.
template <class R, bool THREE_D>
__device__ R sa_update(const Params& p, const R* LBM_RESTRICT v, int x, int y, int z) {
  const Nb<R> c = load_nb<R>(p, v, x, y, z);
  const R nu = psel<R>(p.nu, p.nu_f);
  Nb<R> m[3], pl[3];
  m[0] = neighbour<R>(p, v, x, y, z, 0, -1);
  pl[0] = neighbour<R>(p, v, x, y, z, 0, +1);
  m[1] = neighbour<R>(p, v, x, y, z, 1, -1);
  pl[1] = neighbour<R>(p, v, x, y, z, 1, +1);
  if (THREE_D) {
    m[2] = neighbour<R>(p, v, x, y, z, 2, -1);
    pl[2] = neighbour<R>(p, v, x, y, z, 2, +1);
  } else {
    m[2] = c;
    pl[2] = c;
  }
  const R h = (R)0.5;
  // vorticity by central differences of the previous-step velocity
  const R wx = h * (pl[1].u[2] - m[1].u[2]) - h * (pl[2].u[1] - m[2].u[1]);
  const R wy = h * (pl[2].u[0] - m[2].u[0]) - h * (pl[0].u[2] - m[0].u[2]);
  const R wz = h * (pl[0].u[1] - m[0].u[1]) - h * (pl[1].u[0] - m[1].u[0]);
  const R S = nn_sqrt(wx * wx + wy * wy + wz * wz);
  R conv = 0, diff = 0, grad2 = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R ua = c.u[a];
    conv += ua > (R)0 ? ua * (c.nt - m[a].nt) : ua * (pl[a].nt - c.nt);
    diff += (nu + h * (c.nt + pl[a].nt)) * (pl[a].nt - c.nt) -
            (nu + h * (c.nt + m[a].nt)) * (c.nt - m[a].nt);
    const R g = h * (pl[a].nt - m[a].nt);
    grad2 += g * g;
  }
  const R inv_d2 = inv_wall_dist2<R>(p, x, y);
  const R rhs = -conv + sa_source<R>(c.nt, S, psel<R>(p.inv_nu, p.inv_nu_f), inv_d2) +
                (diff + (R)SAConst::cb2 * grad2) * (R)(1.0 / SAConst::sigma);
  const R nn = c.nt + rhs;
  return nn > (R)0 ? nn : (R)0;
}

// Same update for a cell whose six neighbours are all inside the lattice or
// periodic, from the seven records of the stencil (no ghost logic): x
// neighbours give nu_tilde, u_y, u_z; y neighbours nu_tilde, u_x, u_z; z
// neighbours nu_tilde, u_x, u_y.
template <class R, bool THREE_D>
__device__ __forceinline__ R sa_core(const Params& p, const Rec<R>& cc, const Rec<R>& xm,
                                     const Rec<R>& xp, const Rec<R>& ym, const Rec<R>& yp,
                                     const Rec<R>& zm, const Rec<R>& zp, R inv_d2) {
  const R nu = psel<R>(p.nu, p.nu_f);
  const R h = (R)0.5;
  const R c = cc.n;
  R ntm[3], ntp[3];
  ntm[0] = xm.n;
  ntp[0] = xp.n;
  ntm[1] = ym.n;
  ntp[1] = yp.n;
  const R ux = cc.x, uy = cc.y, uz = THREE_D ? cc.z : (R)0;
  // vorticity by central differences of the previous-step velocity
  R wz = h * ((xp.y - xm.y) - (yp.x - ym.x));
  R S2 = wz * wz;
  if (THREE_D) {
    ntm[2] = zm.n;
    ntp[2] = zp.n;
    const R wx = h * ((yp.z - ym.z) - (zp.y - zm.y));
    const R wy = h * ((zp.x - zm.x) - (xp.z - xm.z));
    S2 += wx * wx + wy * wy;
  } else {
    ntm[2] = c;
    ntp[2] = c;
  }
  const R S = nn_sqrt(S2);
  const R ua[3] = {ux, uy, uz};
  R conv = 0, diff = 0, grad2 = 0;
#pragma unroll
  for (int a = 0; a < (THREE_D ? 3 : 2); ++a) {
    conv += ua[a] * sel_pos(ua[a], c - ntm[a], ntp[a] - c);
    diff += (nu + h * (c + ntp[a])) * (ntp[a] - c) - (nu + h * (c + ntm[a])) * (c - ntm[a]);
    const R g = h * (ntp[a] - ntm[a]);
    grad2 += g * g;
  }
  const R rhs = -conv + sa_source<R>(c, S, psel<R>(p.inv_nu, p.inv_nu_f), inv_d2) +
                (diff + (R)SAConst::cb2 * grad2) * (R)(1.0 / SAConst::sigma);
  return pos_part(c + rhs);
}

// One cell with in-lattice or periodic neighbours (periodic z handled by the
// plane offsets ozm / ozp).
template <class R, bool THREE_D>
__device__ __forceinline__ R sa_update_interior(const Params& p, const R* LBM_RESTRICT v, int id,
                                                int oxm, int oxp, int oym, int oyp, int ozm,
                                                int ozp, int x, int y) {
  const Rec<R> cc = ld_rec(v, id);
  const Rec<R> xm = ld_rec(v, id + oxm), xp = ld_rec(v, id + oxp);
  const Rec<R> ym = ld_rec(v, id + oym), yp = ld_rec(v, id + oyp);
  Rec<R> zm = cc, zp = cc;
  if (THREE_D) {
    zm = ld_rec(v, id + ozm);
    zp = ld_rec(v, id + ozp);
  }
  return sa_core<R, THREE_D>(p, cc, xm, xp, ym, yp, zm, zp, inv_wall_dist2<R>(p, x, y));
}

// --------------------------------------------------------------------------
// Wall functions (Eqs. 15-16, log law) and the FP64 u_tau inversion.
// Eq. 16 is evaluated on its continuous branch, atan2(b, y+ + a).
// --------------------------------------------------------------------------
struct WF {
  static constexpr double kappa = 0.41, cv1 = 7.1;
  static constexpr double Bb = 5.033908790505579, a1 = 8.148221580024245,
                          a2 = -6.9287093849022945, b1 = 7.4600876082527945,
                          b2 = 7.468145790401841, c1 = 2.5496773539754747,
                          c2 = 1.3301651588535228, c3 = 3.599459109332379,
                          c4 = 3.639753186868684494;
};

__host__ __device__ inline double wf_uplus(int law, double kap, double B, double yp) {
  if (law == 1) return log(yp) / kap + B;
  const double s1 = yp + WF::a1, s2 = yp + WF::a2;
  return WF::Bb + WF::c1 * log(s1 * s1 + WF::b1 * WF::b1) - WF::c2 * log(s2 * s2 + WF::b2 * WF::b2) -
         WF::c3 * atan2(WF::b1, s1) - WF::c4 * atan2(WF::b2, s2);
}

__host__ __device__ inline double wf_dudy(int law, double kap, double yp) {
  if (law == 1) return 1.0 / (kap * yp);
  const double ky = WF::kappa * yp, ky3 = ky * ky * ky, cv3 = WF::cv1 * WF::cv1 * WF::cv1;
  return (cv3 + ky3) / (cv3 + (1.0 + ky) * ky3);
}

// The same wall law and slope in FP32, for the wall-function values outside the
// Newton inversion (u_B of Section 3.1, the slope of Eq. 15 in Eq. 27, the four
// values of Eq. 29): a few ulp of FP32 (~1e-7 relative), where the FP64 forms
// would run on GB300's FP64 pipe at 1/64 of the FP32 rate.
// atan2(b, s) for b > 0 is pi/2 - atan(s / b) on the whole continuous branch
// (an absolute error of a few 1e-7 against terms of u+ ~ 10, where the
// two-argument form's quadrant logic costs more instructions).
__device__ __forceinline__ float wf_uplus_f(int law, float kap, float B, float yp) {
  if (law == 1) return logf(yp) / kap + B;
  const float s1 = yp + (float)WF::a1, s2 = yp + (float)WF::a2;
  const float b1 = (float)WF::b1, b2 = (float)WF::b2;
  const float hpi = 1.57079632679489662f;
  const float t1 = hpi - atanf(s1 * (float)(1.0 / WF::b1));
  const float t2 = hpi - atanf(s2 * (float)(1.0 / WF::b2));
  return (float)WF::Bb + (float)WF::c1 * logf(s1 * s1 + b1 * b1) -
         (float)WF::c2 * logf(s2 * s2 + b2 * b2) - (float)WF::c3 * t1 - (float)WF::c4 * t2;
}

__device__ __forceinline__ float wf_dudy_f(int law, float kap, float yp) {
  if (law == 1) return 1.0f / (kap * yp);
  const float ky = (float)WF::kappa * yp, ky3 = ky * ky * ky;
  const float cv3 = (float)(WF::cv1 * WF::cv1 * WF::cv1);
  return (cv3 + ky3) / (cv3 + (1.0f + ky) * ky3);
}

// wall law and slope in the compute type (FP32 forms above, FP64 in the FP64 mode)
template <class R> __device__ __forceinline__ R wf_uplus_r(const Params& p, R yp);
template <> __device__ __forceinline__ float wf_uplus_r<float>(const Params& p, float yp) {
  return wf_uplus_f(p.wall_law, (float)p.law_kappa, (float)p.law_B, yp);
}
template <> __device__ __forceinline__ double wf_uplus_r<double>(const Params& p, double yp) {
  return wf_uplus(p.wall_law, p.law_kappa, p.law_B, yp);
}
template <class R> __device__ __forceinline__ R wf_dudy_r(const Params& p, R yp);
template <> __device__ __forceinline__ float wf_dudy_r<float>(const Params& p, float yp) {
  return wf_dudy_f(p.wall_law, (float)p.law_kappa, yp);
}
template <> __device__ __forceinline__ double wf_dudy_r<double>(const Params& p, double yp) {
  return wf_dudy(p.wall_law, p.law_kappa, yp);
}

// Solve U = u u+(u y / nu) for u >= 0 (FP64).  Newton from the previous
// u_tau (or sqrt(U nu / y), the viscous-sublayer value) inside a sign-change
// bracket [lo, hi] that starts as [0, inf) and tightens with every residual;
// a step that would leave the bracket is replaced by bisection (or doubling
// while hi is still open).  Once a Newton step is below 1e-5 of u_tau the
// stepped value is returned: quadratic convergence leaves an error of order
// step^2 / u_tau (about 1e-10 relative, five orders below the FP32 parity
// bar); warm-started from the previous step's u_tau (which moves by far less
// than 1e-5 per step) this is a single FP64 evaluation of the wall law.  Returns false if the 100-iteration limit was
// reached (the last iterate is still returned).
__host__ __device__ inline bool solve_utau(int law, double kap, double B, double U, double y,
                                           double nu, double guess, double* out) {
  if (!(U > 0.0)) {
    *out = 0.0;
    return true;
  }
  double lo = 0.0, hi = 0.0;  // hi == 0: not bracketed from above yet
  double x = guess > 0.0 ? guess : sqrt(U * nu / y);
  for (int it = 0; it < 100; ++it) {
    const double yp = x * y / nu;
    const double up = wf_uplus(law, kap, B, yp);
    const double g = x * up - U;
    if (g == 0.0) {
      *out = x;
      return true;
    }
    if (g < 0.0) lo = x; else hi = x;
    const double dg = up + yp * wf_dudy(law, kap, yp);
    const double step = g / dg;
    double xn = x - step;
    if (fabs(step) <= 1e-5 * x && xn > 0.0) {
      // quadratic convergence: the error of xn is of order step^2 / x (about 1e-10 x)
      *out = xn;
      return true;
    }
    if (!(xn > lo) || (hi > 0.0 && !(xn < hi)) || !(dg > 0.0)) xn = hi > 0.0 ? 0.5 * (lo + hi) : 2.0 * x;
    x = xn;
  }
  *out = x;
  return false;
}

// The same root with the iterations shared between FP32 and FP64.  Newton runs
// in FP32 from the warm start (the FP32 wall law: logf, atan2f) until its step
// is below 1e-5 of the iterate, which FP32 resolves; one Newton step on the
// exact FP64 residual (Eq. 16 in FP64) then completes the inversion.  That
// step's slope is the FP32 one of the last iteration: it is needed only to
// ~1e-5 relative for a correction of ~1e-6 of u_tau, which leaves ~1e-11.  A
// developing flow, whose u_tau moves by more than 1e-5 per step, thereby costs
// one FP64 evaluation of the wall law per node and step instead of two or
// three with their slopes and divisions; on GB300 the FP64 logarithms and
// arctangents run at 1/64 of the FP32 rate.  Falls back to the FP64 iteration
// (solve_utau) if the FP32 one does not settle or the FP64 step is not small.
// inv_nu = 1 / nu.
__device__ inline bool solve_utau_mixed(int law, double kap, double B, double U, double y,
                                        double nu, double inv_nu, double guess, double* out) {
  if (!(U > 0.0)) {
    *out = 0.0;
    return true;
  }
  const double ynd = y * inv_nu;   // y / nu
  const float Uf = (float)U, yn = (float)ynd, kf = (float)kap, Bf = (float)B;
  float xf = guess > 0.0 ? (float)guess : sqrtf(Uf / yn);
  float dgf = 1.0f;
  bool settled = false;
  for (int it = 0; it < 8; ++it) {
    const float yp = xf * yn;
    const float up = wf_uplus_f(law, kf, Bf, yp);
    const float dg = up + yp * wf_dudy_f(law, kf, yp);
    const float step = (xf * up - Uf) / dg;
    const float xn = xf - step;
    if (!(dg > 0.0f) || !(xn > 0.0f)) break;
    xf = xn;
    dgf = dg;
    if (fabsf(step) <= 1e-5f * xf) {
      settled = true;
      break;
    }
  }
  const double x = settled ? (double)xf : guess;
  if (settled) {
    const double step = (x * wf_uplus(law, kap, B, x * ynd) - U) * (double)__fdividef(1.0f, dgf);
    const double xn = x - step;
    if (fabs(step) <= 1e-4 * x && xn > 0.0) {
      *out = xn;
      return true;
    }
  }
  return solve_utau(law, kap, B, U, y, nu, x, out);
}

// f_i^eq(rho, u) - E_i written in the small quantities drho = rho - 1 and
// du = u - U x (u = U x + du):
//   w [drho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u) + 3 c.du + 4.5 c.du (2 c_x U + c.du)
//      - 1.5 du.(2 U x + du)]
// (second-order Hermite equilibrium, Eq. 17).  uu15 = 1.5 u.u, du15 = 1.5 du.(2Ux + du).
// With cu = c.u, cU = c_x U, cdu = c.du this is w (drho A + D),
//   A = 1 + cu (3 + 4.5 cu) - uu15,  D = cdu (3 + 4.5 (cu + cU)) - du15.
template <int Q, class R>
__device__ __forceinline__ R heq_cdu(int i, R cdu, R drho, R U, R one_m_uu15, R du15) {
  using L = Lat<Q>;
  const R cU = L::c(i, 0) > 0 ? U : (L::c(i, 0) < 0 ? -U : (R)0);
  const R cu = cU + cdu;
  const R A = cu * ((R)3 + (R)4.5 * cu) + one_m_uu15;
  const R D = cdu * ((R)3 + (R)4.5 * (cu + cU)) - du15;
  return (R)L::w(i) * (drho * A + D);
}

template <int Q, class R>
__device__ __forceinline__ R cdot(int i, R vx, R vy, R vz) {
  using L = Lat<Q>;
  R t = 0;
  if (L::c(i, 0)) t += L::c(i, 0) > 0 ? vx : -vx;
  if (L::c(i, 1)) t += L::c(i, 1) > 0 ? vy : -vy;
  if (L::c(i, 2)) t += L::c(i, 2) > 0 ? vz : -vz;
  return t;
}

template <int Q, class R>
__device__ __forceinline__ R heq_dev(int i, R drho, R dux, R duy, R duz, R U, R uu15, R du15) {
  return heq_cdu<Q, R>(i, cdot<Q, R>(i, dux, duy, duz), drho, U, (R)1 - uu15, du15);
}

// --------------------------------------------------------------------------
// Post-stream populations with the face rules (Eq. 3 with Eq. 31, symmetry,
// free stream, zero-gradient outlet).  Returns the deviation g_i at
// (x, y, z) after streaming; `known` is false for Zou-He inlet unknowns and
// for HRFD wall unknowns, whose value is replaced later.
// --------------------------------------------------------------------------
template <int Q, int ST>
__device__ typename Compute<ST>::R pull_bc(const Params& p, int x, int y, int z, int i, bool* known) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  const T* LBM_RESTRICT f = (const T*)p.f_src;
  *known = true;
  const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
  int sx = x - cx;
  if (sx < 0 || sx >= p.nx) {
    if (p.px) {
      sx = sx < 0 ? sx + p.nx : sx - p.nx;
    } else if (sx < 0) {
      *known = false;  // inlet unknown: Zou-He
      return (R)0;
    } else {
      // zero-gradient outlet: the post-stream value of the neighbouring column
      x -= 1;
      sx = x - cx;
    }
  }
  int sz = z - cz;
  sz = sz < 0 ? sz + p.nz : (sz >= p.nz ? sz - p.nz : sz);
  int sy = y - cy;
  if (sy >= 0 && sy < p.ny) return (R)C::ld(f + i * p.ncell + cidx(p, sx, sy, sz));
  if (p.py) {
    sy = sy < 0 ? sy + p.ny : sy - p.ny;
    return (R)C::ld(f + i * p.ncell + cidx(p, sx, sy, sz));
  }
  const int fi = sy < 0 ? 0 : 1;   // 0 = ymin, 1 = ymax
  const int kind = p.kind[YMIN + fi];
  if (kind == BC_FREESTREAM) {
    // incoming populations at f^eq(1, u_inf)
    const R U = psel<R>(p.Ush, p.Ush_f);
    const R ux = psel<R>(p.u_face[YMIN + fi][0], p.u_face_f[YMIN + fi][0]), uy = psel<R>(p.u_face[YMIN + fi][1], p.u_face_f[YMIN + fi][1]),
            uz = psel<R>(p.u_face[YMIN + fi][2], p.u_face_f[YMIN + fi][2]);
    const R dux = ux - U;
    const R uu15 = (R)1.5 * (ux * ux + uy * uy + uz * uz);
    const R du15 = (R)1.5 * (dux * ((R)2 * U + dux) + uy * uy + uz * uz);
    return heq_dev<Q, R>(i, (R)0, dux, uy, uz, U, uu15, du15);
  }
  const bool wall_col = p.wall[fi] && x >= p.xw0[fi];
  if (wall_col && kind == BC_WALL_BB) {
    // Eq. 31: f_i(B, t+1) = f*_{opp i}(B, t) + 2 w rho_w c_i.u_w / c_s^2; in deviations
    // E_{opp i} - E_i = -6 w c_x U adds to the reflected value
    const int node = z * (p.nx - p.xw0[fi]) + (x - p.xw0[fi]);
    const R* uw = (const R*)p.uw[fi] + 3 * node;
    const R cu = (R)cx * uw[0] + (R)cy * uw[1] + (R)cz * uw[2];
    const R rw = ((const R*)p.rhow[fi])[node];
    const long long idB = cidx(p, x, y, z);
    const R K = (R)6 * (R)L::w(i) * (rw * cu - (R)cx * psel<R>(p.Ush, p.Ush_f));
    const R hoB = (R)C::ld(f + opp(i) * p.ncell + idB);
    if (p.interp[fi] == 0) return hoB + K;
    // Eqs. 36-37: the F node of the link is B + c_i (one link into the fluid);
    // z wraps, x wraps when periodic and otherwise stays in the boundary column
    int xf = x + cx;
    if (xf < 0 || xf >= p.nx) xf = p.px ? (xf < 0 ? xf + p.nx : xf - p.nx) : x;
    int zf = z + cz;
    zf = zf < 0 ? zf + p.nz : (zf >= p.nz ? zf - p.nz : zf);
    const R hoF = (R)C::ld(f + opp(i) * p.ncell + cidx(p, xf, y + cy, zf));
    const R hiB = (R)C::ld(f + i * p.ncell + idB);
    const double* a = p.ibb[fi];
    const float* af = p.ibb_f[fi];
    return psel<R>(a[0], af[0]) * hoB + psel<R>(a[1], af[1]) * hoF + psel<R>(a[2], af[2]) * hiB +
           psel<R>(a[3], af[3]) * K;
  }
  if (wall_col) {  // regularized walls: every population of B is rebuilt later
    *known = false;
    return (R)0;
  }
  // symmetry: specular reflection from the same row
  return (R)C::ld(f + L::my(i) * p.ncell + cidx(p, sx, y, sz));
}

// --------------------------------------------------------------------------
// Local collision in deviation form (g below stands for h = f - E).
//   rho = 1 + sum g, rho u = U x + sum g c + F/2 (Eqs. 4-5)
//   g^eq = f^eq(rho, u) - E (heq_dev)
//   BGK: g* = g - omega (g - g^eq) + (1 - omega/2) F_i
//   regularized: g* = g^eq + (1 - omega) P(g - g^eq) + (1 - omega/2) F_i with
//   P the Hermite projection up to second order.
//   F_i = w [3 (c - u).F + 9 (c.u)(c.F)] (Guo).
// The relaxation is written with delta = 2 - omega = 4 eps / (1 + 2 eps),
// eps = tau - 1/2 = nu_eff / c_s^2 (Eq. 8): at the paper's resolutions
// eps ~ 1e-5, and forming omega itself in FP32 would keep only ~0.2 % of
// the viscous part.  With delta the "-1" of (1 - omega) is applied exactly:
//   BGK: g* = 2 g^eq - g + delta (g - g^eq); regularized: g^eq - P + delta P;
//   force prefactor 1 - omega/2 = delta / 2.
// --------------------------------------------------------------------------
template <class R> __device__ __forceinline__ R relax_delta(R eps) {
  return fdiv((R)4 * eps, (R)1 + (R)2 * eps);
}

// SCALE: g holds SCALE x h on entry and on return (the raw storage scale of the
// interior path); the moments are taken back to h once, and the scale enters
// the equilibrium weights and the force prefactor as constants.
// Equilibrium of an opposite pair (i, opp i) from per-weight-class coefficients.
// With s = c_i.u = cU + d (cU = c_x U, d = c_i.du) the deviation equilibrium
//   h^eq_{i / opp} = w [drho (1 + 4.5 s^2 - 1.5 u.u) + 4.5 d (s + cU) - du15] +/- 3 w (drho s + d)
// expands into a polynomial in d whose coefficients depend on the weight only:
//   even part  ev = b2 d^2 + cx c1 d + c0,   odd part  od = d1 d + cx d0,
//   b2 = 4.5 w rho, c1 = 9 w rho U, c0 = w (drho (1 - 1.5 u.u + 4.5 cx^2 U^2) - du15),
//   d1 = 3 w rho, d0 = 3 w drho U
// (two FFMA for ev and one for od, where the expanded form takes seven).
template <class R> struct EqCoef {
  R b2, c1, c0x, c00, d1, d0;   // c0x: c0 for c_x != 0; c00: for c_x = 0
};

template <class R>
__device__ __forceinline__ EqCoef<R> eq_coef(R wS, R rho, R drho, R U, R one_m_uu15, R du15) {
  EqCoef<R> k;
  k.b2 = (R)4.5 * wS * rho;
  k.c1 = (R)9 * wS * rho * U;
  k.c00 = wS * (drho * one_m_uu15 - du15);
  k.c0x = k.c00 + (R)4.5 * wS * drho * U * U;
  k.d1 = (R)3 * wS * rho;
  k.d0 = (R)3 * wS * drho * U;
  return k;
}

template <int Q, class R>
__device__ __forceinline__ void eq_pair(const EqCoef<R>& k, int cx, R d, R* ev, R* od) {
  if (cx == 0) {
    *ev = fmaf_r(d * d, k.b2, k.c00);
    *od = k.d1 * d;
  } else {
    const R c1 = cx > 0 ? k.c1 : -k.c1, d0 = cx > 0 ? k.d0 : -k.d0;
    *ev = fmaf_r(d, fmaf_r(d, k.b2, c1), k.c0x);
    *od = fmaf_r(k.d1, d, d0);
  }
}

// COLL: the collision operator fixed at compile time (COLL_BGK, COLL_REG), or
// COLL_ANY to take p.collision at run time; a kernel compiled for one operator
// needs only that operator's registers.
template <int Q, class R, int SCALE = 1, int COLL = COLL_ANY>
__device__ __forceinline__ void collide(const Params& p, R (&g)[Q], R delta, R* u_out) {
  using L = Lat<Q>;
  // moments over opposite pairs (i, i+1 = opp i): the pair's sum enters rho,
  // its difference rho u
  R drho = g[0], jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const R sp = g[i] + g[i + 1], dp = g[i] - g[i + 1];
    drho += sp;
    if (L::c(i, 0)) jx += L::c(i, 0) > 0 ? dp : -dp;
    if (L::c(i, 1)) jy += L::c(i, 1) > 0 ? dp : -dp;
    if (L::c(i, 2)) jz += L::c(i, 2) > 0 ? dp : -dp;
  }
  if (SCALE != 1) {
    const R is = (R)(1.0 / SCALE);
    drho *= is;
    jx *= is;
    jy *= is;
    jz *= is;
  }
  // sum h c = rho u - U x - F/2: momentum relative to the reference velocity
  const R Fx = psel<R>(p.F[0], p.F_f[0]), Fy = psel<R>(p.F[1], p.F_f[1]), Fz = psel<R>(p.F[2], p.F_f[2]);
  jx += (R)0.5 * Fx;
  jy += (R)0.5 * Fy;
  jz += (R)0.5 * Fz;
  const R U = psel<R>(p.Ush, p.Ush_f);
  const R rho = (R)1 + drho;
  const R inv = fdiv((R)1, rho);
  const R dux = (jx - drho * U) * inv, uy = jy * inv, uz = jz * inv;
  const R ux = U + dux;
  u_out[0] = ux;
  u_out[1] = uy;
  u_out[2] = uz;
  const R one_m_uu15 = (R)1 - (R)1.5 * (ux * ux + uy * uy + uz * uz);
  const R du15 = (R)1.5 * (dux * ((R)2 * U + dux) + uy * uy + uz * uz);
  // equilibrium coefficients of the two weight classes of the moving populations
  // (index 1: axis directions, index 2: diagonals), storage scale folded in
  const EqCoef<R> k1 = eq_coef<R>((R)(L::w(1) * SCALE), rho, drho, U, one_m_uu15, du15);
  const EqCoef<R> k2 = eq_coef<R>((R)(L::w(Q == 19 ? 7 : 5) * SCALE), rho, drho, U, one_m_uu15, du15);
  // (1 - omega/2) w [3 (c - u).F + 9 (c.u)(c.F)] = (delta/2) [A_i (1 + 3 c.u) - 3 w u.F]
  const R fpre = ((R)0.5 * (R)SCALE) * delta;
  const R uF3 = (R)3 * (ux * Fx + uy * Fy + uz * Fz);
  const R fw1 = fpre * (R)L::w(1) * uF3, fw2 = fpre * (R)L::w(Q == 19 ? 7 : 5) * uF3;
  if (COLL == COLL_BGK || (COLL == COLL_ANY && p.collision == 0)) {
    // BGK over opposite pairs: h* = (2 h^eq - h) + delta (h - h^eq) + forcing,
    // the force term of the pair split into its even part fe and odd part fo,
    //   F_{i / opp} = fe +/- fo,  fe = fpre (3 s A_i - 3 w u.F),  fo = fpre A_i
    //   (A_i = 3 w_i c_i.F)
    {
      const R wgt0 = (R)L::w(0);
      const R geq = (R)(L::w(0) * SCALE) * (drho * one_m_uu15 - du15);
      R gi = ((R)2 * geq - g[0]) + delta * (g[0] - geq);
      if (p.has_force) gi -= fpre * wgt0 * uF3;
      g[0] = gi;
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const bool diag = L::w(i) < L::w(1);
      const EqCoef<R>& k = diag ? k2 : k1;
      const int cx = L::c(i, 0);
      const R cdu = cdot<Q, R>(i, dux, uy, uz);
      R gp, od;
      eq_pair<Q, R>(k, cx, cdu, &gp, &od);
      const R gm = gp - od;                                    // h^eq_opp
      gp += od;                                                // h^eq_i
      R np_ = ((R)2 * gp - g[i]) + delta * (g[i] - gp);
      R nm_ = ((R)2 * gm - g[i + 1]) + delta * (g[i + 1] - gm);
      if (p.has_force) {
        const R cU = cx > 0 ? U : (cx < 0 ? -U : (R)0);
        const R su = cU + cdu;                                 // c_i . u
        const R fo = fpre * psel<R>(p.guoA[i], p.guoA_f[i]);
        const R fe = fmaf_r(fo, (R)3 * su, -(diag ? fw2 : fw1));
        np_ += fe + fo;
        nm_ += fe - fo;
      }
      g[i] = np_;
      g[i + 1] = nm_;
    }
    return;
  }
  // regularized, over opposite pairs as above.  With n = h - h^eq, a pair enters
  // the non-equilibrium moments only through s = n_i + n_opp (second order,
  // sum c_a c_b n) and d = n_i - n_opp (first order, sum c n); the rest
  // population enters neither.  The rebuilt populations are
  //   h*_{i / opp} = h^eq + (delta - 1) P + forcing,  P = w (3 c.a + 4.5 Q:Pi),
  // whose even part is 4.5 w Q_i:Pi and odd part 3 w c_i.a.
  const R dm1 = delta - (R)1;
  R ax = 0, ay = 0, az = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const EqCoef<R>& k = L::w(i) < L::w(1) ? k2 : k1;
    const R cdu = cdot<Q, R>(i, dux, uy, uz);
    R ev, od;
    eq_pair<Q, R>(k, L::c(i, 0), cdu, &ev, &od);
    const R sp = (g[i] + g[i + 1]) - (R)2 * ev;
    const R dp = (g[i] - g[i + 1]) - (R)2 * od;
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    if (cx) ax += cx > 0 ? dp : -dp;
    if (cy) ay += cy > 0 ? dp : -dp;
    if (cz) az += cz > 0 ? dp : -dp;
    if (cx) pxx += sp;
    if (cy) pyy += sp;
    if (cz) pzz += sp;
    if (cx && cy) pxy += cx * cy > 0 ? sp : -sp;
    if (cx && cz) pxz += cx * cz > 0 ? sp : -sp;
    if (cy && cz) pyz += cy * cz > 0 ? sp : -sp;
    g[i] = ev;       // the equilibrium parts are all the rebuild needs
    g[i + 1] = od;
  }
  const R tr = (pxx + pyy + pzz) * (R)(1.0 / 3.0);
  {
    const R wgt0 = (R)L::w(0);
    R gi = (wgt0 * (R)SCALE) * (drho * one_m_uu15 - du15) + dm1 * (wgt0 * (R)4.5 * -tr);
    if (p.has_force) gi -= fpre * wgt0 * uF3;
    g[0] = gi;
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const R w = (R)L::w(i);
    const bool diag = L::w(i) < L::w(1);
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    R qp = -tr, ca = 0;
    if (cx) { qp += pxx; ca += cx > 0 ? ax : -ax; }
    if (cy) { qp += pyy; ca += cy > 0 ? ay : -ay; }
    if (cz) { qp += pzz; ca += cz > 0 ? az : -az; }
    if (cx && cy) qp += (R)2 * (cx * cy > 0 ? pxy : -pxy);
    if (cx && cz) qp += (R)2 * (cx * cz > 0 ? pxz : -pxz);
    if (cy && cz) qp += (R)2 * (cy * cz > 0 ? pyz : -pyz);
    R E = g[i] + dm1 * (w * (R)4.5 * qp);
    R O = g[i + 1] + dm1 * (w * (R)3 * ca);
    if (p.has_force) {
      const R cU = cx > 0 ? U : (cx < 0 ? -U : (R)0);
      const R su = cU + cdot<Q, R>(i, dux, uy, uz);
      const R fo = fpre * psel<R>(p.guoA[i], p.guoA_f[i]);
      E += fmaf_r(fo, (R)3 * su, -(diag ? fw2 : fw1));
      O += fo;
    }
    g[i] = E + O;
    g[i + 1] = E - O;
  }
}

}  // namespace lbm
