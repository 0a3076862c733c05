// lbm_kernels.cuh -- the kernels of one LBM-RANS step and their helpers.
//
// Per step (buffers src -> dst):
//   k_wall  : wall pre-pass over the compacted wall-node list of each y face
//             (slip-velocity bounce-back: Newton for u_tau, Eq. 35 slip
//             velocity and rho_w; HRFD: rho_F, u_F after streaming (Eqs.
//             20-22), Newton, u_B, rho_B (Eq. 23), the Eq. 27-28 gradient and
//             the Eq. 19/26 populations), Dirichlet nu_tilde_B = nu kappa y_B+.
//   k_bulk  : every cell: SA update (Eq. 11), pull streaming (Eq. 3) with the
//             face rules, Zou-He inlet, HRFD populations at wall nodes,
//             moments (Eqs. 4-5), omega from nu + nu_t (Eq. 8), collision.
#pragma once
#include "lbm_device.cuh"
#include "lbm_tma.cuh"

namespace lbm {

// ----------------------------------------------------------------------------
// Cells with no non-periodic face within one cell: the six neighbour offsets
// (periodic wrap folded in) replace all face logic; 32-bit indexing (the
// lattice is checked at creation to satisfy Q * pitch * ny * nz < 2^31).
// ----------------------------------------------------------------------------
struct NbOff {
  int id, nc, oxm, oxp, oym, oyp, ozm, ozp;
};

// Cell index and the offsets to the neighbours at x-1, x+1, y-1, y+1, z-1, z+1
// (periodic wrap folded in).
__device__ __forceinline__ NbOff nb_offsets(const Params& p, int x, int y, int z) {
  NbOff o;
  const int pitch = p.pitch;
  const int plane = pitch * p.ny;
  o.nc = (int)p.ncell;
  o.id = (z * p.ny + y) * pitch + x;
  o.oxm = x == 0 ? p.nx - 1 : -1;
  o.oxp = x == p.nx - 1 ? -(p.nx - 1) : 1;
  o.oym = y == 0 ? (p.ny - 1) * pitch : -pitch;
  o.oyp = y == p.ny - 1 ? -(p.ny - 1) * pitch : pitch;
  o.ozm = z == 0 ? (p.nz - 1) * plane : -plane;
  o.ozp = z == p.nz - 1 ? -(p.nz - 1) * plane : plane;
  return o;
}

// Post-stream deviation g_i (storage scale removed) at the cell of o, for a
// source inside the lattice or across a periodic face: the neighbour offsets
// stand in for the face logic of pull_bc.
template <int Q, int ST>
__device__ __forceinline__ typename Compute<ST>::R pull_nb(const Params& p, const NbOff& o, int i) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using T = typename C::T;
  const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
  const int off = (cx > 0 ? o.oxm : (cx < 0 ? o.oxp : 0)) + (cy > 0 ? o.oym : (cy < 0 ? o.oyp : 0)) +
                  (cz > 0 ? o.ozm : (cz < 0 ? o.ozp : 0));
  return (typename Compute<ST>::R)C::ld((const T*)p.f_src + (i * o.nc + o.id + off));
}

// Everything after streaming for a cell with in-lattice (or periodic)
// neighbours: SA update, relaxation rate, collision, stores.  g holds the
// pulled populations in the raw storage scale (Codec::ld_raw).
template <int Q, int ST>
__device__ __forceinline__ void interior_finish(const Params& p, const NbOff& o,
                                                typename Compute<ST>::R (&g)[Q], int x, int y) {
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  T* LBM_RESTRICT fd = (T*)p.f_dst;
  const R* LBM_RESTRICT vs = (const R*)p.v_src;
  R* LBM_RESTRICT vd = (R*)p.v_dst;
  // SA working variable of the new step (Eq. 11)
  R ntn;
  if (p.turbulent)
    ntn = sa_update_interior<R, (Q == 19)>(p, vs, o.id, o.oxm, o.oxp, o.oym, o.oyp, o.ozm, o.ozp,
                                            x, y);
  else
    ntn = vs[4 * o.id + 3];
  const R nu = psel<R>(p.nu, p.nu_f);
  const R nut = p.turbulent ? sa_nut<R>(ntn, psel<R>(p.inv_nu, p.inv_nu_f)) : (R)0;
  const R delta = relax_delta<R>((R)3 * (nu + nut));   // 2 - omega (Eq. 8)
  // moments and collision
  R u[3];
  collide<Q, R, C::kScale>(p, g, delta, u);   // g in raw storage scale
  // store
#pragma unroll
  for (int i = 0; i < Q; ++i) C::st_raw(fd + (i * o.nc + o.id), g[i]);
  st_rec(vd, o.id, u[0], u[1], u[2], ntn);
}

// Pull streaming (Eq. 3) of a cell with in-lattice or periodic neighbours:
// g_i = f*_i(x - c_i) in the raw storage scale.
template <int Q, int ST>
__device__ __forceinline__ void pull_interior(const Params& p, const NbOff& o,
                                              typename Compute<ST>::R (&g)[Q]) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  const T* LBM_RESTRICT fs = (const T*)p.f_src;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const int off = (cx > 0 ? o.oxm : (cx < 0 ? o.oxp : 0)) + (cy > 0 ? o.oym : (cy < 0 ? o.oyp : 0)) +
                    (cz > 0 ? o.ozm : (cz < 0 ? o.ozp : 0));
    g[i] = (R)C::ld_raw(fs + (i * o.nc + o.id + off));
  }
}

template <int Q, int ST>
__device__ __forceinline__ void bulk_interior(const Params& p, int x, int y, int z) {
  using R = typename Compute<ST>::R;
  const NbOff o = nb_offsets(p, x, y, z);
  // the pulled loads are issued first, in flight while the SA stencil is evaluated
  R g[Q];
  pull_interior<Q, ST>(p, o, g);
  interior_finish<Q, ST>(p, o, g, x, y);
}

// Two neighbouring cells A = (x0, y, z) and B = (x0 + 1, y, z) of one row, x0
// even, both with in-lattice or periodic neighbours, in one thread: the
// populations of the directions with c_x = 0 are read for both cells with one
// paired access, every post-collision pair is written with one, the SA stencil
// reads 12 records for both cells instead of 14, the index arithmetic is
// shared, and the FP32 arithmetic runs on packed lanes (f2).  Each cell follows
// the steps of bulk_interior; the packed lanes round products and sums
// separately where the scalar code may fuse them.
template <int Q, int ST, int COLL>
__device__ __forceinline__ void bulk_interior2(const Params& p, int x0, int y, int z) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  // FP32 arithmetic of the pair on packed lanes (f2); FP64 as two scalars
  using V = typename std::conditional<std::is_same<R, float>::value, f2, R>::type;
  constexpr bool kPacked = std::is_same<V, f2>::value;
  // the SA stencil on packed lanes too for 16-bit storage (measured 0.1148 against
  // 0.1168 ms per step, FP16 channel 256x128x128); FP32 storage keeps it scalar,
  // whose registers fit the budget (packed: 0.1334 against 0.1252 ms, spilling)
  constexpr bool kPackedSA = kPacked && ST != ST_FP32;
  using T = typename C::T;
  const T* LBM_RESTRICT fs = (const T*)p.f_src;
  T* LBM_RESTRICT fd = (T*)p.f_dst;
  const R* LBM_RESTRICT vs = (const R*)p.v_src;
  R* LBM_RESTRICT vd = (R*)p.v_dst;
  const NbOff o = nb_offsets(p, x0, y, z);     // cell A; B has x - 1 = A
  const int oxpB = x0 + 1 == p.nx - 1 ? -(p.nx - 1) : 1;
  // pull streaming (Eq. 3) for both cells, issued first; the pairs are kept as
  // loaded (16-bit storage: one 32-bit register per direction) through the SA
  // stencil and converted just before the collision
  typename C::P2 hp[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const int yz = (cy > 0 ? o.oym : (cy < 0 ? o.oyp : 0)) + (cz > 0 ? o.ozm : (cz < 0 ? o.ozp : 0));
    const T* pa = fs + (i * o.nc + o.id + yz);   // element x0 of the source row
    if (cx == 0) hp[i] = C::ld_pair(pa);
    else if (cx > 0) hp[i] = C::pair(pa + o.oxm, pa);      // sources x0 - 1 (wrapped) and x0
    else hp[i] = C::pair(pa + 1, pa + 1 + oxpB);           // sources x0 + 1 and x0 + 2 (wrapped)
  }
  // SA working variable of the new step (Eq. 11): the records of both stencils
  R ntA, ntB;
  const int idB = o.id + 1;
  if (p.turbulent) {
    const Rec<R> cA = ld_rec(vs, o.id), cB = ld_rec(vs, idB);
    const Rec<R> xmA = ld_rec(vs, o.id + o.oxm), xpB = ld_rec(vs, idB + oxpB);
    const Rec<R> ymA = ld_rec(vs, o.id + o.oym), ymB = ld_rec(vs, idB + o.oym);
    const Rec<R> ypA = ld_rec(vs, o.id + o.oyp), ypB = ld_rec(vs, idB + o.oyp);
    Rec<R> zmA = cA, zpA = cA, zmB = cB, zpB = cB;
    if (Q == 19) {
      zmA = ld_rec(vs, o.id + o.ozm);
      zpA = ld_rec(vs, o.id + o.ozp);
      zmB = ld_rec(vs, idB + o.ozm);
      zpB = ld_rec(vs, idB + o.ozp);
    }
    const R* itab = (const R*)p.invd2 + y * p.pitch + x0;
    if constexpr (kPackedSA) {
      // lanes (A, B) of each stencil position: x - 1 of B is A, x + 1 of A is B
      const auto pk = [](const Rec<float>& a, const Rec<float>& b) {
        return Rec<f2>{f2(a.x, b.x), f2(a.y, b.y), f2(a.z, b.z), f2(a.n, b.n)};
      };
      const float2 id2 = LBM_LDG(reinterpret_cast<const float2*>(itab));
      const f2 nt = sa_core<f2, (Q == 19)>(p, pk(cA, cB), pk(xmA, cA), pk(cB, xpB), pk(ymA, ymB),
                                           pk(ypA, ypB), pk(zmA, zmB), pk(zpA, zpB), f2(id2));
      ntA = nt.v.x;
      ntB = nt.v.y;
    } else {
      ntA = sa_core<R, (Q == 19)>(p, cA, xmA, cB, ymA, ypA, zmA, zpA, LBM_LDG(itab));
      ntB = sa_core<R, (Q == 19)>(p, cB, cA, xpB, ymB, ypB, zmB, zpB, LBM_LDG(itab + 1));
    }
  } else {
    ntA = vs[4 * o.id + 3];
    ntB = vs[4 * idB + 3];
  }
  if constexpr (kPacked) {
    f2 g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = f2(C::both(hp[i]));
    const f2 nt(ntA, ntB), nu = psel<f2>(p.nu, p.nu_f), inu = psel<f2>(p.inv_nu, p.inv_nu_f);
    const f2 nut = p.turbulent ? sa_nut<f2>(nt, inu) : f2(0.0f);
    f2 u[3];
    collide<Q, f2, C::kScale, COLL>(p, g, relax_delta<f2>(f2(3.0f) * (nu + nut)), u);   // 2 - omega (Eq. 8)
#pragma unroll
    for (int i = 0; i < Q; ++i) C::st2_raw(fd + (i * o.nc + o.id), g[i].v.x, g[i].v.y);
    st_rec(vd, o.id, u[0].v.x, u[1].v.x, u[2].v.x, ntA);
    st_rec(vd, idB, u[0].v.y, u[1].v.y, u[2].v.y, ntB);
  } else {
    const R nu = psel<R>(p.nu, p.nu_f), inu = psel<R>(p.inv_nu, p.inv_nu_f);
    const R nutA = p.turbulent ? sa_nut<R>(ntA, inu) : (R)0;
    const R nutB = p.turbulent ? sa_nut<R>(ntB, inu) : (R)0;
    R gA[Q], gB[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      gA[i] = C::lo(hp[i]);
      gB[i] = C::hi(hp[i]);
    }
    R uA[3], uB[3];
    collide<Q, R, C::kScale, COLL>(p, gA, relax_delta<R>((R)3 * (nu + nutA)), uA);   // 2 - omega (Eq. 8)
    collide<Q, R, C::kScale, COLL>(p, gB, relax_delta<R>((R)3 * (nu + nutB)), uB);
#pragma unroll
    for (int i = 0; i < Q; ++i) C::st2_raw(fd + (i * o.nc + o.id), gA[i], gB[i]);
    st_rec(vd, o.id, uA[0], uA[1], uA[2], ntA);
    st_rec(vd, idB, uB[0], uB[1], uB[2], ntB);
  }
}

// ----------------------------------------------------------------------------
// Bulk: one thread per cell, x fastest within a warp.  Cells next to a face
// take the general path with the face rules.
// ----------------------------------------------------------------------------
// GENERAL = false: the launch holds only cells without a non-periodic face
// within one cell (checked by the host), so the face logic is not compiled in.
// Minimum resident blocks per SM requested from the compiler for k_bulk
// (sets its register budget; 0 leaves the choice to the compiler).  A budget
// of 64 registers (1024 threads per SM) measured fastest on GB300 for the
// D3Q19 FP32 channel (0.159 ms per step against 0.172 ms with the
// compiler's 80), and small blocks faster than large ones: 64 / 128 / 256 /
// 512 threads gave 0.135 / 0.137 / 0.143 / 0.153 ms per step (the wall pass
// and the wall rows interleave better with the inner rows' smaller blocks).
#ifndef LBM_BULK_MINB
#define LBM_BULK_MINB 16
#endif
#if LBM_BULK_MINB > 0
#define LBM_BULK_BOUNDS __launch_bounds__(LBM_BULK_THREADS, LBM_BULK_MINB)
#else
#define LBM_BULK_BOUNDS __launch_bounds__(LBM_BULK_THREADS)
#endif

// A bounce-back wall node on a lattice with periodic x: the sources of the
// directions leaving the wall are replaced by the face's rule (Eq. 31, or
// Eqs. 36-37 through the affine weights of Params::ibb), every other source is
// in the lattice; nu_tilde is the Dirichlet value the wall pass stored.
template <int Q, int ST>
__device__ __forceinline__ void bulk_wall_bb(const Params& p, int fi, int x, int y, int z) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  const T* LBM_RESTRICT fs = (const T*)p.f_src;
  T* LBM_RESTRICT fd = (T*)p.f_dst;
  R* LBM_RESTRICT vd = (R*)p.v_dst;
  const NbOff o = nb_offsets(p, x, y, z);
  const int node = z * (p.nx - p.xw0[fi]) + (x - p.xw0[fi]);
  const R* uw = (const R*)p.uw[fi] + 3 * node;
  const R rw = ((const R*)p.rhow[fi])[node];
  const R rux = rw * uw[0], ruy = rw * uw[1], ruz = rw * uw[2];
  const R U = psel<R>(p.Ush, p.Ush_f);
  const bool interp = p.interp[fi] != 0;
  const R a0 = psel<R>(p.ibb[fi][0], p.ibb_f[fi][0]), aF = psel<R>(p.ibb[fi][1], p.ibb_f[fi][1]),
          ai = psel<R>(p.ibb[fi][2], p.ibb_f[fi][2]), aK = psel<R>(p.ibb[fi][3], p.ibb_f[fi][3]);
  R g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    const bool from_wall = fi == 0 ? cy > 0 : cy < 0;
    if (from_wall) {
      // Eq. 31 in deviations: h*_{opp i}(B) + K, K = 6 w (rho_w c_i.u_w - c_x U)
      const R cu = (R)cx * rux + (R)cy * ruy + (R)cz * ruz;
      const R K = (R)6 * (R)L::w(i) * (cu - (R)cx * U);
      const R hoB = (R)C::ld(fs + (opp(i) * o.nc + o.id));
      if (interp) {
        // Eqs. 36-37: h*_opp at F = B + c_i (one link into the fluid) and h*_i(B)
        const int offF = (cx > 0 ? o.oxp : (cx < 0 ? o.oxm : 0)) + (cy > 0 ? o.oyp : o.oym) +
                         (cz > 0 ? o.ozp : (cz < 0 ? o.ozm : 0));
        const R hoF = (R)C::ld(fs + (opp(i) * o.nc + o.id + offF));
        const R hiB = (R)C::ld(fs + (i * o.nc + o.id));
        g[i] = a0 * hoB + aF * hoF + ai * hiB + aK * K;
      } else {
        g[i] = hoB + K;
      }
    } else {
      const int off = (cx > 0 ? o.oxm : (cx < 0 ? o.oxp : 0)) + (cy > 0 ? o.oym : (cy < 0 ? o.oyp : 0)) +
                      (cz > 0 ? o.ozm : (cz < 0 ? o.ozp : 0));
      g[i] = (R)C::ld(fs + (i * o.nc + o.id + off));
    }
  }
  // the Dirichlet nu_tilde_B the wall pass wrote into this step's record
  const R ntB = vd[4 * o.id + 3];
  const R nu = psel<R>(p.nu, p.nu_f);
  const R nut = p.turbulent ? sa_nut<R>(ntB, psel<R>(p.inv_nu, p.inv_nu_f)) : (R)0;
  const R delta = relax_delta<R>((R)3 * (nu + nut));
  R u[3];
  collide<Q, R>(p, g, delta, u);
#pragma unroll
  for (int i = 0; i < Q; ++i) C::st(fd + (i * o.nc + o.id), g[i]);
  st_rec(vd, o.id, u[0], u[1], u[2], ntB);
}

// One cell of the bulk update (every cell of the lattice takes this path).
template <int Q, int ST, bool GENERAL>
__device__ __forceinline__ void bulk_cell(const Params& p, int x, int y, int z) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  if (!GENERAL || ((p.px || (x >= 1 && x <= p.nx - 2)) && (p.py || (y >= 1 && y <= p.ny - 2)))) {
    bulk_interior<Q, ST>(p, x, y, z);
    return;
  }
  if (p.px && p.turbulent && p.ny >= 3) {
    // slip bounce-back rows (half-way or interpolated)
    const int fw = (y == 0 && p.wall[0] == BC_WALL_BB && x >= p.xw0[0]) ? 0
                 : ((y == p.ny - 1 && p.wall[1] == BC_WALL_BB && x >= p.xw0[1]) ? 1 : -1);
    if (fw >= 0) {
      bulk_wall_bb<Q, ST>(p, fw, x, y, z);
      return;
    }
  }
  const long long id = cidx(p, x, y, z);
  T* LBM_RESTRICT fd = (T*)p.f_dst;
  const R* LBM_RESTRICT vs = (const R*)p.v_src;
  R* LBM_RESTRICT vd = (R*)p.v_dst;

  int wf = -1;
  if (y == 0 && p.wall[0] && x >= p.xw0[0]) wf = 0;
  else if (y == p.ny - 1 && p.wall[1] && x >= p.xw0[1]) wf = 1;
  if (wf >= 0 && p.wall[wf] != BC_WALL_BB) return;   // regularized wall node: done by the wall pass
  const bool inlet = (x == 0 && p.kind[XMIN] == BC_INLET);

  // 1. SA working variable of the new step (Dirichlet at wall nodes and inlet)
  R ntn;
  if (p.turbulent) {
    if (wf >= 0) {
      ntn = vd[4 * id + 3];   // Dirichlet value written by the wall pass
    } else {
      ntn = inlet ? psel<R>(p.nt_face[XMIN], p.nt_face_f[XMIN]) : sa_update<R, (Q == 19)>(p, vs, x, y, z);
    }
  } else {
    ntn = vs[4 * id + 3];
  }
  const R nu = psel<R>(p.nu, p.nu_f);
  const R nut = p.turbulent ? sa_nut<R>(ntn, psel<R>(p.inv_nu, p.inv_nu_f)) : (R)0;
  const R delta = relax_delta<R>((R)3 * (nu + nut));   // 2 - omega (Eq. 8)

  // 2. post-stream populations (regularized wall nodes are rebuilt by the wall pass)
  R g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    bool known;
    g[i] = pull_bc<Q, ST>(p, x, y, z, i, &known);
  }
  if (inlet) {
    // Zou-He velocity inlet: unknowns c_x > 0 from the non-equilibrium
    // bounce-back of the normal direction plus transverse corrections.
    const R ux = psel<R>(p.u_face[XMIN][0], p.u_face_f[XMIN][0]), uy = psel<R>(p.u_face[XMIN][1], p.u_face_f[XMIN][1]), uz = psel<R>(p.u_face[XMIN][2], p.u_face_f[XMIN][2]);
    R s0 = 0, sm = 0, ky = 0, kz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::c(i, 0) == 0) {
        s0 += g[i];
        ky += (R)L::c(i, 1) * g[i];
        kz += (R)L::c(i, 2) * g[i];
      } else if (L::c(i, 0) < 0) {
        sm += g[i];
      }
    }
    // in deviations from E = f^eq(1, U x): sum_{cx=0} E + 2 sum_{cx<0} E = 1 - U and
    // E_{opp i} - E_i = -6 w c_x U
    const R U = psel<R>(p.Ush, p.Ush_f);
    const R rho = fdiv(((R)1 - U) + s0 + (R)2 * sm, (R)1 - ux);
    const R Ny = (R)0.5 * ky - rho * uy * (R)(1.0 / 3.0);
    const R Nz = (R)0.5 * kz - rho * uz * (R)(1.0 / 3.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::c(i, 0) > 0) {
        const R cu = (R)L::c(i, 0) * ux + (R)L::c(i, 1) * uy + (R)L::c(i, 2) * uz;
        g[i] = g[opp(i)] + (R)6 * (R)L::w(i) * (rho * cu - (R)L::c(i, 0) * U) -
               (R)L::c(i, 1) * Ny - (R)L::c(i, 2) * Nz;
      }
    }
  }

  // 3. moments and collision
  R u[3];
  collide<Q, R>(p, g, delta, u);

  // 4. store
#pragma unroll
  for (int i = 0; i < Q; ++i) C::st(fd + i * p.ncell + id, g[i]);
  st_rec(vd, id, u[0], u[1], u[2], ntn);
}

// Face-free rows with two cells per thread (x0 = 2 * thread x index): pairs
// inside the lattice take bulk_interior2, the lone cell of a row end (odd nx,
// or a pair cut by the x-face columns of a non-periodic x axis) bulk_interior.
// Registers: two cells' populations are live at once; the budget is set by
// LBM_BULK2_MINB blocks of LBM_BULK_THREADS per SM (LBM_BULK2_MINB16 for
// 16-bit storage).  One instantiation per collision operator (COLL): with the
// operator chosen at run time the regularized operator's moments set the
// register peak of BGK lattices too (BGK channel 256x128x128, 1000 steps: FP16
// 36.5k -> 39.2k MLUPS, BF16 36.4k -> 37.1k, FP32 unchanged at 34.8k).  A
// budget of 80 registers for 16-bit storage (12 blocks of 64 threads per SM)
// gave 39.4k / 37.3k against 96 registers' 39.2k / 37.1k.
#ifndef LBM_BULK2_MINB
#define LBM_BULK2_MINB 10
#endif
#ifndef LBM_BULK2_MINB16
#define LBM_BULK2_MINB16 12
#endif
template <int Q, int ST, int COLL>
__global__ void __launch_bounds__(LBM_BULK_THREADS, (ST == ST_FP16 || ST == ST_BF16) ? LBM_BULK2_MINB16
                                                                                      : LBM_BULK2_MINB)
    k_bulk2(const Params p, int rows_arg) {
  const bool zy = rows_arg & ROWS_ZY;
  const int rows = rows_arg & ROWS_MASK;
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int r = (zy ? blockIdx.z : blockIdx.y) * blockDim.y + threadIdx.y;
  const int z = zy ? blockIdx.y : blockIdx.z;
  const int y = rows == ROWS_INNER ? r + 1 : r;
  if (x0 >= p.nx || y >= (rows == ROWS_INNER ? p.ny - 1 : p.ny)) return;
  // x-face columns of a non-periodic x axis belong to the ROWS_XEDGE launch
  const bool inA = p.px || (x0 >= 1 && x0 <= p.nx - 2);
  const bool inB = x0 + 1 < p.nx && (p.px || x0 + 1 <= p.nx - 2);
  if (inA && inB) bulk_interior2<Q, ST, COLL>(p, x0, y, z);
  else if (inA) bulk_interior<Q, ST>(p, x0, y, z);
  else if (inB) bulk_interior<Q, ST>(p, x0 + 1, y, z);
}

template <int Q, int ST, bool GENERAL>
__global__ void LBM_BULK_BOUNDS k_bulk(const Params p, int rows_arg) {
  const bool zy = rows_arg & ROWS_ZY;
  const int rows = rows_arg & ROWS_MASK;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = (zy ? blockIdx.z : blockIdx.y) * blockDim.y + threadIdx.y;
  const int z = zy ? blockIdx.y : blockIdx.z;
  int y = r;
  int xx = x;
  if (rows == ROWS_INNER) y = r + 1;
  else if (rows == ROWS_WALL) y = r == 0 ? 0 : (r == 1 ? p.ny - 1 : p.ny);
  else if (rows == ROWS_XEDGE) {
    y = r + 1;
    xx = x == 0 ? 0 : (x == 1 ? p.nx - 1 : p.nx);
    if (x == 1 && p.nx == 1) return;   // a single column is column 0
  }
  if (xx >= p.nx || y >= p.ny || ((rows == ROWS_INNER || rows == ROWS_XEDGE) && y >= p.ny - 1)) return;
  // x-face columns of a non-periodic x axis belong to the ROWS_XEDGE launch
  if (rows == ROWS_INNER && !p.px && (xx == 0 || xx == p.nx - 1)) return;
  bulk_cell<Q, ST, GENERAL>(p, xx, y, z);
}

// ----------------------------------------------------------------------------
// Inner rows with TMA staging.  Block = 32 x 8 cells of one z plane; it marches
// over `zchunk` planes.  For every plane one thread issues Q tiled loads, one
// per direction i: the box of source cells x - c_i of the tile, i.e. rows
// y0 - c_iy .. y0 - c_iy + 7 of plane z - c_iz, widened in x to start at the
// 16-byte boundary x0 - XOFF.  Two stages: the next plane is in flight while
// the current one is computed.  The wrap-around columns of a periodic x axis
// (x = -1 and x = nx), which a tiled load fills with zeros, are patched from
// global memory.  Waits are bounded; on expiry the block records
// FLAG_TMA_TIMEOUT, waits (bounded) for its copies in flight and leaves.
// ----------------------------------------------------------------------------
template <int Q, int ST>
struct TmaTile {
  using T = typename Codec<ST>::T;
  static constexpr int XOFF = 16 / (int)sizeof(T);   // elements in 16 bytes
  static constexpr int BW = 32 + 2 * XOFF;           // box width (x)
  static constexpr int BH = 8;                       // box height (y)
  static constexpr uint32_t BOX_BYTES = BW * BH * sizeof(T);
  static constexpr uint32_t STAGE_BYTES = Q * BOX_BYTES;
  static constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 128 + 16;   // stages, alignment, barriers
  static_assert(BOX_BYTES % 128 == 0, "boxes keep 128-byte alignment");
  static_assert((XOFF * sizeof(T)) % 16 == 0 && (BW * sizeof(T)) % 16 == 0, "16-byte tiles");
};

// Polls of an mbarrier before a block of the TMA-staged kernel gives up on a
// tile (the default of Params::wait_limit) and the bound of the drain that
// follows a give-up.
constexpr int kTmaDrainLimit = 1 << 24;

// Minimum resident blocks per SM for the TMA-staged kernel (its register
// budget); its two shared-memory stages take 2 x Q boxes per block.
#ifndef LBM_TMA_MINB
#define LBM_TMA_MINB 4
#endif

template <int Q, int ST>
__global__ void __launch_bounds__(256, LBM_TMA_MINB)
    k_bulk_tma(const Params p, const __grid_constant__ CUtensorMap tmap, int zchunk) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  using TT = TmaTile<Q, ST>;
  constexpr int XOFF = TT::XOFF, BW = TT::BW, BH = TT::BH;
  // dynamic shared memory, aligned here to the 128 bytes a tiled bulk copy
  // destination needs: [2][Q][BH][BW] elements, then the two mbarriers
  extern __shared__ unsigned char tma_smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tma_smem_raw + 127) & ~(uintptr_t)127);
  T* sm = (T*)base;
  uint64_t* bar = (uint64_t*)(base + 2 * TT::STAGE_BYTES);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const int x0 = blockIdx.x * 32, y0 = 1 + blockIdx.y * BH;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(p.nz, z0 + zchunk);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < p.nx && y <= p.ny - 2;
  const T* LBM_RESTRICT fs = (const T*)p.f_src;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int issued = 0;   // loads issued (thread 0)
  if (tid == 0 && z0 < z1) {
    mbar_arrive_expect_tx(&bar[0], TT::STAGE_BYTES);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      int zs = z0 - L::c(i, 2);
      zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
      tma_load_4d(sm + (0 * Q + i) * BH * BW, &tmap, x0 - XOFF, y0 - L::c(i, 1), zs, i, &bar[0]);
    }
    issued = 1;
  }
  for (int z = z0, k = 0; z < z1; ++z, ++k) {
    const int s = k & 1;
    if (tid == 0 && z + 1 < z1) {
      // stage s^1 was last read before the barrier that closed iteration k-1
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[s ^ 1], TT::STAGE_BYTES);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        int zs = z + 1 - L::c(i, 2);
        zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
        tma_load_4d(sm + ((s ^ 1) * Q + i) * BH * BW, &tmap, x0 - XOFF, y0 - L::c(i, 1), zs, i,
                    &bar[s ^ 1]);
      }
      ++issued;
    }
    bool ok = false;
    for (long long it = 0; it < p.wait_limit; ++it) {
      if (mbar_try_wait(&bar[s], (uint32_t)((k >> 1) & 1))) {
        ok = true;
        break;
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(p.flags, FLAG_TMA_TIMEOUT);
        // copies may still be in flight into this block's stages: wait for both
        // (bounded by the default limit, whatever p.wait_limit is) before leaving
        for (int it = 0; it < kTmaDrainLimit && !mbar_try_wait(&bar[s], (uint32_t)((k >> 1) & 1)); ++it) {
        }
        if (issued > k + 1)
          for (int it = 0; it < kTmaDrainLimit && !mbar_try_wait(&bar[s ^ 1], (uint32_t)(((k + 1) >> 1) & 1)); ++it) {
          }
      }
      return;
    }
    T* st = sm + s * Q * BH * BW;
    if (p.px && (x0 == 0 || x0 + 32 >= p.nx)) {
      // periodic x: source column x = -1 is column nx-1, source column x = nx is column 0
      int j = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int cx = L::c(i, 0);
        if (cx == 0) continue;
        const int col = cx > 0 ? XOFF - 1 : p.nx - x0 + XOFF;
        const bool need = cx > 0 ? x0 == 0 : x0 + 32 >= p.nx;
        if (need && tid >= j * BH && tid < (j + 1) * BH) {
          const int r = tid - j * BH;
          const int ys = y0 + r - L::c(i, 1);
          int zs = z - L::c(i, 2);
          zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
          if (ys >= 0 && ys < p.ny)
            st[(i * BH + r) * BW + col] = fs[i * p.ncell + ((long long)zs * p.ny + ys) * p.pitch +
                                             (cx > 0 ? p.nx - 1 : 0)];
        }
        ++j;
      }
      __syncthreads();
    }
    // x-face cells of a non-periodic x axis are left to the ROWS_XEDGE launch
    if (active && (p.px || (x != 0 && x != p.nx - 1))) {
      R g[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = (R)C::ld_raw(st + (i * BH + ty) * BW + tx + XOFF - L::c(i, 0));
      const NbOff o = nb_offsets(p, x, y, z);
      interior_finish<Q, ST>(p, o, g, x, y);
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// Wall pre-pass: one thread per wall node of face fi (0 = ymin, 1 = ymax).
// ----------------------------------------------------------------------------
// WALLS: the wall class the caller has checked (WALLS_BB: slip bounce-back,
// WALLS_REG: regularized, HRFD or Cai-Degrigny), whose branch alone is compiled;
// WALLS_ANY decides per face at run time.
// COLL: the collision operator of a regularized node's own step (COLL_ANY:
// p.collision at run time).
enum { WALLS_ANY = 0, WALLS_BB = 1, WALLS_REG = 2 };
template <int Q, int ST, int WALLS = WALLS_ANY, int COLL = COLL_ANY>
__device__ __forceinline__ void wall_node(const Params& p, int fi, int node) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  const int nwx = p.nx - p.xw0[fi];
  const int z = node / nwx;
  const int x = p.xw0[fi] + node % nwx;
  const int yB = fi == 0 ? 0 : p.ny - 1;
  const int s = fi == 0 ? 1 : -1;   // inward direction along y
  const R* LBM_RESTRICT vs = (const R*)p.v_src;
  R* LBM_RESTRICT vd = (R*)p.v_dst;
  const T* LBM_RESTRICT fs = (const T*)p.f_src;
  const double nu = p.nu;
  const long long idB = cidx(p, x, yB, z);
  double ut = 0.0;
  bool ok = true;

  const bool bb = WALLS == WALLS_BB || (WALLS == WALLS_ANY && p.wall[fi] == BC_WALL_BB);
  if (bb) {
    // Section 3.2: u_tau from the tangential velocity at the reference node.
    // Everything but the Newton inversion runs in the compute type R.
    const int yR = yB + s * (p.ref_node[fi] - 1);
    const double dw = p.d_w[fi];                       // y_B (1/2 half-way)
    const double yref = (double)(p.ref_node[fi] - 1) + dw;
    const long long idR = cidx(p, x, yR, z);
    const R Ux = vs[4 * idR], Uz = vs[4 * idR + 2];
    const R Um = nn_sqrt(Ux * Ux + Uz * Uz);
    const R iU = Um > (R)0 ? (R)1 / Um : (R)0;
    const R tx = Um > (R)0 ? Ux * iU : (R)1, tz = Uz * iU;
    R* uw = (R*)p.uw[fi] + 3 * node;
    if (!isfinite(Um)) atomicOr(p.flags, FLAG_NONFINITE);   // reported, not turned into u_tau = 0
    if (p.turbulent) {
      ok = solve_utau_mixed(p.wall_law, p.law_kappa, p.law_B, (double)Um, yref, nu, p.inv_nu,
                            p.utau[fi][node], &ut);
      const R utr = (R)ut, nur = psel<R>(p.nu, p.nu_f), kap = (R)WF::kappa;
      const R ypB = utr * (R)dw * psel<R>(p.inv_nu, p.inv_nu_f);
      // Eq. 35 with Delta_w = y_B = d_w and nu_t|_B = nu kappa y_B+
      const R slip = fdiv(utr * utr * (R)dw, nur * ((R)1 + kap * ypB));
      uw[0] = vs[4 * idB] - slip * tx;
      uw[1] = (R)0;
      uw[2] = vs[4 * idB + 2] - slip * tz;
      vd[4 * idB + 3] = nur * kap * ypB;
    } else {
      uw[0] = uw[1] = uw[2] = (R)0;
    }
    R rho = (R)1;
#pragma unroll
    for (int i = 0; i < Q; ++i) rho += (R)C::ld(fs + i * p.ncell + idB);
    ((R*)p.rhow[fi])[node] = rho;
  } else {
    // Section 3.1: regularized node with the HRFD gradient
    const int yF = yB + s, yFF = yB + 2 * s;
    // With periodic x every source below is inside the lattice or across a
    // periodic face (F takes all directions from rows yB..yB+2s, B only those
    // with c.n >= 0, from rows yB and yF): plain neighbour offsets.
    const bool px = p.px != 0;
    const NbOff oF = nb_offsets(p, x, yF, z), oB = nb_offsets(p, x, yB, z);
    R jF[3] = {(R)0.5 * psel<R>(p.F[0], p.F_f[0]), (R)0.5 * psel<R>(p.F[1], p.F_f[1]), (R)0.5 * psel<R>(p.F[2], p.F_f[2])};
    R rhoF = (R)1;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      bool known;
      const R gi = px ? pull_nb<Q, ST>(p, oF, i) : pull_bc<Q, ST>(p, x, yF, z, i, &known);
      rhoF += gi;
      jF[0] += (R)L::c(i, 0) * gi;
      jF[1] += (R)L::c(i, 1) * gi;
      jF[2] += (R)L::c(i, 2) * gi;
    }
    // everything but the Newton inversion runs in the compute type R
    const R irF = fdiv((R)1, rhoF);
    const R Ux = (jF[0] + psel<R>(p.Ush, p.Ush_f)) * irF, Uz = jF[2] * irF;
    const R Um = nn_sqrt(Ux * Ux + Uz * Uz);
    const R iU = Um > (R)0 ? (R)1 / Um : (R)0;
    const R tx = Um > (R)0 ? Ux * iU : (R)1, tz = Uz * iU;
    const double dw = p.d_w[fi];                       // y_B; y_F = 1 + d_w
    if (!isfinite(Um)) atomicOr(p.flags, FLAG_NONFINITE);
    if (p.turbulent)
      ok = solve_utau_mixed(p.wall_law, p.law_kappa, p.law_B, (double)Um, 1.0 + dw, nu, p.inv_nu,
                            p.utau[fi][node], &ut);
    const R utr = (R)ut, inu = psel<R>(p.inv_nu, p.inv_nu_f);
    const R ypB = utr * (R)dw * inu;
    const R uplB = p.turbulent ? wf_uplus_r<R>(p, ypB) : (R)0;         // u+(y_B+)
    const R upB = utr * uplB;                                          // u_B = u_tau u+(y_B+)
    const R uB[3] = {upB * tx, (R)0, upB * tz};
    // Eq. 23 with u_B . n = 0: rho_B = f_par + 2 f_perp (deviations: weights sum to 1)
    R gpar = 0, gperp = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cn = -s * L::c(i, 1);   // c . n with n the outward normal
      if (cn >= 0) {
        bool known;
        const R gi = px ? pull_nb<Q, ST>(p, oB, i) : pull_bc<Q, ST>(p, x, yB, z, i, &known);
        if (cn == 0) gpar += gi; else gperp += gi;
      }
    }
    const R rhoB = (R)1 + gpar + (R)2 * gperp;
    // velocity gradient G[a][c] = d_a u_c at B from the previous-step velocity
    R G[3][3];
    if (px) {
      const Rec<R> xm = ld_rec(vs, oB.id + oB.oxm), xp = ld_rec(vs, oB.id + oB.oxp);
      G[0][0] = (R)0.5 * (xp.x - xm.x);
      G[0][1] = (R)0.5 * (xp.y - xm.y);
      G[0][2] = (R)0.5 * (xp.z - xm.z);
    } else {
      const Nb<R> xm = neighbour<R>(p, vs, x, yB, z, 0, -1);
      const Nb<R> xp = neighbour<R>(p, vs, x, yB, z, 0, +1);
#pragma unroll
      for (int c = 0; c < 3; ++c) G[0][c] = (R)0.5 * (xp.u[c] - xm.u[c]);
    }
    if (Q == 19) {
      const Rec<R> zm = ld_rec(vs, oB.id + oB.ozm), zp = ld_rec(vs, oB.id + oB.ozp);   // z periodic
      G[2][0] = (R)0.5 * (zp.x - zm.x);
      G[2][1] = (R)0.5 * (zp.y - zm.y);
      G[2][2] = (R)0.5 * (zp.z - zm.z);
    } else {
      G[2][0] = G[2][1] = G[2][2] = (R)0;
    }
    const long long idF = cidx(p, x, yF, z), idFF = cidx(p, x, yFF, z);
    const bool cai = p.wall[fi] == BC_WALL_CAI;
    R ana;
    if (cai) {
      // Eq. 29: (u_tau / Delta)(-11/6 u+(y_B+) + 3 u+(y_B+ + D+) - 3/2 u+(y_B+ + 2D+)
      //          + 1/3 u+(y_B+ + 3D+)), Delta = 1, D+ = u_tau / nu
      const R dp = utr * inu;
      ana = ut > 0.0 ? utr * ((R)(-11.0 / 6.0) * uplB +
                              (R)3 * wf_uplus_r<R>(p, ypB + dp) -
                              (R)1.5 * wf_uplus_r<R>(p, ypB + (R)2 * dp) +
                              wf_uplus_r<R>(p, ypB + (R)3 * dp) * (R)(1.0 / 3.0))
                     : (R)0;
    } else {
      const R dup = ypB > (R)0 ? wf_dudy_r<R>(p, ypB) : (R)1;
      ana = ut > 0.0 ? utr * utr * inu * dup : (R)0;   // Eq. 15
    }
    const R tdir[3] = {tx, (R)0, tz};
    const R beta = cai ? (R)1 : (R)p.beta[fi];     // Eq. 30: beta = 1 with Eq. 29
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R fd = (R)0.5 * ((R)-3 * vs[4 * idB + c] + (R)4 * vs[4 * idF + c] -
                             vs[4 * idFF + c]);                              // Eq. 28
      R dn = fd;
      if (c != 1 && p.turbulent) dn = beta * (ana * tdir[c]) + ((R)1 - beta) * fd;  // Eq. 27
      G[1][c] = (R)s * dn;
    }
    const R ntB = vs[4 * idB + 3];
    const R nutB = p.turbulent ? sa_nut<R>(ntB, psel<R>(p.inv_nu, p.inv_nu_f)) : (R)0;
    const R tau = (R)0.5 + (R)3 * (psel<R>(p.nu, p.nu_f) + nutB);
    const R Sxx = G[0][0], Syy = G[1][1], Szz = G[2][2];
    const R Sxy = (R)0.5 * (G[0][1] + G[1][0]), Sxz = (R)0.5 * (G[0][2] + G[2][0]),
            Syz = (R)0.5 * (G[1][2] + G[2][1]);
    const R trS = (Sxx + Syy + Szz) * (R)(1.0 / 3.0);
    const R Us = psel<R>(p.Ush, p.Ush_f);
    const R dux = uB[0] - Us;
    const R uu15 = (R)1.5 * (uB[0] * uB[0] + uB[2] * uB[2]);
    const R du15 = (R)1.5 * (dux * ((R)2 * Us + dux) + uB[2] * uB[2]);
    // Eqs. 19, 26: f_i = f_i^eq(rho_B, u_B) - 3 w_i rho_B tau Q_i:S, over opposite
    // pairs (i, i+1): Q_i:S is even in c_i, the equilibrium splits into the even
    // and odd parts of the per-weight-class polynomial (eq_pair)
    R g[Q];
    const R drB = rhoB - (R)1, one_m_uu15 = (R)1 - uu15, rt3 = (R)3 * rhoB * tau;
    const EqCoef<R> k1 = eq_coef<R>((R)L::w(1), rhoB, drB, Us, one_m_uu15, du15);
    const EqCoef<R> k2 = eq_coef<R>((R)L::w(Q == 19 ? 7 : 5), rhoB, drB, Us, one_m_uu15, du15);
    g[0] = (R)L::w(0) * ((drB * one_m_uu15 - du15) + rt3 * trS);   // Q_0:S = -tr(S)/3
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
      const EqCoef<R>& k = L::w(i) < L::w(1) ? k2 : k1;
      R ev, od;
      eq_pair<Q, R>(k, cx, cdot<Q, R>(i, dux, (R)0, uB[2]), &ev, &od);
      const R qs = (R)(cx * cx) * Sxx + (R)(cy * cy) * Syy + (R)(cz * cz) * Szz +
                   (R)2 * ((R)(cx * cy) * Sxy + (R)(cx * cz) * Sxz + (R)(cy * cz) * Syz) - trS;
      const R e = ev - (R)L::w(i) * rt3 * qs;
      g[i] = e + od;
      g[i + 1] = e - od;
    }
    // the node's own step, in the wall pass: nu_tilde_B (Dirichlet), relaxation
    // rate, collision of the rebuilt populations and the stores (the wall-row
    // kernels leave regularized wall nodes alone)
    const R ntn = p.turbulent ? psel<R>(p.nu, p.nu_f) * (R)WF::kappa * ypB : ntB;
    const R nutn = p.turbulent ? sa_nut<R>(ntn, psel<R>(p.inv_nu, p.inv_nu_f)) : (R)0;
    R u[3];
    collide<Q, R, 1, COLL>(p, g, relax_delta<R>((R)3 * (psel<R>(p.nu, p.nu_f) + nutn)), u);   // Eq. 8
    T* LBM_RESTRICT fdst = (T*)p.f_dst;
#pragma unroll
    for (int i = 0; i < Q; ++i) C::st(fdst + i * p.ncell + idB, g[i]);
    st_rec(vd, idB, u[0], u[1], u[2], ntn);
  }
  p.utau[fi][node] = ut;
  if (!ok) {   // Newton reached its iteration limit: flag and count the node update
    atomicOr(p.flags, FLAG_NEWTON);
    atomicAdd(p.flags + 1, 1u);
  }
}

// One face per grid row (blockIdx.y); the blocks of a row stride over the
// face's nodes.  The grid is sized by the host to a few blocks per SM: the
// pass is bound by the FP64 pipe, which a few warps per SM keep busy, and the
// registers it does not hold stay with the inner-row kernel running beside it.
// Minimum resident wall-pass blocks per SM requested from the compiler: its
// register budget (8: 64 registers), which is also what the pass takes from
// the inner-row kernel running beside it.
#ifndef LBM_WALL_MINB
#define LBM_WALL_MINB 8
#endif
#ifndef LBM_WALL_REG_MINB
#define LBM_WALL_REG_MINB LBM_WALL_MINB   // the regularized class's budget
#endif
// One kernel per wall class (WALLS_BB / WALLS_REG), so that a warp's code holds
// one scheme only; a face of the other class is left to the other kernel.  The
// regularized class is compiled once per collision operator of the nodes' own
// step (FP32, 64 registers: 44 B of spill stores per thread with the operator
// chosen at run time, 4 B for BGK only).
template <int Q, int ST, int WALLS, int COLL = COLL_ANY>
__global__ void __launch_bounds__(128, WALLS == WALLS_BB ? LBM_WALL_MINB : LBM_WALL_REG_MINB)
    k_wall(const Params p) {
  const int fi = blockIdx.y;
  if (!p.wall[fi] || (p.wall[fi] == BC_WALL_BB) != (WALLS == WALLS_BB)) return;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < p.nwall[fi];
       node += gridDim.x * blockDim.x)
    wall_node<Q, ST, WALLS, COLL>(p, fi, node);
}

// ----------------------------------------------------------------------------
// Initial state from physical fields: f* = f^eq(rho, u), u^0 = u.
// ----------------------------------------------------------------------------
template <int Q, int ST>
__global__ void k_init(const Params p, const double* rho, const double* u, const double* nt,
                       double rho0, double ucv, double nucv) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  const long long n = (long long)p.nx * p.ny * p.nz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % p.nx);
    const int y = (int)((k / p.nx) % p.ny);
    const int z = (int)(k / ((long long)p.nx * p.ny));
    const long long id = cidx(p, x, y, z);
    const double uxd = u[k] * ucv;
    const R drho = (R)(rho[k] / rho0 - 1.0);
    const R ux = (R)uxd, uy = (R)(u[k + n] * ucv), uz = (R)(u[k + 2 * n] * ucv);
    const R U = psel<R>(p.Ush, p.Ush_f);
    const R dux = (R)(uxd - p.Ush);
    const R uu15 = (R)1.5 * (ux * ux + uy * uy + uz * uz);
    const R du15 = (R)1.5 * (dux * ((R)2 * U + dux) + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      C::st((T*)p.f_dst + i * p.ncell + id, heq_dev<Q, R>(i, drho, dux, uy, uz, U, uu15, du15));
    st_rec((R*)p.v_dst, id, ux, uy, uz, (R)(nt[k] * nucv));
  }
}

// ----------------------------------------------------------------------------
// Physical-unit export of rho, u, nu_t, nu_tilde into dense float64 arrays.
// ----------------------------------------------------------------------------
template <int Q, int ST>
__global__ void k_fields(const Params p, double* rho, double* u, double* nut, double* nt,
                         double rho0, double vel, double visc) {
  using C = Codec<ST>;
  using R = typename Compute<ST>::R;
  using T = typename C::T;
  const long long n = (long long)p.nx * p.ny * p.nz;
  const T* fs = (const T*)p.f_src;
  const R* vs = (const R*)p.v_src;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % p.nx);
    const int y = (int)((k / p.nx) % p.ny);
    const int z = (int)(k / ((long long)p.nx * p.ny));
    const long long id = cidx(p, x, y, z);
    double r = 1.0;
    bool fin = true;
    for (int i = 0; i < Q; ++i) {
      const double gi = (double)C::ld(fs + i * p.ncell + id);
      fin = fin && isfinite(gi);
      r += gi;
    }
    if (rho) rho[k] = r * rho0;
    double ntl, ux0 = 0.0;
    if (u) {
      const Rec<R> rec = ld_rec(vs, id);
      ux0 = (double)rec.x;
      u[k] = ux0 * vel;
      u[k + n] = (double)rec.y * vel;
      u[k + 2 * n] = (double)rec.z * vel;
      ntl = (double)rec.n;
    } else {
      ntl = (double)vs[4 * id + 3];   // nu_tilde alone
    }
    if (nt) nt[k] = ntl * visc;
    if (nut) {
      const double chi = ntl / p.nu, c3 = chi * chi * chi;
      nut[k] = p.turbulent ? ntl * c3 / (c3 + 7.1 * 7.1 * 7.1) * visc : 0.0;
    }
    fin = fin && isfinite(ux0) && isfinite(ntl);
    if (!fin) atomicOr(p.flags, FLAG_NONFINITE);
  }
}

// ----------------------------------------------------------------------------
// Deterministic FP64 reduction of mass and momentum.  Block b sums the cells
// [b*chunk, (b+1)*chunk) with a fixed thread stride and a fixed tree; the
// partials are summed in block order by k_reduce_final.
// ----------------------------------------------------------------------------
template <int Q, int ST>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(const Params p, double* partial,
                                                        long long chunk) {
  using L = Lat<Q>;
  using C = Codec<ST>;
  using T = typename C::T;
  __shared__ double sh[RED_VALS][RED_THREADS];
  const long long n = (long long)p.nx * p.ny * p.nz;
  const long long b0 = blockIdx.x * chunk;
  const long long b1 = b0 + chunk < n ? b0 + chunk : n;
  const T* fs = (const T*)p.f_src;
  double acc[RED_VALS] = {0, 0, 0, 0};
  bool fin = true;
  for (long long k = b0 + threadIdx.x; k < b1; k += RED_THREADS) {
    const int x = (int)(k % p.nx);
    const int y = (int)((k / p.nx) % p.ny);
    const int z = (int)(k / ((long long)p.nx * p.ny));
    const long long id = cidx(p, x, y, z);
    double m = 1.0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double gi = (double)C::ld(fs + i * p.ncell + id);
      fin = fin && isfinite(gi);
      m += gi;
      jx += L::c(i, 0) * gi;
      jy += L::c(i, 1) * gi;
      jz += L::c(i, 2) * gi;
    }
    acc[0] += m;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
  }
  if (!fin) atomicOr(p.flags, FLAG_NONFINITE);
#pragma unroll
  for (int v = 0; v < RED_VALS; ++v) sh[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int v = 0; v < RED_VALS; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < RED_VALS; ++v) partial[blockIdx.x * RED_VALS + v] = sh[v][0];
  }
}

__global__ void k_reduce_final(const double* partial, int nblocks, double* out);
__global__ void k_wall_stats(const Params p, double* prev, double* out);

}  // namespace lbm
