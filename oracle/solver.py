"""The LBM-RANS step with both wall schemes (oracle, FP64, numpy).

Test infrastructure only (see the package docstring).

Lattice units throughout the step (dx = dt = 1, c_s^2 = 1/3).  Physical inputs
are converted with the acoustic scaling of Section 4.1.1:
dt = M dx / (sqrt(3) U_ref), u_lb = u dt/dx, nu_lb = nu dt/dx^2, and the body
force F = rho0 g becomes g dt^2/dx per unit lattice density.

One step n -> n+1, in the order used throughout this project (each stage a
separate plain loop over the whole field, no fusion):

1. SA update (Section 2.2): nu_tilde^{n+1} from nu_tilde^n and u^n on all cells
   that are not Dirichlet nodes.
2. Bounce-back wall pre-pass (Section 3.2): at each boundary node B the
   tangential velocity u^n at the reference node (B or F) gives u_tau by Newton
   on the wall law; y_B+ = u_tau y_B / nu; nu_t|_B = nu kappa y_B+; the slip
   velocity is Eq. 35, u_w = u_B - u_tau^2 Delta_w / (nu + nu_t|_B) with
   Delta_w = d_w, the wall-to-B distance (1/2 for the half-way placement,
   Section 4.1.2.5); rho_w = rho^n(B); the Dirichlet value
   nu_tilde_B = nu kappa y_B+ with y_B = d_w.
3. Streaming (Eq. 3) by pulling f*^n(x - c_i); periodic axes wrap; populations
   whose source lies outside a non-periodic face are unknown.
4. y-face conditions: half-way bounce-back with the moving-wall term (Eq. 31)
   or its interpolated forms for d_w != 1/2 (Bouzidi, Eq. 36; Yu, Eq. 37),
   specular reflection (symmetry), or equilibrium at the free-stream state.
5. x-face conditions: Zou-He velocity inlet, zero-gradient outlet (copy of the
   post-stream populations of the neighbouring column).
6. Regularized (HRFD) wall nodes (Section 3.1): rho_F, u_F after streaming
   (Eqs. 20-22); Newton at F (y_F = 1 + d_w); u_B = u_tau u+(y_B+) t with
   y_B = d_w; rho_B by Eq. 23; strain
   rate with the blended wall-normal derivative of Eqs. 27-28 on the velocity
   of the previous step; all populations of B replaced by Eq. 19 with Eq. 26.
7. Moments (Eqs. 4-5), nu_t^{n+1} = nu_tilde^{n+1} f_v1, omega from Eq. 8 with
   nu + nu_t, collision (BGK or regularized, Guo forcing).

Readings where the paper is silent are stated at the point of use.
"""
from __future__ import annotations

import math

import numpy as np

from . import bounce as BB
from . import lattice as L
from . import sa as SA
from .wallfn import KAPPA, WallLaw, solve_u_tau

_AX = {"x": 0, "y": 1, "z": 2}


class Oracle:
    """Plain FP64 solver for one case.

    ``case`` supplies the attributes of ``lbm_cases.Case``; ``rho``, ``u``, ``nut``
    are the initial density (kg/m^3), velocity (m/s, [3, z, y, x]) and SA working
    variable (m^2/s) in physical units.
    """

    def __init__(self, case, rho, u, nut):
        self.case = case
        self.vs = L.VelocitySet(case.lattice)
        self.nx, self.ny, self.nz = case.nx, case.ny, case.nz
        bcs = case.bcs
        for f in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax"):
            if f not in bcs:
                raise ValueError(f"missing boundary {f}")
        self.bc = bcs
        if bcs["zmin"].kind != "periodic" or bcs["zmax"].kind != "periodic":
            raise ValueError("z faces must be periodic")
        for ax in ("x", "y"):
            a, b = bcs[ax + "min"].kind, bcs[ax + "max"].kind
            if (a == "periodic") != (b == "periodic"):
                raise ValueError(f"{ax} faces: periodic must be paired")
        for f in ("xmin", "xmax"):
            if bcs[f].kind in ("wall_bb", "wall_hrfd", "wall_cai_degrigny", "symmetry",
                               "freestream"):
                raise ValueError("x faces: periodic, inlet or outlet only")
        if bcs["xmin"].kind == "outlet_zerograd" or bcs["xmax"].kind == "inlet_zouhe":
            raise ValueError("inlet on xmin, outlet on xmax only")
        for f in ("ymin", "ymax"):
            if bcs[f].kind in ("inlet_zouhe", "outlet_zerograd"):
                raise ValueError("y faces: periodic, wall, symmetry or free stream")
            b = bcs[f]
            if b.kind in ("wall_bb", "wall_hrfd", "wall_cai_degrigny"):
                if not (0.0 < b.d_w <= 1.0):
                    raise ValueError("d_w must lie in (0, 1]")
                if b.kind == "wall_bb" and b.interp == "none" and b.d_w != 0.5:
                    raise ValueError("half-way bounce-back needs d_w = 1/2")
            if b.interp != "none" and b.kind != "wall_bb":
                raise ValueError("interpolation applies to bounce-back walls only")
        self.periodic = {ax: bcs[ax + "min"].kind == "periodic" for ax in "xyz"}

        # acoustic scaling (Section 4.1.1)
        self.dt = case.mach * case.dx / (math.sqrt(3.0) * case.u_ref)
        self.ucv = self.dt / case.dx
        self.nucv = self.dt / case.dx ** 2
        self.nu = case.nu * self.nucv
        self.F = np.array(case.force, dtype=np.float64) * self.dt ** 2 / case.dx
        self.turbulent = case.turbulence == "sa"
        self.law = WallLaw(case.wall_law, case.kappa, case.B)

        # initial state: f*^0 = f^eq(rho, u), u^0 = u
        self.rho = np.asarray(rho, dtype=np.float64) / case.rho0
        self.u = np.asarray(u, dtype=np.float64) * self.ucv
        self.nt = np.asarray(nut, dtype=np.float64) * self.nucv
        self.fs = L.equilibrium(self.vs, self.rho, self.u)

        # geometry: cell centres (physical x), wall columns, wall distance
        self.xc = case.origin[0] + (np.arange(self.nx) + 0.5) * case.dx
        self.walls = {}
        for f in ("ymin", "ymax"):
            if bcs[f].kind in ("wall_bb", "wall_hrfd", "wall_cai_degrigny"):
                self.walls[f] = self.xc >= bcs[f].x_start
        self.inv_d2 = self._inv_wall_distance_sq()
        self.utau = {f: np.zeros((self.nz, self.nx)) for f in self.walls}
        self.nsteps = 0

    # ------------------------------------------------------------------ geometry
    def _row(self, face):
        return 0 if face == "ymin" else self.ny - 1

    def _inward(self, face):
        return 1 if face == "ymin" else -1

    def _inv_wall_distance_sq(self):
        """1/d^2 with d the distance from the cell centre to the nearest wall
        (lattice units).  A wall face with a leading edge at x_start is the
        half-line x >= x_start; upstream cells measure to its edge point."""
        j = np.arange(self.ny, dtype=np.float64)
        d = np.full((self.ny, self.nx), np.inf)
        for f in self.walls:
            dw = self.bc[f].d_w
            dy = j + dw if f == "ymin" else (self.ny - 1 - j) + dw
            xs = self.bc[f].x_start
            dxl = np.where(self.xc >= xs, 0.0, (self.xc - xs) / self.case.dx) if np.isfinite(xs) \
                else np.zeros(self.nx)
            d = np.minimum(d, np.sqrt(dy[:, None] ** 2 + dxl[None, :] ** 2))
        with np.errstate(divide="ignore"):
            inv = np.where(np.isfinite(d), 1.0 / d ** 2, 0.0)
        return np.broadcast_to(inv[None], (self.nz, self.ny, self.nx))

    # ---------------------------------------------------------------- ghosts
    def _pad(self, nt, u):
        """One ghost layer for the SA stencil.  Periodic: wrap; symmetry and
        wall faces: mirror (normal velocity negated); free stream and inlet: the
        prescribed state; outlet: zero gradient."""
        ntp = np.pad(nt, 1, mode="wrap")
        up = np.pad(u, ((0, 0), (1, 1), (1, 1), (1, 1)), mode="wrap")
        nu_in = {}
        for f in ("xmin", "xmax", "ymin", "ymax"):
            b = self.bc[f]
            if b.kind == "periodic":
                continue
            ax = f[0]
            axi = 2 - _AX[ax]
            lo = f.endswith("min")
            ghost = [slice(None)] * 3
            inner = [slice(None)] * 3
            ghost[axi] = 0 if lo else -1
            inner[axi] = 1 if lo else -2
            g, i = tuple(ghost), tuple(inner)
            if b.kind in ("symmetry", "wall_bb", "wall_hrfd", "wall_cai_degrigny"):
                ntp[g] = ntp[i]
                for c in range(3):
                    up[(c,) + g] = up[(c,) + i] * (-1.0 if c == _AX[ax] else 1.0)
            elif b.kind == "outlet_zerograd":
                ntp[g] = ntp[i]
                for c in range(3):
                    up[(c,) + g] = up[(c,) + i]
            else:  # inlet or free stream
                ntp[g] = b.nut_ratio_in * self.nu
                uin = np.array(b.u_in) * self.ucv
                for c in range(3):
                    up[(c,) + g] = uin[c]
        return ntp, up

    # ------------------------------------------------------------------ stages
    def sa_update(self):
        """Stage 1: explicit Euler step of Eq. 11 on every non-Dirichlet cell."""
        if not self.turbulent:
            return self.nt.copy()
        ntp, up = self._pad(self.nt, self.u)
        new = np.maximum(self.nt + SA.rhs(ntp, up, self.nu, self.inv_d2), 0.0)
        if self.bc["xmin"].kind == "inlet_zouhe":
            new[:, :, 0] = self.bc["xmin"].nut_ratio_in * self.nu
        return new

    def _tangential(self, uvec):
        """Tangential part (y component removed), its magnitude and unit vector."""
        ut = uvec.copy()
        ut[1] = 0.0
        U = np.sqrt((ut * ut).sum(axis=0))
        t = np.zeros_like(ut)
        t[0] = 1.0
        nz = U > 0.0
        t[:, nz] = ut[:, nz] / U[nz]
        return ut, U, t

    def bb_prepass(self, face, nt_new):
        """Stage 2 for one slip-velocity bounce-back face (Eq. 35, Section 3.2)."""
        b = self.bc[face]
        row, s = self._row(face), self._inward(face)
        cols = self.walls[face]
        ref = row + s * (b.ref_node - 1)
        y_ref = (b.ref_node - 1) + b.d_w
        uB = self.u[:, :, row, :][:, :, cols]
        uR = self.u[:, :, ref, :][:, :, cols]
        ubt, _, _ = self._tangential(uB)
        _, U, t = self._tangential(uR)
        if self.turbulent:
            ut = solve_u_tau(self.law, U.ravel(), y_ref, self.nu).reshape(U.shape)
            ypB = ut * b.d_w / self.nu
            nutB = self.nu * KAPPA * ypB
            uw = ubt - (ut * ut * b.d_w / (self.nu + nutB))[None] * t
            tmp = nt_new[:, row, :]
            tmp[:, cols] = nutB
            nt_new[:, row, :] = tmp
        else:
            ut = np.zeros_like(U)
            uw = np.zeros_like(uB)
        rho_w = self.fs[:, :, row, :][:, :, cols].sum(axis=0)
        full = np.zeros((self.nz, self.nx))
        full[:, cols] = ut
        self.utau[face] = full
        return uw, rho_w

    def _link_neighbour(self, i, row):
        """f*_i at x_F = x_B - c_i for every column of the boundary row, [z, x].
        z wraps; x wraps when periodic, otherwise a link whose F node would leave
        the lattice through an x face takes F in the boundary column itself
        (zero gradient along x; reading)."""
        cx, cy, cz = (int(v) for v in self.vs.c[i])
        xs = np.arange(self.nx) - cx
        xs = np.mod(xs, self.nx) if self.periodic["x"] else np.clip(xs, 0, self.nx - 1)
        zs = np.mod(np.arange(self.nz) - cz, self.nz)
        plane = self.fs[i][:, row - cy, :]
        return plane[zs][:, xs]

    def stream(self):
        """Stage 3: f_i(x, t+1) = f*_i(x - c_i, t); unknowns are NaN."""
        vs = self.vs
        f = np.empty_like(self.fs)
        for i in range(vs.q):
            cx, cy, cz = (int(v) for v in vs.c[i])
            g = np.roll(self.fs[i], shift=(cz, cy, cx), axis=(0, 1, 2))
            if not self.periodic["x"]:
                if cx == 1:
                    g[:, :, 0] = np.nan
                elif cx == -1:
                    g[:, :, -1] = np.nan
            if not self.periodic["y"]:
                if cy == 1:
                    g[:, 0, :] = np.nan
                elif cy == -1:
                    g[:, -1, :] = np.nan
            f[i] = g
        return f

    def y_faces(self, f, bb):
        """Stage 4: bounce-back (Eq. 31), symmetry, free stream on y faces."""
        vs = self.vs
        mir = vs.mirror(1)
        for face in ("ymin", "ymax"):
            b = self.bc[face]
            if b.kind == "periodic":
                continue
            row = self._row(face)
            n_y = -1 if face == "ymin" else 1                  # outward normal
            cn = vs.c[:, 1] * n_y
            unknown = np.where(cn < 0)[0]
            toward = np.where(cn > 0)[0]
            wallcols = self.walls.get(face, np.zeros(self.nx, dtype=bool))
            symcols = ~wallcols
            if b.kind == "freestream":
                uinf = (np.array(b.u_in) * self.ucv).reshape(3, 1, 1)
                feq = L.equilibrium(vs, np.ones((1, 1)), uinf)
                for j in unknown:
                    f[j][:, row, :] = feq[j]
                continue
            # specular reflection on symmetry columns (and whole symmetry faces)
            for j in unknown:
                m = mir[j]
                cx, cz = int(vs.c[j, 0]), int(vs.c[j, 2])
                src = np.roll(self.fs[m][:, row, :], shift=(cz, cx), axis=(0, 1))
                if not self.periodic["x"]:
                    if cx == 1:
                        src[:, 0] = np.nan
                    elif cx == -1:
                        src[:, -1] = np.nan
                cur = f[j][:, row, :]
                cur[:, symcols] = src[:, symcols]
                f[j][:, row, :] = cur
            if b.kind == "wall_bb":
                uw, rho_w = bb[face]
                for i in toward:
                    o = vs.opp[i]
                    cu = (vs.cf[i][:, None, None] * uw).sum(axis=0)
                    mw = 2.0 * vs.w[i] * rho_w * cu / L.CS2
                    fs_i_B = self.fs[i][:, row, :][:, wallcols]
                    if b.interp == "none":
                        val = BB.halfway(fs_i_B, mw)                       # Eq. 31
                    else:
                        fs_i_F = self._link_neighbour(i, row)[:, wallcols]
                        fs_o_B = self.fs[o][:, row, :][:, wallcols]
                        val = BB.RULES[b.interp](b.d_w, fs_i_B, fs_i_F, fs_o_B, mw)
                    cur = f[o][:, row, :]
                    cur[:, wallcols] = val
                    f[o][:, row, :] = cur
        return f

    def x_faces(self, f):
        """Stage 5: Zou-He velocity inlet on xmin, zero-gradient outlet on xmax."""
        vs = self.vs
        b = self.bc["xmin"]
        if b.kind == "inlet_zouhe":
            col = f[:, :, :, 0]
            u = np.array(b.u_in) * self.ucv
            cx = vs.c[:, 0]
            rho = (col[cx == 0].sum(axis=0) + 2.0 * col[cx < 0].sum(axis=0)) / (1.0 - u[0])
            K = {t: (col[cx == 0] * vs.cf[cx == 0, t][:, None, None]).sum(axis=0) for t in (1, 2)}
            N = {t: 0.5 * K[t] - rho * u[t] / 3.0 for t in (1, 2)}
            for j in np.where(cx > 0)[0]:
                val = col[vs.opp[j]] + 2.0 * vs.w[j] * rho * (vs.cf[j] @ u) / L.CS2
                for t in (1, 2):
                    val = val - vs.c[j, t] * N[t]
                f[j][:, :, 0] = val
        if self.bc["xmax"].kind == "outlet_zerograd":
            for j in np.where(vs.c[:, 0] < 0)[0]:
                f[j][:, :, -1] = f[j][:, :, -2]
        return f

    def cai_degrigny_derivative(self, ut, d_w=0.5):
        """Eq. 29: third-order one-sided difference of the wall function at B,
        (u_tau / Delta) (-11/6 u+(y_B+) + 3 u+(y_B+ + D+) - 3/2 u+(y_B+ + 2 D+)
        + 1/3 u+(y_B+ + 3 D+)), Delta = 1 (lattice), D+ = u_tau / nu,
        y_B = d_w."""
        yp = ut * d_w / self.nu
        dp = ut / self.nu
        up = self.law.u_plus
        return ut * (-11.0 / 6.0 * up(yp) + 3.0 * up(yp + dp) - 1.5 * up(yp + 2 * dp)
                     + up(yp + 3 * dp) / 3.0)

    def hrfd(self, f, nt_new):
        """Stage 6: regularized wall nodes with the HRFD gradient (Section 3.1),
        or with the Cai-Degrigny gradient (Section 3.1.2, Eq. 29).

        Parity pinned: the rebuilt populations carry rho_B (Eq. 23), rho_B u_B and
        the non-equilibrium second moment -2 rho_B tau_eff c_s^2 S with S written
        out from Eqs. 15, 27-28 (and Eq. 29) on states whose finite differences are
        known in closed form, for beta in {0, 0.28, 1}."""
        vs = self.vs
        Q = L.second_order_Q(vs)
        _, up = self._pad(self.nt, self.u)
        for face, cols in self.walls.items():
            b = self.bc[face]
            if b.kind not in ("wall_hrfd", "wall_cai_degrigny"):
                continue
            cai = b.kind == "wall_cai_degrigny"
            row, s = self._row(face), self._inward(face)
            F_, FF = row + s, row + 2 * s
            n_y = -1.0 if face == "ymin" else 1.0
            fF = f[:, :, F_, :][:, :, cols]
            rhoF = fF.sum(axis=0)
            uF = (np.tensordot(vs.cf.T, fF, axes=(1, 0)) + 0.5 * self.F[:, None, None]) / rhoF
            _, U, t = self._tangential(uF)
            if self.turbulent:
                ut = solve_u_tau(self.law, U.ravel(), 1.0 + b.d_w, self.nu).reshape(U.shape)
            else:
                ut = np.zeros_like(U)
            ypB = ut * b.d_w / self.nu
            uB = (ut * self.law.u_plus(ypB))[None] * t if self.turbulent else np.zeros_like(t)
            fB = f[:, :, row, :][:, :, cols]
            cn = vs.c[:, 1] * n_y
            f_par = fB[cn == 0].sum(axis=0)
            f_perp = fB[cn > 0].sum(axis=0)
            rhoB = (f_par + 2.0 * f_perp) / (1.0 + uB[1] * n_y)
            # velocity gradient G[a, g] = d_a u_g at B, previous-step velocity
            G = np.zeros((3, 3) + U.shape)
            yB, yF, yFF = row + 1, F_ + 1, FF + 1        # padded row indices
            for a in (0, 2):                             # tangential: central FD
                for g in range(3):
                    comp = up[g]
                    if a == 0:
                        plus = comp[1:-1, yB, 2:][:, cols]
                        minus = comp[1:-1, yB, :-2][:, cols]
                    else:
                        plus = comp[2:, yB, 1:-1][:, cols]
                        minus = comp[:-2, yB, 1:-1][:, cols]
                    G[a, g] = 0.5 * (plus - minus)
            dup = self.law.dudy_plus(np.where(ypB > 0, ypB, 1.0))
            for g in range(3):
                uBn = up[g][1:-1, yB, 1:-1][:, cols]
                uFn = up[g][1:-1, yF, 1:-1][:, cols]
                uFFn = up[g][1:-1, yFF, 1:-1][:, cols]
                fd = 0.5 * (-3.0 * uBn + 4.0 * uFn - uFFn)          # Eq. 28
                if g != 1 and self.turbulent and cai:
                    dn = self.cai_degrigny_derivative(ut, b.d_w) * t[g]   # Eqs. 29-30
                elif g != 1 and self.turbulent:
                    ana = np.where(ut > 0, ut * ut / self.nu * dup, 0.0) * t[g]   # Eq. 15
                    dn = b.beta * ana + (1.0 - b.beta) * fd               # Eq. 27
                else:
                    dn = fd
                G[1, g] = s * dn
            Sab = 0.5 * (G + G.transpose(1, 0, *range(2, G.ndim)))
            ntB = self.nt[:, row, :][:, cols]
            nutB = SA.nu_t(ntB, self.nu) if self.turbulent else 0.0 * ntB
            tau = 0.5 + (self.nu + nutB) / L.CS2
            feq = L.equilibrium(vs, rhoB, uB)
            qs = np.einsum("iab,ab...->i...", Q, Sab)
            fnew = feq - vs.w[:, None, None] * rhoB * tau / L.CS2 * qs   # Eqs. 19, 26
            for i in range(vs.q):
                cur = f[i][:, row, :]
                cur[:, cols] = fnew[i]
                f[i][:, row, :] = cur
            if self.turbulent:
                tmp = nt_new[:, row, :]
                tmp[:, cols] = self.nu * KAPPA * ypB
                nt_new[:, row, :] = tmp
            full = np.zeros((self.nz, self.nx))
            full[:, cols] = ut
            self.utau[face] = full
        return f

    def collide(self, f, nt_new):
        """Stage 7: moments (Eqs. 4-5), omega (Eq. 8) with nu + nu_t, collision."""
        rho, u = L.moments(self.vs, f, self.F)
        nut = SA.nu_t(nt_new, self.nu) if self.turbulent else np.zeros_like(rho)
        omega = L.omega_from_viscosity(self.nu + nut)
        if self.case.collision == "bgk":
            fs = L.collide_bgk(self.vs, f, rho, u, omega, self.F)
        elif self.case.collision == "regularized":
            fs = L.collide_regularized(self.vs, f, rho, u, omega, self.F)
        else:
            raise ValueError(self.case.collision)
        return fs, rho, u

    # ------------------------------------------------------------------- step
    def step(self):
        nt_new = self.sa_update()
        bb = {face: self.bb_prepass(face, nt_new)
              for face in self.walls if self.bc[face].kind == "wall_bb"}
        f = self.stream()
        f = self.y_faces(f, bb)
        f = self.x_faces(f)
        f = self.hrfd(f, nt_new)
        self.fs, self.rho, self.u = self.collide(f, nt_new)
        self.nt = nt_new
        self.nsteps += 1

    def run(self, nsteps):
        for _ in range(int(nsteps)):
            self.step()
        return self

    # ---------------------------------------------------------------- outputs
    def fields(self):
        """Physical-unit outputs: rho, u, nu_t, nu_tilde; per wall face u_tau and
        C_f = 2 (u_tau / U_ref)^2, arrays [z, x] (zero off the wall columns)."""
        c = self.case
        dxdt = c.dx / self.dt
        nu_scale = c.dx ** 2 / self.dt
        nut = SA.nu_t(self.nt, self.nu) if self.turbulent else np.zeros_like(self.nt)
        out = dict(rho=self.rho * c.rho0, u=self.u * dxdt, nu_t=nut * nu_scale,
                   nu_tilde=self.nt * nu_scale)
        for face, ut in self.utau.items():
            out["u_tau_" + face] = ut * dxdt
            out["cf_" + face] = 2.0 * (ut * dxdt / c.u_ref) ** 2
        return out

    def mass(self):
        return float(self.fs.sum())

    def momentum(self):
        return np.tensordot(self.vs.cf.T, self.fs, axes=(1, 0)).reshape(3, -1).sum(axis=1)
