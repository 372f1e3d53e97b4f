"""Seeded synthetic workloads shaped like the examples of Zhao & Choo (Sec. 5).

This module lays out material points, material fields, boundary masks and load
schedules, and nothing else: it holds no arithmetic of the method (no Lame
conversion, no stabilization parameter, no mass).  Both the CUDA path and the
CPU oracle consume what it returns, so it is the only module they share.

Every workload is synthetic.  The paper's examples use no dataset; the shapes,
sizes and distributions below follow the example set-ups (Terzaghi column,
strip footing, 3D consolidation block) with seeded random fields where the
workload asks for heterogeneity.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

ORIG, GIMP = 0, 1
TAU_WHITE, TAU_SUN, TAU_MONFORTE = 0, 1, 2   # expressions of the PPP parameter (Sec. 4.3)
PERM_CONSTANT, PERM_KOZENY_CARMAN = 0, 1     # permeability model (Eq. kozeny-carman)
P2G_LUMPED, P2G_CONSISTENT = 0, 1             # Stage-1 mapping (Eqs. map-from-particles-to-nodes[-consistent])
MODEL_NEOHOOKE, MODEL_HENCKY = 0, 1           # hyperelastic model of the solid skeleton


@dataclass
class Workload:
    name: str
    dim: int
    shape: int                      # ORIG or GIMP
    ncell: Tuple[int, int, int]
    origin: Tuple[float, float, float]
    h: float
    # material points (input order = caller's particle ids)
    x: np.ndarray                   # (n, d)
    vol: np.ndarray                 # (n,)
    lp: np.ndarray                  # (n, d) GIMP half lengths
    p0: np.ndarray                  # (n,)
    v0: Optional[np.ndarray]        # (n, d) or None
    E: np.ndarray                   # (n,)
    nu: np.ndarray                  # (n,)
    k: np.ndarray                   # (n,) intrinsic permeability, m^2
    surf_id: np.ndarray             # (n,) int32, -1 = interior
    surf_normal: np.ndarray         # (n, d)
    surf_area: np.ndarray           # (n,)
    trac_full: np.ndarray           # (n_surf, d) traction at full load
    # mixture and fluid
    rho_s: float = 2500.0
    rho_f: float = 1000.0
    phi0: float = 0.33
    mu_f: float = 1.0e-3
    alpha_vis: float = 0.0
    g: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    # time integration and stabilization
    dynamic: bool = False
    beta: float = 0.3025
    gamma: float = 0.6
    stabilize: bool = True
    tau_scale: float = 1.0
    tau_kind: int = 0               # TAU_WHITE, TAU_SUN or TAU_MONFORTE (Sec. 4.3)
    permeability: int = 0           # PERM_CONSTANT, or PERM_KOZENY_CARMAN (k = k0 at phi0)
    dt_growth: float = 1.0          # the time step is multiplied by this after each step
    p2g_mass: int = 0               # P2G_LUMPED, or P2G_CONSISTENT (Stage-1 mapping)
    model: int = 0                  # MODEL_NEOHOOKE, or MODEL_HENCKY (Sec. 2.2)
    dt: float = 1.0
    nsteps: int = 1
    ramp_time: float = 0.0          # load scale min(t / ramp_time, 1); 0 = applied at once
    load_omega: float = 0.0         # > 0: harmonic load scale 1 - cos(load_omega t) instead of the ramp
    # Dirichlet data per grid node
    u_fixed: np.ndarray = field(default=None)   # (nnodes, d) uint8
    u_value: np.ndarray = field(default=None)   # (nnodes, d) increment over a step
    p_fixed: np.ndarray = field(default=None)   # (nnodes,) uint8
    p_value: np.ndarray = field(default=None)   # (nnodes,)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_surf(self) -> int:
        return int(self.trac_full.shape[0])

    @property
    def nn(self) -> Tuple[int, ...]:
        return tuple(self.ncell[k] + 1 for k in range(self.dim))

    @property
    def nnodes(self) -> int:
        return int(np.prod(self.nn))

    def load_scale(self, t: float) -> float:
        if self.load_omega > 0.0:
            return 1.0 - float(np.cos(self.load_omega * t))
        if self.ramp_time <= 0.0:
            return 1.0
        return min(t / self.ramp_time, 1.0)

    def traction(self, t: float) -> np.ndarray:
        return np.ascontiguousarray(self.load_scale(t) * self.trac_full)

    def step_sizes(self, nsteps: int):
        """dt of steps 0 .. nsteps-1: dt, then multiplied by dt_growth after each step."""
        return [self.dt * self.dt_growth ** i for i in range(nsteps)]


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------
def lattice(dim, body_cells, h, ppc_axis, origin=(0.0, 0.0, 0.0), cell_offset=(0, 0, 0)):
    """Material points at the regular sub-cell centres of `body_cells` cells."""
    axes = []
    for k in range(dim):
        c = np.arange(cell_offset[k], cell_offset[k] + body_cells[k])
        s = (np.arange(ppc_axis) + 0.5) / ppc_axis
        axes.append(((c[:, None] + s[None, :]).reshape(-1)) * h + origin[k])
    mesh = np.meshgrid(*axes, indexing="ij")
    # Fortran order: x index fastest, then y, then z
    x = np.stack([m.reshape(-1, order="F") for m in mesh], axis=1)
    n = x.shape[0]
    vol = np.full(n, h ** dim / ppc_axis ** dim)
    lp = np.full((n, dim), 0.5 * h / ppc_axis)
    return np.ascontiguousarray(x), vol, lp


def node_coords(dim, ncell):
    nn = [ncell[k] + 1 for k in range(dim)]
    idx = np.indices(nn[::-1]).reshape(dim, -1)[::-1]  # idx[0] fastest
    return idx.T  # (nnodes, dim) integer node coordinates


def empty_bcs(dim, ncell):
    nnodes = int(np.prod([ncell[k] + 1 for k in range(dim)]))
    return (np.zeros((nnodes, dim), np.uint8), np.zeros((nnodes, dim)),
            np.zeros(nnodes, np.uint8), np.zeros(nnodes))


def _surface(x, top_axis, top_value, h, ppc_axis, select):
    """Top-row material points (upper sub-row) for which select(x) holds."""
    y = x[:, top_axis]
    top = np.abs(y - (top_value - 0.5 * h / ppc_axis)) < 1e-9 * max(1.0, abs(top_value))
    return np.nonzero(top & select(x))[0]


def _finish(dim, x, surf_idx, normal_axis, area, trac_vec):
    n = x.shape[0]
    surf_id = np.full(n, -1, np.int32)
    surf_id[surf_idx] = np.arange(len(surf_idx), dtype=np.int32)
    surf_normal = np.zeros((n, dim))
    surf_normal[surf_idx, normal_axis] = 1.0
    surf_area = np.zeros(n)
    surf_area[surf_idx] = area
    trac = np.tile(np.asarray(trac_vec, float)[None, :dim], (len(surf_idx), 1))
    return surf_id, surf_normal, surf_area, np.ascontiguousarray(trac)


def _perm(rng, n):
    return rng.permutation(n) if rng is not None else np.arange(n)


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
def terzaghi_column(ncell_y=40, ncell_x=4, h=0.25, E=10e6, nu=0.3, k=1e-10, mu_f=1e-3,
                    load=10e3, dt=1.0, nsteps=10, ppc_axis=(2, 2), stabilize=True,
                    tau_scale=1.0, shape=ORIG, name="terzaghi-4x40"):
    """2D plane-strain consolidation column (Sec. 5.1 set-up): drained loaded top,
    impermeable rollers on the sides, fixed impermeable bottom, no gravity."""
    dim = 2
    ncell = (ncell_x, ncell_y, 0)
    px, py = ppc_axis
    axes = [((np.arange(ncell_x)[:, None] + (np.arange(px) + 0.5)[None, :] / px).reshape(-1)) * h,
            ((np.arange(ncell_y)[:, None] + (np.arange(py) + 0.5)[None, :] / py).reshape(-1)) * h]
    X, Y = np.meshgrid(axes[0], axes[1], indexing="xy")
    x = np.ascontiguousarray(np.stack([X.reshape(-1), Y.reshape(-1)], axis=1))
    n = x.shape[0]
    vol = np.full(n, h * h / (px * py))
    lp = np.ascontiguousarray(np.tile([0.5 * h / px, 0.5 * h / py], (n, 1)))
    H = ncell_y * h
    top = np.nonzero(np.abs(x[:, 1] - (H - 0.5 * h / py)) < 1e-9 * H)[0]
    surf_id, surf_normal, surf_area, trac = _finish(dim, x, top, 1, h / px, (0.0, -load))
    uf, uv, pf, pv = empty_bcs(dim, ncell)
    nc = node_coords(dim, ncell)
    uf[nc[:, 0] == 0, 0] = 1
    uf[nc[:, 0] == ncell_x, 0] = 1
    uf[nc[:, 1] == 0, :] = 1
    pf[nc[:, 1] == ncell_y] = 1
    return Workload(name=name, dim=dim, shape=shape, ncell=ncell, origin=(0.0, 0.0, 0.0), h=h,
                    x=x, vol=vol, lp=lp, p0=np.zeros(n), v0=None,
                    E=np.full(n, E), nu=np.full(n, nu), k=np.full(n, k),
                    surf_id=surf_id, surf_normal=surf_normal, surf_area=surf_area, trac_full=trac,
                    mu_f=mu_f, dynamic=False, stabilize=stabilize, tau_scale=tau_scale,
                    dt=dt, nsteps=nsteps, u_fixed=uf, u_value=uv, p_fixed=pf, p_value=pv)


def paper_terzaghi(n_elem=40, stabilize=True, tau_scale=1.0, shape=ORIG):
    """Sec. 5.1 verification column: K = 1 MPa, nu = 0.25, c_v = 1.8e-5 m^2/s,
    H = 1 m, w = 1 kPa, dt = 0.1 s, one step, 2 material points per element
    (one column of elements, points stacked vertically)."""
    K, nu = 1.0e6, 0.25
    G = 3.0 * K * (1.0 - 2.0 * nu) / (2.0 * (1.0 + nu))
    E = 2.0 * G * (1.0 + nu)
    M = K + 4.0 * G / 3.0
    mu_f = 1.0e-3
    k = 1.8e-5 / M * mu_f          # c_v = M k / mu_f
    h = 1.0 / n_elem
    return terzaghi_column(ncell_y=n_elem, ncell_x=1, h=h, E=E, nu=nu, k=k, mu_f=mu_f,
                           load=1.0e3, dt=0.1, nsteps=1, ppc_axis=(1, 2), stabilize=stabilize,
                           tau_scale=tau_scale, shape=shape, name=f"paper-terzaghi-{n_elem}")


def self_weight_consolidation(ncell=(16, 16), h=0.125, ppc_axis=5, K=15e3, nu=0.3, k0=1e-14, phi0=0.5,
                              mu_f=1e-3, rho_s=2600.0, rho_f=1000.0, g=9.81, dt=0.1, dt_growth=1.2,
                              nsteps=20, shape=ORIG, stabilize=True, name=None):
    """Self-weight consolidation (Sec. 5.3 set-up): the right half of a soft
    deposit 4 m wide and 2 m tall (here ncell * h), K = 15 kPa, nu = 0.3,
    k0 = 1e-14 m^2 with the permeability following the porosity (Eq.
    kozeny-carman, phi0 = 0.5), mu_f = 1e-6 kPa s, rho_s = 2.6, rho_f = 1.0 Mg/m^3,
    quasi-static; gravity applied at t = 0 on a stress-free, pressure-free
    state; dt = 0.1 s multiplied by 1.2 after each step; the paper's two grids
    are h = 0.125 m with 25 points per cell and h = 0.0625 m with 16.  Drained
    (p = 0) top and right side, rigid impermeable bottom, the symmetry plane a
    roller.  The right side is read as a roller too (the paper fixes its
    pressure only; a free side would let the deposit spread out of the
    modelled domain)."""
    dim = 2
    nc = (int(ncell[0]), int(ncell[1]), 0)
    x, vol, lp = lattice(dim, nc[:2], h, ppc_axis)
    n = x.shape[0]
    G = 3.0 * K * (1.0 - 2.0 * nu) / (2.0 * (1.0 + nu))
    E = 2.0 * G * (1.0 + nu)
    uf, uv, pf, pv = empty_bcs(dim, nc)
    nco = node_coords(dim, nc)
    uf[nco[:, 0] == 0, 0] = 1              # symmetry plane
    uf[nco[:, 0] == nc[0], 0] = 1          # right side (roller)
    uf[nco[:, 1] == 0, :] = 1              # rigid bottom
    pf[(nco[:, 1] == nc[1]) | (nco[:, 0] == nc[0])] = 1   # drained top and right side
    return Workload(name=name or f"self-weight-{nc[0]}x{nc[1]}", dim=dim, shape=shape, ncell=nc,
                    origin=(0.0, 0.0, 0.0), h=h, x=x, vol=vol, lp=lp, p0=np.zeros(n), v0=None,
                    E=np.full(n, E), nu=np.full(n, nu), k=np.full(n, k0),
                    surf_id=np.full(n, -1, np.int32), surf_normal=np.zeros((n, dim)),
                    surf_area=np.zeros(n), trac_full=np.zeros((0, dim)),
                    rho_s=rho_s, rho_f=rho_f, phi0=phi0, mu_f=mu_f, g=(0.0, -g, 0.0),
                    dynamic=False, stabilize=stabilize, dt=dt, nsteps=nsteps, dt_growth=dt_growth,
                    permeability=PERM_KOZENY_CARMAN,
                    u_fixed=uf, u_value=uv, p_fixed=pf, p_value=pv)


def strip_footing(body=(200, 100), pad=2, h=0.1, seed=2, ppc_axis=2, E0=20e6, nu=0.3, k=1e-14,
                  w_max=200e3, ramp=0.1, dt=1e-3, nsteps=200, half_width=1.0,
                  shape=GIMP, dynamic=True, alpha_vis=0.04, name=None):
    """2D plane-strain dynamic strip footing (Sec. 5.2 shape): a block with empty
    padding rows above the surface, a rigid strip of half width 1 m at the top
    centre loaded by a linear ramp, drained top outside the strip, fixed bottom,
    rollers on the sides; lognormal stiffness field E = E0 exp(0.05 Z)."""
    rng = np.random.default_rng(seed)
    dim = 2
    ncell = (body[0], body[1] + pad, 0)
    x, vol, lp = lattice(dim, body, h, ppc_axis)
    n = x.shape[0]
    E = E0 * np.exp(0.05 * rng.standard_normal(n))
    W, H = body[0] * h, body[1] * h
    xc = 0.5 * W
    top = _surface(x, 1, H, h, ppc_axis, lambda q: np.abs(q[:, 0] - xc) <= half_width + 1e-12)
    surf_id, surf_normal, surf_area, trac = _finish(dim, x, top, 1, h / ppc_axis, (0.0, -w_max))
    uf, uv, pf, pv = empty_bcs(dim, ncell)
    nc = node_coords(dim, ncell)
    uf[nc[:, 1] == 0, :] = 1
    uf[nc[:, 0] == 0, 0] = 1
    uf[nc[:, 0] == ncell[0], 0] = 1
    strip = int(round(half_width / h))
    mid = body[0] // 2
    drained = (nc[:, 1] == body[1]) & ((nc[:, 0] < mid - strip) | (nc[:, 0] > mid + strip))
    pf[drained] = 1
    return Workload(name=name or f"footing-{body[0]}x{body[1]}", dim=dim, shape=shape, ncell=ncell,
                    origin=(0.0, 0.0, 0.0), h=h, x=x, vol=vol, lp=lp, p0=np.zeros(n),
                    v0=np.zeros((n, dim)), E=E, nu=np.full(n, nu), k=np.full(n, k),
                    surf_id=surf_id, surf_normal=surf_normal, surf_area=surf_area, trac_full=trac,
                    alpha_vis=alpha_vis if dynamic else 0.0, dynamic=dynamic, dt=dt,
                    nsteps=nsteps, ramp_time=ramp, u_fixed=uf, u_value=uv, p_fixed=pf, p_value=pv)


def consolidation_block(body=(64, 64, 32), pad=1, h=0.1, seed=3, ppc_axis=2, E=10e6, nu=0.3,
                        logk=(-13.0, -11.0), load=50e3, patch_half=1.0, dt=5.0, nsteps=20,
                        shape=GIMP, name=None):
    """3D quasi-static consolidation block: per-point permeability log-uniform,
    surface load on a central square patch, drained top, fixed bottom, rollers."""
    rng = np.random.default_rng(seed)
    dim = 3
    ncell = (body[0], body[1], body[2] + pad)
    x, vol, lp = lattice(dim, body, h, ppc_axis)
    n = x.shape[0]
    k = 10.0 ** rng.uniform(logk[0], logk[1], n)
    cx, cy, H = 0.5 * body[0] * h, 0.5 * body[1] * h, body[2] * h
    top = _surface(x, 2, H, h, ppc_axis,
                   lambda q: (np.abs(q[:, 0] - cx) <= patch_half + 1e-12)
                   & (np.abs(q[:, 1] - cy) <= patch_half + 1e-12))
    surf_id, surf_normal, surf_area, trac = _finish(dim, x, top, 2, (h / ppc_axis) ** 2,
                                                    (0.0, 0.0, -load))
    uf, uv, pf, pv = empty_bcs(dim, ncell)
    nc = node_coords(dim, ncell)
    uf[nc[:, 2] == 0, :] = 1
    uf[(nc[:, 0] == 0) | (nc[:, 0] == ncell[0]), 0] = 1
    uf[(nc[:, 1] == 0) | (nc[:, 1] == ncell[1]), 1] = 1
    pf[nc[:, 2] == body[2]] = 1
    return Workload(name=name or "block-{}x{}x{}".format(*body), dim=dim, shape=shape,
                    ncell=ncell, origin=(0.0, 0.0, 0.0), h=h, x=x, vol=vol, lp=lp,
                    p0=np.zeros(n), v0=None, E=np.full(n, E), nu=np.full(n, nu), k=k,
                    surf_id=surf_id, surf_normal=surf_normal, surf_area=surf_area,
                    trac_full=trac, dynamic=False, dt=dt, nsteps=nsteps,
                    u_fixed=uf, u_value=uv, p_fixed=pf, p_value=pv)


def slope_3d(ncell=(128, 128, 64), h=0.1, ppc_axis=2, E=5e6, nu=0.35, k=1e-12, slope_deg=30.0,
             z_toe=1.2, z_crest=5.2, x_toe=2.9, water_table=None, dt=10.0, nsteps=100,
             shape=GIMP, name=None):
    """3D slope under gravity: the cells whose centre lies below the ground
    surface z(x) = z_toe + tan(slope) (x - x_toe), clipped to [z_toe, z_crest]
    (a 30 degree slope between a toe and a crest plateau, about half of a
    128 x 128 x 64 box at 0.1 m: 4.2M points at 2^3 per cell); gravity from
    t = 0 on a stress-free skeleton with a hydrostatic pore pressure below the
    water table (default mid-height of the box); the ground surface drained to
    the water table's level, p = max(rho_f g (z_w - z), 0); fixed bottom,
    rollers on the four sides (impermeable)."""
    dim = 3
    nc = (int(ncell[0]), int(ncell[1]), int(ncell[2]))
    zw = 0.5 * nc[2] * h if water_table is None else water_table
    tan = np.tan(np.deg2rad(slope_deg))
    xc = (np.arange(nc[0]) + 0.5) * h
    zsurf = np.clip(z_toe + tan * (xc - x_toe), z_toe, z_crest)          # per column of cells
    ncol = np.floor(zsurf / h + 0.5).astype(int)                         # filled cells per column
    filled = np.zeros((nc[0], nc[2]), bool)                              # [x cell][z cell]
    for i in range(nc[0]):
        filled[i, :ncol[i]] = True
    x, vol, lp = lattice(dim, nc, h, ppc_axis)
    ci = np.minimum((x[:, 0] / h).astype(int), nc[0] - 1)
    ck = np.minimum((x[:, 2] / h).astype(int), nc[2] - 1)
    keep = filled[ci, ck]
    x, vol, lp = np.ascontiguousarray(x[keep]), vol[keep], np.ascontiguousarray(lp[keep])
    n = x.shape[0]
    rho_f, g = 1000.0, 9.81
    p0 = np.maximum(rho_f * g * (zw - x[:, 2]), 0.0)
    uf, uv, pf, pv = empty_bcs(dim, nc)
    nco = node_coords(dim, nc)
    uf[nco[:, 2] == 0, :] = 1
    uf[(nco[:, 0] == 0) | (nco[:, 0] == nc[0]), 0] = 1
    uf[(nco[:, 1] == 0) | (nco[:, 1] == nc[1]), 1] = 1
    # ground-surface nodes: a filled and an empty cell among the cells around the node (x-z plane)
    ix, iz = nco[:, 0], nco[:, 2]
    any_f = np.zeros(len(nco), bool)
    any_e = np.zeros(len(nco), bool)
    for dx in (-1, 0):
        for dz in (-1, 0):
            cxi, czi = ix + dx, iz + dz
            ok = (cxi >= 0) & (cxi < nc[0]) & (czi >= 0) & (czi < nc[2])
            f = np.zeros(len(nco), bool)
            f[ok] = filled[cxi[ok], czi[ok]]
            any_f |= f
            any_e |= ok & ~f
    surf = any_f & any_e & (iz > 0)
    pf[surf] = 1
    pv[surf] = np.maximum(rho_f * g * (zw - iz[surf] * h), 0.0)
    return Workload(name=name or "slope-{}x{}x{}".format(*nc), dim=dim, shape=shape, ncell=nc,
                    origin=(0.0, 0.0, 0.0), h=h, x=x, vol=vol, lp=lp, p0=p0, v0=None,
                    E=np.full(n, E), nu=np.full(n, nu), k=np.full(n, k),
                    surf_id=np.full(n, -1, np.int32), surf_normal=np.zeros((n, dim)),
                    surf_area=np.zeros(n), trac_full=np.zeros((0, dim)),
                    rho_f=rho_f, g=(0.0, 0.0, -g), dynamic=False, dt=dt, nsteps=nsteps,
                    u_fixed=uf, u_value=uv, p_fixed=pf, p_value=pv)


def jittered(w: Workload, seed: int, frac: float = 0.15, shuffle: bool = True,
             E_spread: float = 0.2, logk_spread: float = 1.0) -> Workload:
    """A copy of `w` whose points are displaced by up to `frac` of their spacing
    (so GIMP domains straddle cell faces), whose E and k are perturbed, and whose
    input order is shuffled: the parity workloads."""
    rng = np.random.default_rng(seed)
    n, d = w.x.shape
    spacing = 2.0 * w.lp
    x = w.x + frac * spacing * rng.uniform(-1.0, 1.0, (n, d))
    E = w.E * np.exp(E_spread * rng.standard_normal(n))
    k = w.k * 10.0 ** (logk_spread * rng.uniform(-1.0, 1.0, n))
    p0 = 1e3 * rng.standard_normal(n)
    perm = _perm(rng, n) if shuffle else np.arange(n)
    surf_id = w.surf_id[perm]

    def take(a):
        return None if a is None else np.ascontiguousarray(a[perm])

    v0 = None if w.v0 is None else np.ascontiguousarray(0.01 * rng.standard_normal((n, d)))
    return replace(w, name=w.name + f"-jit{seed}", x=take(x), vol=take(w.vol), lp=take(w.lp),
                   p0=take(p0), v0=take(v0) if v0 is not None else None, E=take(E), nu=take(w.nu),
                   k=take(k), surf_id=np.ascontiguousarray(surf_id),
                   surf_normal=take(w.surf_normal), surf_area=take(w.surf_area))


def harmonic_footing(body=(40, 40), pad=4, h=0.25, ppc_axis=2, lam=8.4e6, G=5.6e6, k=1e-14,
                     w_amp=3e6, omega=100.0, half_width=1.0, dt=1e-3, nsteps=400, alpha_vis=0.04,
                     shape=GIMP, model=MODEL_HENCKY, p2g_mass=P2G_CONSISTENT, name=None):
    """Strip footing under harmonic loading (Sec. 5.2 set-up): the right half of a
    20 m wide, 10 m deep saturated ground (symmetry plane at x = 0), 1,600
    cells of h = 0.25 m with 4 points each and 160 empty cells above the
    surface; a 2 m wide footing at the top centre (here 0 <= x <= 1 m) loaded by
    w = 3 - 3 cos(100 t) MPa, impermeable, the rest of the top drained; bottom
    fixed, the symmetry plane and the far side rollers, all impermeable but the
    top.  lambda = 8.4 MPa, G = 5.6 MPa (Hencky), k = 1e-14 m^2, alpha_vis = 0.04,
    mu_f = 1e-3 Pa s, rho_s = 2500, rho_f = 1000 kg/m^3, phi0 = 0.33; Newmark,
    dt = 1e-3 s to t = 0.4 s, consistent-mass mapping (the paper's choice for
    this cyclic load)."""
    dim = 2
    ncell = (body[0], body[1] + pad, 0)
    x, vol, lp = lattice(dim, body, h, ppc_axis)
    n = x.shape[0]
    nu = lam / (2.0 * (lam + G))
    E = 2.0 * G * (1.0 + nu)
    H = body[1] * h
    top = _surface(x, 1, H, h, ppc_axis, lambda q: q[:, 0] <= half_width + 1e-12)
    surf_id, surf_normal, surf_area, trac = _finish(dim, x, top, 1, h / ppc_axis, (0.0, -w_amp))
    uf, uv, pf, pv = empty_bcs(dim, ncell)
    nc = node_coords(dim, ncell)
    uf[nc[:, 1] == 0, :] = 1
    uf[nc[:, 0] == 0, 0] = 1
    uf[nc[:, 0] == ncell[0], 0] = 1
    strip = int(round(half_width / h))
    pf[(nc[:, 1] == body[1]) & (nc[:, 0] > strip)] = 1
    return Workload(name=name or f"harmonic-footing-{body[0]}x{body[1]}", dim=dim, shape=shape,
                    ncell=ncell, origin=(0.0, 0.0, 0.0), h=h, x=x, vol=vol, lp=lp, p0=np.zeros(n),
                    v0=np.zeros((n, dim)), E=np.full(n, E), nu=np.full(n, nu), k=np.full(n, k),
                    surf_id=surf_id, surf_normal=surf_normal, surf_area=surf_area, trac_full=trac,
                    rho_s=2500.0, rho_f=1000.0, phi0=0.33, mu_f=1e-3, alpha_vis=alpha_vis,
                    dynamic=True, dt=dt, nsteps=nsteps, load_omega=omega, model=model,
                    p2g_mass=p2g_mass, u_fixed=uf, u_value=uv, p_fixed=pf, p_value=pv)


def small_footing(seed=7, shape=GIMP, dynamic=True, body=(24, 12), pad=2, h=0.25, dt=2e-3,
                  k=1e-12, jitter=0.15):
    """A footing a few tiles wide with jittered, shuffled points: parity case."""
    w = strip_footing(body=body, pad=pad, h=h, seed=seed, k=k, w_max=100e3, ramp=4 * dt, dt=dt,
                      nsteps=4, half_width=1.0, shape=shape, dynamic=dynamic,
                      alpha_vis=0.04 if dynamic else 0.0, name=f"small-footing-{body[0]}x{body[1]}")
    return jittered(w, seed + 100, frac=jitter) if jitter > 0 else w


def small_block(seed=11, shape=GIMP, body=(6, 5, 4), pad=1, h=0.25, dt=1.0, jitter=0.15):
    w = consolidation_block(body=body, pad=pad, h=h, seed=seed, patch_half=0.25, dt=dt, nsteps=3,
                            shape=shape, name="small-block-{}x{}x{}".format(*body))
    return jittered(w, seed + 100, frac=jitter) if jitter > 0 else w


CONFIGS = {
    "terzaghi": lambda: terzaghi_column(),
    "footing": lambda: strip_footing(),
    "block3d": lambda: consolidation_block(),
}


def batch_instances(count=256, seed=5, kind="alternate", h=0.1, nx=(16, 128), ny=(32, 64),
                    logk=(-15.0, -10.0), load=(10e3, 200e3)):
    """Independent 2D instances of uneven size for batched stepping: grid
    nx x ny cells drawn uniformly from the ranges, 2 x 2 points per cell,
    permeability 10^U(logk), load U(load).  kind: "terzaghi" (consolidation
    under a uniform top load: original MPM, quasi-static, dt = 1 s),
    "footing" (strip load of half width min(1 m, W/4): GIMP, Newmark,
    dt = 1e-3 s, ramp 0.1 s) or "alternate" (even i Terzaghi, odd i footing)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        cx = int(rng.integers(nx[0], nx[1] + 1))
        cy = int(rng.integers(ny[0], ny[1] + 1))
        k = float(10.0 ** rng.uniform(logk[0], logk[1]))
        w = float(rng.uniform(load[0], load[1]))
        kd = kind if kind != "alternate" else ("terzaghi" if i % 2 == 0 else "footing")
        if kd == "terzaghi":
            out.append(terzaghi_column(ncell_y=cy, ncell_x=cx, h=h, k=k, load=w, dt=1.0, nsteps=20,
                                       ppc_axis=(2, 2), shape=ORIG, name=f"terzaghi-{i}-{cx}x{cy}"))
        else:
            out.append(strip_footing(body=(cx, cy), pad=2, h=h, seed=seed * 100003 + i, k=k, w_max=w,
                                     ramp=0.1, dt=1e-3, nsteps=20,
                                     half_width=min(1.0, 0.25 * cx * h), name=f"footing-{i}-{cx}x{cy}"))
    return out
