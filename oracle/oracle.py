"""CPU FP64 oracle of the stabilized implicit u-p MPM step (Zhao & Choo).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import this module; the product path never
does.  It shares no code with the CUDA path: the particle and grid loops are in
oracle/upmpm_oracle.c (built here with gcc), the Newton loop, the Dirichlet
elimination and the linear solve are below.  The linear solve is a direct
sparse LU (scipy SuperLU) of the row/column-equilibrated Jacobian: a library
primitive standing in for "solve J dX = -R".

One load step follows the four stages of Sec. 3.1:
  1. map point state to the nodes (Eq. map-from-particles-to-nodes),
  2. Newton on the discrete equations (Eq. newton-tolerance, Eq.
     jacobian-system-stabilized-ppp) with unknowns [dU, P] per node,
  3./4. update the points from the nodes, convect them, update the GIMP
     domains (Sec. 3.5).

The dynamic terms whose linearization the paper leaves out (Kelvin damping
geometry, Darcy acceleration) are pinned through eval_frozen: the Jacobian
matches central differences of the residual with exactly those terms frozen.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libupmpm_oracle.so")
MAXS = 4

OK, ERR_BAD_ARG, ERR_OUT_OF_GRID, ERR_NEGATIVE_J = 0, -1, -2, -3


TAU_WHITE, TAU_SUN, TAU_MONFORTE = 0, 1, 2   # expressions of the PPP parameter, Sec. 4.3
P2G_LUMPED, P2G_CONSISTENT = 0, 1             # Stage-1 mapping, Eqs. map-from-particles-to-nodes(-consistent)
MODEL_NEOHOOKE, MODEL_HENCKY = 0, 1           # hyperelastic model of the solid skeleton
PERM_CONSTANT, PERM_KOZENY_CARMAN = 0, 1     # permeability model, Eq. kozeny-carman


def kozeny_carman(k0, phi0, J):
    """Eq. kozeny-carman with the porosity of incompressible constituents,
    phi = 1 - (1 - phi0) / J: k = k0 (1 - phi0)^2 / phi0^3 * phi^3 / (1 - phi)^2;
    zero once the pores are closed (phi <= 0)."""
    phi = 1.0 - (1.0 - phi0) / np.asarray(J, float)
    k = k0 * ((1.0 - phi0) ** 2 / phi0 ** 3) * (phi ** 3 / (1.0 - phi) ** 2)
    return np.where(phi > 0.0, k, 0.0)


def stabilization_parameter(w, lam, G, kappa, dt):
    """PPP parameter tau per point for a step of length dt (Sec. 4.3), times
    w.tau_scale; zero when unstabilized.  With the P-wave modulus M = K + 4G/3
    = lambda + 2G and the consolidation coefficient c_v = M kappa:
      tau_W = 1 / (2 G)                                          (Eq. tau-white)
      tau_S = (1/M) (1 - 3 c_v dt/h^2) [1 + tanh(2 - 12 c_v dt/h^2)]  (Eq. tau-sun)
      tau_M = max(2 kappa/c_v - (beta/gamma) 12 kappa dt/h^2, 0)    (Eq. tau-monforte)
    with 2 kappa / c_v evaluated as 2 / M (equal for kappa > 0, its limit at
    kappa = 0).  tau_M uses the Newmark parameters: dynamic problems only."""
    n = len(G)
    if not w.stabilize:
        return np.zeros(n)
    if w.tau_kind == TAU_WHITE:
        return w.tau_scale / (2.0 * G)
    M = lam + 2.0 * G
    h = w.h
    if w.tau_kind == TAU_SUN:
        cv = M * kappa
        r = cv * dt / (h * h)
        return w.tau_scale * ((1.0 - 3.0 * r) * (1.0 + np.tanh(2.0 - 12.0 * r)) / M)
    if w.tau_kind == TAU_MONFORTE:
        if not w.dynamic:
            raise ValueError("tau_M (Eq. tau-monforte) uses the Newmark parameters: dynamic steps only")
        return w.tau_scale * np.maximum(2.0 / M - (w.beta / w.gamma) * (12.0 * kappa * dt / (h * h)), 0.0)
    raise ValueError(f"unknown tau_kind {w.tau_kind}")


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle's C loops with the host compiler (plain -O2, IEEE
    arithmetic, no FMA contraction)."""
    src = os.path.join(_HERE, "upmpm_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("shape", C.c_int32), ("ncell", C.c_int32 * 3),
                ("origin", C.c_double * 3), ("h", C.c_double)]


class _Particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("lp", C.c_void_p), ("F", C.c_void_p),
                ("V", C.c_void_p), ("m", C.c_void_p), ("lam", C.c_void_p), ("G", C.c_void_p),
                ("kappa", C.c_void_p), ("tau", C.c_void_p), ("surf", C.c_void_p),
                ("surf_n", C.c_void_p), ("surf_A", C.c_void_p)]


class _Step(C.Structure):
    _fields_ = [("dt", C.c_double), ("dynamic", C.c_int32), ("beta", C.c_double),
                ("gamma", C.c_double), ("rho_f", C.c_double), ("alpha_vis", C.c_double),
                ("g", C.c_double * 3), ("kozeny", C.c_int32), ("phi0", C.c_double),
                ("hencky", C.c_int32)]


class _Nodal(C.Structure):
    _fields_ = [("P", C.c_void_p), ("v", C.c_void_p), ("a", C.c_void_p), ("pd", C.c_void_p),
                ("pdd", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_pattern.restype = C.c_int64
        _lib.orc_nnodes.restype = C.c_int64
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != OK:
        names = {ERR_BAD_ARG: "bad argument", ERR_OUT_OF_GRID: "material point out of grid",
                 ERR_NEGATIVE_J: "non-positive Jacobian"}
        raise OracleError(f"{what}: {names.get(rc, rc)}")


def grid_struct(dim, shape, ncell, origin, h):
    g = _Grid()
    g.dim, g.shape = dim, shape
    for k in range(3):
        g.ncell[k] = int(ncell[k]) if k < len(ncell) else 0
        g.origin[k] = float(origin[k]) if k < len(origin) else 0.0
    g.h = float(h)
    return g


# ---------------------------------------------------------------------------
# thin wrappers over the C loops
# ---------------------------------------------------------------------------
def shape_1d(shape, dx, lp, h, ncell):
    first, count = C.c_int32(), C.c_int32()
    S, dS, S0 = (np.zeros(MAXS) for _ in range(3))
    rc = lib().orc_shape_1d(C.c_int32(shape), C.c_double(dx), C.c_double(lp), C.c_double(h),
                            C.c_int32(ncell), C.byref(first), C.byref(count), _p(S), _p(dS), _p(S0))
    _check(rc, "shape_1d")
    c = count.value
    return first.value, S[:c].copy(), dS[:c].copy(), S0[:c].copy()


def shape(g, x, lp):
    n = x.shape[0]
    first = np.zeros((n, 3), np.int32)
    count = np.zeros((n, 3), np.int32)
    S, dS, S0 = (np.zeros((n, 3, MAXS)) for _ in range(3))
    _check(lib().orc_shape(C.byref(g), C.c_int64(n), _p(x), _p(lp), _p(first), _p(count),
                           _p(S), _p(dS), _p(S0)), "shape")
    return first, count, S, dS, S0


def binning(g, x):
    n = x.shape[0]
    cell = np.zeros(n, np.int32)
    order = np.zeros(n, np.int64)
    _check(lib().orc_bin(C.byref(g), C.c_int64(n), _p(x), _p(cell), _p(order)), "bin")
    return cell, order


def pattern(g, first, count):
    n = first.shape[0]
    nn = lib().orc_nnodes(C.byref(g))
    row_ptr = np.zeros(nn + 1, np.int64)
    nnz = lib().orc_pattern(C.byref(g), C.c_int64(n), _p(first), _p(count), _p(row_ptr), None,
                            C.c_int64(0))
    col = np.zeros(max(nnz, 1), np.int32)
    nnz2 = lib().orc_pattern(C.byref(g), C.c_int64(n), _p(first), _p(count), _p(row_ptr),
                             _p(col), C.c_int64(nnz))
    if nnz2 != nnz:
        raise OracleError("pattern size changed")
    return row_ptr, col[:nnz]


def point_basis(g, p, first, count, S, dS, S0, active=None):
    """Basis of point p as the residual and the update use it (reading R7):
    node ids of its support box, S, the t_n gradient (nodes x d) and S0, with
    inactive nodes removed and the rest renormalised."""
    d = g.dim
    cap = MAXS ** d
    node = np.zeros(cap, np.int64)
    Sv, S0v = np.zeros(cap), np.zeros(cap)
    Gv = np.zeros(cap * d)
    act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    ns = lib().orc_point_basis(C.byref(g), C.c_int64(p), _p(first), _p(count), _p(S), _p(dS),
                               _p(S0), _p(act), _p(node), _p(Sv), _p(Gv), _p(S0v))
    if ns < 0:
        _check(ns, "point_basis")
    return node[:ns].copy(), Sv[:ns].copy(), Gv[:ns * d].reshape(ns, d).copy(), S0v[:ns].copy()


def p2g(g, first, count, S, m, fld):
    n = first.shape[0]
    nn = lib().orc_nnodes(C.byref(g))
    fld = np.ascontiguousarray(fld, dtype=np.float64).reshape(n, -1)
    nf = fld.shape[1]
    M = np.zeros(nn)
    out = np.zeros((nn, nf))
    _check(lib().orc_p2g(C.byref(g), C.c_int64(n), _p(first), _p(count), _p(S), _p(m),
                         C.c_int32(nf), _p(fld), _p(M), _p(out)), "p2g")
    return M, out


def consistent_map(g, first, count, S, m, M, active, lumped, row_ptr, col):
    """Eq. map-from-particles-to-nodes-consistent: sum_j M_ij f_j = sum_mp S_i m f
    with the consistent mass M_ij = sum_mp S_i S_j m, solved for the active
    nodes; the other nodes keep the values of the lumped mapping (Eq.
    map-from-particles-to-nodes), their couplings moved to the right-hand
    side, whose point sum is taken as M_i f_i of the lumped mapping.  (The
    consistent mass of nodes that a GIMP domain barely reaches is singular;
    the active set is the one of the Newton system.)  Solved directly."""
    nn = M.shape[0]
    mc = np.zeros(len(col))
    _check(lib().orc_consistent_mass(C.byref(g), C.c_int64(first.shape[0]), _p(first), _p(count), _p(S),
                                     _p(np.ascontiguousarray(m)), _p(row_ptr), _p(col), _p(mc)),
           "consistent mass")
    A = sps.csr_matrix((mc, col, row_ptr), shape=(nn, nn))
    ia = np.nonzero(active)[0]
    ii = np.nonzero(~active)[0]
    rhs = (M[:, None] * lumped)[ia] - A[ia][:, ii] @ lumped[ii]
    out = lumped.copy()
    out[ia] = spla.splu(A[ia][:, ia].tocsc()).solve(np.ascontiguousarray(rhs)).reshape(len(ia), -1)
    return out


# ---------------------------------------------------------------------------
# material constants from (E, nu), mixture mass (taken by each side itself)
# ---------------------------------------------------------------------------
def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    G = E / (2.0 * (1.0 + nu))
    return lam, G


def det(F, d):
    F = F.reshape(-1, d, d)
    return np.linalg.det(F)


@dataclass
class StepInfo:
    newton_iters: int
    res_hist: list


class Oracle:
    """State of one problem, stepped on the CPU in FP64."""

    def __init__(self, w, newton_rtol=1e-8, newton_max=25, newton_stag=0.0,
                 min_volume_fraction=1e-4):
        self.w = w
        d = w.dim
        self.d = d
        self.g = grid_struct(d, w.shape, w.ncell, w.origin, w.h)
        n = w.n
        self.n = n
        self.x = np.ascontiguousarray(w.x, dtype=np.float64).copy()
        self.u = np.zeros((n, d))
        self.F = np.tile(np.eye(d).reshape(1, d * d), (n, 1)).copy()
        self.V = np.asarray(w.vol, float).copy()
        self.V0 = self.V.copy()
        self.lp = np.ascontiguousarray(w.lp, float).copy()
        self.lp0 = self.lp.copy()
        self.p = np.asarray(w.p0, float).copy()
        self.v = np.zeros((n, d)) if w.v0 is None else np.asarray(w.v0, float).copy()
        self.a = np.zeros((n, d))
        self.pd = np.zeros(n)
        self.pdd = np.zeros(n)
        self.lam, self.G = lame(np.asarray(w.E, float), np.asarray(w.nu, float))
        self.kappa = np.asarray(w.k, float) / w.mu_f
        self.tau = stabilization_parameter(w, self.lam, self.G, self.kappa, w.dt)
        self.surf = np.ascontiguousarray(w.surf_id, dtype=np.int32)
        self.surf_n = np.ascontiguousarray(w.surf_normal, float)
        self.surf_A = np.ascontiguousarray(w.surf_area, float)
        self.t = 0.0
        self.newton_rtol = newton_rtol
        self.newton_max = newton_max
        self.newton_stag = newton_stag
        self.phi_min = min_volume_fraction
        self.u_fixed = np.asarray(w.u_fixed, np.uint8).copy()
        self.u_value = np.asarray(w.u_value, float).copy()
        self.p_fixed = np.asarray(w.p_fixed, np.uint8).copy()
        self.p_value = np.asarray(w.p_value, float).copy()
        self.nn = int(lib().orc_nnodes(C.byref(self.g)))
        self.last = None

    # -- mixture mass of each point for this step: incompressible constituents
    def mixture_mass(self):
        w = self.w
        J = det(self.F, self.d)
        phi = 1.0 - (1.0 - w.phi0) / J
        rho = (1.0 - phi) * w.rho_s + phi * w.rho_f
        return rho * self.V

    def _step_struct(self, dt):
        w = self.w
        s = _Step()
        s.dt, s.dynamic, s.beta, s.gamma = dt, int(w.dynamic), w.beta, w.gamma
        s.rho_f, s.alpha_vis = w.rho_f, (w.alpha_vis if w.dynamic else 0.0)
        for k in range(3):
            s.g[k] = w.g[k]
        s.kozeny, s.phi0 = int(w.permeability == PERM_KOZENY_CARMAN), w.phi0
        s.hencky = int(w.model == MODEL_HENCKY)
        return s

    def _particles_struct(self, m):
        pp = _Particles()
        pp.n = self.n
        self._keep = [np.ascontiguousarray(m)]
        pp.x, pp.lp, pp.F, pp.V = _p(self.x), _p(self.lp), _p(self.F), _p(self.V)
        pp.m = _p(self._keep[0])
        pp.lam, pp.G, pp.kappa, pp.tau = _p(self.lam), _p(self.G), _p(self.kappa), _p(self.tau)
        pp.surf, pp.surf_n, pp.surf_A = _p(self.surf), _p(self.surf_n), _p(self.surf_A)
        return pp

    # -- Stage 1 + pattern: everything that is fixed over the Newton loop
    def prepare(self, dt):
        d = self.d
        kap_n = self.kappa
        if self.w.permeability == PERM_KOZENY_CARMAN:   # the mobility at the start of the step
            kap_n = kozeny_carman(self.kappa, self.w.phi0, det(self.F, d))
        self.tau = stabilization_parameter(self.w, self.lam, self.G, kap_n, dt)
        first, count, S, dS, S0 = shape(self.g, self.x, self.lp)
        m = self.mixture_mass()
        fld = [self.p[:, None]]
        if self.w.dynamic:
            fld += [self.v, self.a, self.pd[:, None], self.pdd[:, None]]
        M, out = p2g(self.g, first, count, S, m, np.concatenate(fld, axis=1))
        # nodal volume fraction sum_p S_ip V_p / h^d (activity of the node)
        Mv, _ = p2g(self.g, first, count, S, self.V, np.zeros(self.n))
        phi = Mv / self.w.h ** d
        Pn = np.ascontiguousarray(out[:, 0])
        nodal = {"P": Pn}
        if self.w.dynamic:
            nodal["v"] = np.ascontiguousarray(out[:, 1:1 + d])
            nodal["a"] = np.ascontiguousarray(out[:, 1 + d:1 + 2 * d])
            nodal["pd"] = np.ascontiguousarray(out[:, 1 + 2 * d])
            nodal["pdd"] = np.ascontiguousarray(out[:, 2 + 2 * d])
        row_ptr, col = pattern(self.g, first, count)
        if self.w.p2g_mass == P2G_CONSISTENT:
            act = (M > 0.0) & (phi > self.phi_min)
            out = consistent_map(self.g, first, count, S, m, M, act, out, row_ptr, col)
            nodal["P"] = np.ascontiguousarray(out[:, 0])
            if self.w.dynamic:
                nodal["v"] = np.ascontiguousarray(out[:, 1:1 + d])
                nodal["a"] = np.ascontiguousarray(out[:, 1 + d:1 + 2 * d])
                nodal["pd"] = np.ascontiguousarray(out[:, 1 + 2 * d])
                nodal["pdd"] = np.ascontiguousarray(out[:, 2 + 2 * d])
        active = (M > 0.0) & (phi > self.phi_min)
        return dict(first=first, count=count, S=S, dS=dS, S0=S0, m=m, M=M, phi=phi,
                    active=active, active_u8=np.ascontiguousarray(active.astype(np.uint8)),
                    nodal=nodal, row_ptr=row_ptr, col=col, dt=dt)

    def _nodal_struct(self, nodal):
        nd = _Nodal()
        nd.P = _p(nodal["P"])
        nd.v = _p(nodal.get("v"))
        nd.a = _p(nodal.get("a"))
        nd.pd = _p(nodal.get("pd"))
        nd.pdd = _p(nodal.get("pdd"))
        return nd

    def eval(self, prep, X, traction, flux=None, want_J=True):
        """Residual R(X) and the Jacobian block values (pattern of `prep`)."""
        d, nb = self.d, self.d + 1
        X = np.ascontiguousarray(X, float).reshape(-1)
        R = np.zeros(self.nn * nb)
        nnzb = int(prep["row_ptr"][-1])
        Jv = np.zeros(nnzb * nb * nb) if want_J else None
        sp = self._step_struct(prep["dt"])
        pp = self._particles_struct(prep["m"])
        nd = self._nodal_struct(prep["nodal"])
        trac = np.ascontiguousarray(traction, float).reshape(-1) if traction is not None \
            else np.zeros(max(1, self.w.n_surf * d))
        flx = None if flux is None else np.ascontiguousarray(flux, float)
        rc = lib().orc_eval(C.byref(self.g), C.byref(sp), C.byref(pp), _p(prep["first"]),
                            _p(prep["count"]), _p(prep["S"]), _p(prep["dS"]), _p(prep["S0"]),
                            _p(prep["active_u8"]), C.byref(nd), _p(trac), _p(flx), _p(X),
                            _p(prep["row_ptr"]), _p(prep["col"]), _p(R), _p(Jv))
        _check(rc, "eval")
        return R, Jv

    def eval_frozen(self, prep, X, Xf, traction, flux=None):
        """Residual with the terms the Jacobian leaves unlinearized (Sec. 3.4:
        the Kelvin stress's geometry, Darcy's acceleration) frozen at the
        iterate Xf; its derivative at X = Xf is the Jacobian of eval."""
        d, nb = self.d, self.d + 1
        X = np.ascontiguousarray(X, float).reshape(-1)
        Xf = np.ascontiguousarray(Xf, float).reshape(-1)
        R = np.zeros(self.nn * nb)
        sp = self._step_struct(prep["dt"])
        pp = self._particles_struct(prep["m"])
        nd = self._nodal_struct(prep["nodal"])
        trac = np.ascontiguousarray(traction, float).reshape(-1) if traction is not None \
            else np.zeros(max(1, self.w.n_surf * d))
        flx = None if flux is None else np.ascontiguousarray(flux, float)
        rc = lib().orc_eval_frozen(C.byref(self.g), C.byref(sp), C.byref(pp), _p(prep["first"]),
                                   _p(prep["count"]), _p(prep["S"]), _p(prep["dS"]), _p(prep["S0"]),
                                   _p(prep["active_u8"]), C.byref(nd), _p(trac), _p(flx), _p(X), _p(Xf),
                                   _p(R))
        _check(rc, "eval_frozen")
        return R

    def fixed_dofs(self, prep):
        """Dirichlet DOFs plus every DOF of an inactive node: a node whose
        volume fraction sum_p S_ip V_p / h^d is at most the threshold (the
        minimum-mass rule of GIMP codes)."""
        d, nb = self.d, self.d + 1
        fixed = np.zeros((self.nn, nb), bool)
        fixed[:, :d] = self.u_fixed.astype(bool)
        fixed[:, d] = self.p_fixed.astype(bool)
        fixed[~prep["active"], :] = True
        return fixed.reshape(-1)

    def initial_guess(self, prep):
        d, nb = self.d, self.d + 1
        X = np.zeros((self.nn, nb))
        X[:, d] = prep["nodal"]["P"]
        uf = self.u_fixed.astype(bool)
        X[:, :d][uf] = self.u_value[uf]
        pf = self.p_fixed.astype(bool)
        X[pf, d] = self.p_value[pf]
        X[~prep["active"], :] = 0.0
        return X.reshape(-1)

    def jacobian_matrix(self, prep, Jv, fixed):
        nb = self.d + 1
        nnzb = int(prep["row_ptr"][-1])
        J = sps.bsr_matrix((Jv.reshape(nnzb, nb, nb), prep["col"], prep["row_ptr"]),
                           shape=(self.nn * nb, self.nn * nb)).tocsr()
        free = sps.diags((~fixed).astype(float))
        return (free @ J @ free + sps.diags(fixed.astype(float))).tocsc()

    @staticmethod
    def solve(J, b):
        """Direct solve of J x = b after row then column max-norm equilibration."""
        J = J.tocsr()
        r = np.asarray(abs(J).max(axis=1).todense()).reshape(-1)
        r[r == 0] = 1.0
        Dr = sps.diags(1.0 / r)
        Js = (Dr @ J).tocsc()
        c = np.asarray(abs(Js).max(axis=0).todense()).reshape(-1)
        c[c == 0] = 1.0
        Dc = sps.diags(1.0 / c)
        Js = (Js @ Dc).tocsc()
        lu = spla.splu(Js)
        y = lu.solve(Dr @ b)
        return Dc @ y

    def newton(self, prep, traction, flux=None):
        X = self.initial_guess(prep)
        fixed = self.fixed_dofs(prep)
        R, Jv = self.eval(prep, X, traction, flux)
        R[fixed] = 0.0
        r0 = float(np.linalg.norm(R))
        hist = [r0]
        k = 0
        while True:
            rk = hist[-1]
            if r0 == 0.0 or rk <= self.newton_rtol * r0:
                break
            # round-off floor: the previous iterate was already small and this
            # one failed to halve it (quadratic convergence has stopped)
            if self.newton_stag > 0.0 and k >= 2 and hist[-2] <= self.newton_stag * r0 \
                    and rk > 0.5 * hist[-2]:
                break
            if k >= self.newton_max:
                raise OracleError(f"Newton did not converge: {hist}")
            Jm = self.jacobian_matrix(prep, Jv, fixed)
            dX = self.solve(Jm, -R)
            dX[fixed] = 0.0
            X = X + dX
            R, Jv = self.eval(prep, X, traction, flux)
            R[fixed] = 0.0
            hist.append(float(np.linalg.norm(R)))
            k += 1
        return X, StepInfo(newton_iters=k, res_hist=hist)

    def update(self, prep, X):
        sp = self._step_struct(prep["dt"])
        nd = self._nodal_struct(prep["nodal"])
        rc = lib().orc_g2p(C.byref(self.g), C.byref(sp), C.c_int64(self.n), _p(prep["first"]),
                           _p(prep["count"]), _p(prep["S"]), _p(prep["dS"]), _p(prep["S0"]),
                           _p(prep["active_u8"]), C.byref(nd),
                           _p(np.ascontiguousarray(X)), _p(self.x), _p(self.u), _p(self.F),
                           _p(self.V), _p(self.lp), _p(self.lp0), _p(self.p), _p(self.v),
                           _p(self.a), _p(self.pd), _p(self.pdd))
        _check(rc, "g2p")

    def step(self, dt=None, traction=None, flux=None):
        dt = self.w.dt if dt is None else dt
        if traction is None:
            traction = self.w.traction(self.t + dt)
        prep = self.prepare(dt)
        X, info = self.newton(prep, traction, flux)
        self.update(prep, X)
        self.t += dt
        self.last = (prep, X, info)
        return info

    def state(self):
        return dict(x=self.x.copy(), u=self.u.copy(), p=self.p.copy(), v=self.v.copy(),
                    F=self.F.copy(), V=self.V.copy(), lp=self.lp.copy(), a=self.a.copy(),
                    pd=self.pd.copy(), pdd=self.pdd.copy())
