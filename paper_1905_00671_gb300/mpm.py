"""Thin ctypes binding of the C-ABI in include/mpm.h (argument marshalling only).

Every function of the C-ABI is exposed under the same name; `Simulation` wraps
a context for a `inputs.Workload`.  The CUDA library is loaded on first use;
if it has not been built this module raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

MPM_OK = 0
ERRORS = {-1: "MPM_ERR_BAD_ARG", -2: "MPM_ERR_OUT_OF_GRID", -3: "MPM_ERR_NEGATIVE_J",
          -4: "MPM_ERR_NONFINITE", -5: "MPM_ERR_NEWTON_DIVERGED", -6: "MPM_ERR_KRYLOV_STAGNATED",
          -7: "MPM_ERR_TIMEOUT", -8: "MPM_ERR_CUDA", -9: "MPM_ERR_NO_MEMORY"}
MPM_SHAPE_ORIG, MPM_SHAPE_GIMP = 0, 1
MPM_QUASISTATIC, MPM_NEWMARK = 0, 1
MPM_FP64, MPM_MIXED = 0, 1
MPM_TAU_WHITE, MPM_TAU_SUN, MPM_TAU_MONFORTE = 0, 1, 2
MPM_PERM_CONSTANT, MPM_PERM_KOZENY_CARMAN = 0, 1
MPM_P2G_LUMPED, MPM_P2G_CONSISTENT = 0, 1
MPM_MODEL_NEOHOOKE, MPM_MODEL_HENCKY = 0, 1
MPM_PRECOND_BLOCK_JACOBI, MPM_PRECOND_SCHUR_MG = 0, 1
MPM_SCHUR_LOWER, MPM_SCHUR_UPPER = 0, 1
MPM_MAX_NEWTON = 64
PROF = {"spmv": 0, "jacobian": 1, "residual": 2, "point": 3, "orth": 4, "p2g": 5, "g2p": 6,
        "precond": 7, "setup": 8, "prep": 9}

EXPORTED = ["mpm_default_options", "mpm_create", "mpm_step", "mpm_read", "mpm_get_stats",
            "mpm_last_error", "mpm_destroy", "mpm_debug_bin", "mpm_debug_prepare",
            "mpm_debug_pattern", "mpm_debug_nodal", "mpm_debug_eval", "mpm_debug_precond",
            "mpm_debug_jacobian32"]


class MPMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class mpm_grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("ncell", C.c_int32 * 3), ("origin", C.c_double * 3),
                ("h", C.c_double)]


class mpm_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("vol", C.c_void_p), ("lp", C.c_void_p),
                ("p0", C.c_void_p), ("v0", C.c_void_p), ("surf_id", C.c_void_p),
                ("surf_normal", C.c_void_p), ("surf_area", C.c_void_p), ("n_surf", C.c_int32)]


class mpm_material(C.Structure):
    _fields_ = [("E", C.c_void_p), ("nu", C.c_void_p), ("rho_s", C.c_double),
                ("rho_f", C.c_double), ("phi0", C.c_double), ("mu_f", C.c_double),
                ("alpha_vis", C.c_double), ("g", C.c_double * 3)]


class mpm_options(C.Structure):
    _fields_ = [("shape", C.c_int32), ("scheme", C.c_int32), ("beta", C.c_double),
                ("gamma", C.c_double), ("stabilize", C.c_int32), ("tau_scale", C.c_double),
                ("precision", C.c_int32), ("newton_rtol", C.c_double), ("newton_max", C.c_int32),
                ("newton_stag", C.c_double), ("krylov_rtol", C.c_double),
                ("krylov_restart", C.c_int32), ("krylov_max", C.c_int32), ("precond", C.c_int32),
                ("min_volume_fraction", C.c_double), ("profile", C.c_int32),
                ("precond_lag", C.c_int32), ("schur_approx", C.c_int32), ("stream", C.c_void_p),
                ("tau_kind", C.c_int32), ("permeability", C.c_int32), ("p2g_mass", C.c_int32),
                ("model", C.c_int32), ("schur_order", C.c_int32), ("mg_sweeps", C.c_int32),
                ("mg_omega", C.c_double), ("autotune", C.c_int32),
                ("precond_reuse", C.c_int32)]


class mpm_loads(C.Structure):
    _fields_ = [("traction", C.c_void_p), ("flux", C.c_void_p), ("scale", C.c_double)]


class mpm_bcs(C.Structure):
    _fields_ = [("u_fixed", C.c_void_p), ("u_value", C.c_void_p), ("p_fixed", C.c_void_p),
                ("p_value", C.c_void_p)]


class mpm_particles_out(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("x", "u", "p", "v", "a", "F", "V", "lp", "pd", "pdd")]


class mpm_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("krylov_iters", C.c_int32 * MPM_MAX_NEWTON),
                ("res_norm", C.c_double * (MPM_MAX_NEWTON + 1)), ("krylov_total", C.c_int32),
                ("steps", C.c_int64), ("t", C.c_double), ("nnzb", C.c_int64),
                ("kernel_launches", C.c_int64), ("prof_ms", C.c_double * 10),
                ("prof_launches", C.c_int64 * 10), ("jac_terms", C.c_int64),
                ("jac_point_nodes", C.c_int64), ("jac_config", C.c_int32 * 2),
                ("jac_tuned", C.c_int32 * 2), ("jac_tune_ms", (C.c_float * 6) * 2)]


_lib = None


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = False):
    """Loads libupmpm.so; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.SO):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {_build.SO} is not built; run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        _build.build()
    lib = C.CDLL(_build.SO)
    P = C.c_void_p
    lib.mpm_default_options.argtypes = [C.POINTER(mpm_options)]
    lib.mpm_default_options.restype = None
    lib.mpm_create.argtypes = [C.POINTER(mpm_grid), C.POINTER(mpm_particles), C.POINTER(mpm_material),
                               P, C.POINTER(mpm_options), C.POINTER(P)]
    lib.mpm_step.argtypes = [P, C.c_double, C.POINTER(mpm_loads), C.POINTER(mpm_bcs)]
    lib.mpm_read.argtypes = [P, C.POINTER(mpm_particles_out)]
    lib.mpm_get_stats.argtypes = [P, C.POINTER(mpm_stats)]
    lib.mpm_last_error.argtypes = [P]
    lib.mpm_last_error.restype = C.c_char_p
    lib.mpm_destroy.argtypes = [P]
    lib.mpm_destroy.restype = None
    lib.mpm_debug_bin.argtypes = [P, P, P]
    lib.mpm_debug_prepare.argtypes = [P, C.c_double, C.POINTER(mpm_loads), C.POINTER(mpm_bcs)]
    lib.mpm_debug_pattern.argtypes = [P, P, P, C.c_int64]
    lib.mpm_debug_pattern.restype = C.c_int64
    lib.mpm_debug_nodal.argtypes = [P, P, P, P]
    lib.mpm_debug_eval.argtypes = [P, P, P, P, C.c_int32]
    lib.mpm_debug_precond.argtypes = [P, P, P, P]
    lib.mpm_debug_jacobian32.argtypes = [P, P, C.c_int32, C.c_int32, P, C.c_int32]
    lib.mpm_restore.argtypes = [P, C.POINTER(mpm_particles_out), C.c_double, C.c_int64]
    lib.mpm_batch_pack.argtypes = [C.c_int32, C.POINTER(mpm_grid), P, P]
    lib.mpm_create_batch.argtypes = [C.c_int32, C.POINTER(mpm_grid), C.POINTER(mpm_particles),
                                     C.POINTER(mpm_material), P, C.POINTER(mpm_options), C.POINTER(P)]
    lib.mpm_step_batch.argtypes = [P, C.c_double, P, P]
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def default_options() -> mpm_options:
    o = mpm_options()
    load().mpm_default_options(C.byref(o))
    return o


def _grid(w) -> mpm_grid:
    g = mpm_grid()
    g.dim = w.dim
    for k in range(3):
        g.ncell[k] = int(w.ncell[k]) if k < w.dim else 0
        g.origin[k] = float(w.origin[k]) if k < w.dim else 0.0
    g.h = float(w.h)
    return g


def _point_structs(w):
    """(arrays kept alive, mpm_particles, mpm_material) of a Workload."""
    K = {
        "x": _f64(w.x), "vol": _f64(w.vol), "lp": _f64(w.lp), "p0": _f64(w.p0),
        "v0": _f64(w.v0), "surf_id": np.ascontiguousarray(w.surf_id, dtype=np.int32),
        "sn": _f64(w.surf_normal), "sa": _f64(w.surf_area), "E": _f64(w.E), "nu": _f64(w.nu),
        "k": _f64(w.k),
    }
    P = mpm_particles(n=w.n, x=_p(K["x"]), vol=_p(K["vol"]), lp=_p(K["lp"]), p0=_p(K["p0"]),
                      v0=_p(K["v0"]), surf_id=_p(K["surf_id"]), surf_normal=_p(K["sn"]),
                      surf_area=_p(K["sa"]), n_surf=w.n_surf)
    M = mpm_material(E=_p(K["E"]), nu=_p(K["nu"]), rho_s=w.rho_s, rho_f=w.rho_f, phi0=w.phi0,
                     mu_f=w.mu_f, alpha_vis=w.alpha_vis)
    for k in range(3):
        M.g[k] = w.g[k] if k < len(w.g) else 0.0
    return K, P, M


def _options(w, stream, opts) -> mpm_options:
    o = default_options()
    o.shape = int(w.shape)
    o.scheme = MPM_NEWMARK if w.dynamic else MPM_QUASISTATIC
    o.beta, o.gamma = w.beta, w.gamma
    o.stabilize = int(bool(w.stabilize))
    o.tau_scale = w.tau_scale
    o.tau_kind = int(w.tau_kind)
    o.permeability = int(w.permeability)
    o.p2g_mass = int(w.p2g_mass)
    o.model = int(w.model)
    for key, val in opts.items():
        setattr(o, key, val)
    if stream is not None:
        o.stream = stream
    return o


_FIELDS = ("x", "u", "p", "v", "a", "F", "V", "lp", "pd", "pdd")


def _read(lib, ctx, n, d, fields, check):
    comps = {"x": d, "u": d, "p": 1, "v": d, "a": d, "F": d * d, "V": 1, "lp": d, "pd": 1,
             "pdd": 1}
    out = {k: np.zeros((n, comps[k])) if comps[k] > 1 else np.zeros(n) for k in fields}
    o = mpm_particles_out(**{k: _p(v) for k, v in out.items()})
    check(lib.mpm_read(ctx, C.byref(o)), "mpm_read")
    return out


def batch_pack(grids_of):
    """mpm_batch_pack for a list of Workloads (host only): (offsets (count, 3),
    background ncell (3,))."""
    lib = load()
    gs = (mpm_grid * len(grids_of))(*[_grid(w) for w in grids_of])
    offs = np.zeros((len(grids_of), 3), np.int32)
    nc = np.zeros(3, np.int32)
    rc = lib.mpm_batch_pack(len(grids_of), gs, _p(offs), _p(nc))
    if rc != MPM_OK:
        raise MPMError(rc, "mpm_batch_pack failed")
    return offs, nc


class Simulation:
    """One context for a Workload (see inputs.py).  Host arrays in, host arrays
    out; all computation in the CUDA library."""

    def __init__(self, w, stream: Optional[int] = None, **opts):
        lib = load()
        self.w = w
        self.lib = lib
        g = _grid(w)
        K, P, M = _point_structs(w)
        self._keep = K
        o = _options(w, stream, opts)
        self.options = o
        ctx = C.c_void_p()
        rc = lib.mpm_create(C.byref(g), C.byref(P), C.byref(M), _p(K["k"]), C.byref(o), C.byref(ctx))
        if rc != MPM_OK:
            raise MPMError(rc, "mpm_create: " + lib.mpm_last_error(None).decode())
        self.ctx = ctx
        self.t = 0.0
        self._bcs_sent = False
        self.set_bcs(w.u_fixed, w.u_value, w.p_fixed, w.p_value)

    # -- marshalling helpers
    def set_bcs(self, u_fixed, u_value, p_fixed, p_value):
        self._bc = {"uf": np.ascontiguousarray(u_fixed, dtype=np.uint8),
                    "uv": _f64(u_value), "pf": np.ascontiguousarray(p_fixed, dtype=np.uint8),
                    "pv": _f64(p_value)}
        self._bcs_sent = False

    def _bcs_struct(self):
        if self._bcs_sent:
            return None
        b = self._bc
        return mpm_bcs(u_fixed=_p(b["uf"]), u_value=_p(b["uv"]), p_fixed=_p(b["pf"]),
                       p_value=_p(b["pv"]))

    def _loads_struct(self, t_next, traction, resident):
        if resident and self._bcs_sent:
            return mpm_loads(traction=None, flux=None, scale=self.w.load_scale(t_next))
        if traction is None:
            self._trac = np.ascontiguousarray(self.w.trac_full, dtype=np.float64)
            scale = self.w.load_scale(t_next)
        else:
            self._trac = np.ascontiguousarray(traction, dtype=np.float64)
            scale = 1.0
        return mpm_loads(traction=_p(self._trac) if self.w.n_surf else None, flux=None,
                         scale=scale)

    def _check(self, rc, what):
        if rc != MPM_OK:
            msg = self.lib.mpm_last_error(self.ctx)
            raise MPMError(rc, f"{what}: {msg.decode() if msg else ''}")

    # -- the C-ABI calls
    def step(self, dt=None, traction=None, resident=False):
        """mpm_step for t -> t + dt.  traction: host array (n_surf, d) applied as
        is; None applies the workload's traction at t + dt; resident=True keeps
        the traction already on the device and sends only its scale."""
        dt = self.w.dt if dt is None else dt
        L = self._loads_struct(self.t + dt, traction, resident)
        B = self._bcs_struct()
        rc = self.lib.mpm_step(self.ctx, C.c_double(dt), C.byref(L),
                               C.byref(B) if B is not None else None)
        self._check(rc, "mpm_step")
        self._bcs_sent = True
        self.t += dt
        return self.stats()

    def read(self, fields=_FIELDS):
        return _read(self.lib, self.ctx, self.w.n, self.w.dim, fields, self._check)

    def checkpoint(self):
        """The full point state (every field of mpm_read) and the time."""
        return {"state": self.read(_FIELDS), "t": self.t, "steps": self.stats()["steps"]}

    def restore(self, ck):
        """mpm_restore of a checkpoint taken from a context of the same workload."""
        keep = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in ck["state"].items()}
        o = mpm_particles_out(**{k: _p(v) for k, v in keep.items()})
        self._check(self.lib.mpm_restore(self.ctx, C.byref(o), C.c_double(ck["t"]),
                                         C.c_int64(ck["steps"])), "mpm_restore")
        self.t = ck["t"]

    def stats(self):
        s = mpm_stats()
        self._check(self.lib.mpm_get_stats(self.ctx, C.byref(s)), "mpm_get_stats")
        k = s.newton_iters
        return {"newton_iters": k, "krylov_iters": list(s.krylov_iters[:k]),
                "res_norm": list(s.res_norm[:k + 1]), "krylov_total": s.krylov_total,
                "steps": s.steps, "t": s.t, "nnzb": s.nnzb, "kernel_launches": s.kernel_launches,
                "prof_ms": {k: s.prof_ms[i] for k, i in PROF.items()},
                "prof_launches": {k: s.prof_launches[i] for k, i in PROF.items()},
                "jac_terms": s.jac_terms, "jac_point_nodes": s.jac_point_nodes,
                "jac_config": list(s.jac_config), "jac_tuned": list(s.jac_tuned),
                "jac_tune_ms": [list(r) for r in s.jac_tune_ms]}

    # -- inspection
    def debug_bin(self):
        n = self.w.n
        cell = np.zeros(n, np.int32)
        order = np.zeros(n, np.int64)
        self._check(self.lib.mpm_debug_bin(self.ctx, _p(cell), _p(order)), "mpm_debug_bin")
        return cell, order

    def debug_prepare(self, dt=None):
        dt = self.w.dt if dt is None else dt
        L = self._loads_struct(self.t + dt, None, False)
        B = self._bcs_struct()
        rc = self.lib.mpm_debug_prepare(self.ctx, C.c_double(dt), C.byref(L),
                                        C.byref(B) if B is not None else None)
        self._check(rc, "mpm_debug_prepare")
        self._bcs_sent = True

    def debug_pattern(self):
        nn = self.w.nnodes
        row_ptr = np.zeros(nn + 1, np.int64)
        nnz = self.lib.mpm_debug_pattern(self.ctx, _p(row_ptr), None, 0)
        if nnz < 0:
            self._check(int(nnz), "mpm_debug_pattern")
        col = np.zeros(max(nnz, 1), np.int32)
        nnz2 = self.lib.mpm_debug_pattern(self.ctx, _p(row_ptr), _p(col), nnz)
        if nnz2 != nnz:
            self._check(int(nnz2) if nnz2 < 0 else -8, "mpm_debug_pattern")
        return row_ptr, col[:nnz]

    def debug_nodal(self):
        nn = self.w.nnodes
        M, Pn, phi = np.zeros(nn), np.zeros(nn), np.zeros(nn)
        self._check(self.lib.mpm_debug_nodal(self.ctx, _p(M), _p(Pn), _p(phi)), "mpm_debug_nodal")
        return M, Pn, phi

    def debug_eval(self, X, nnzb=None, apply_bc=False):
        nb = self.w.dim + 1
        X = _f64(X).reshape(-1)
        R = np.zeros_like(X)
        Jv = np.zeros(nnzb * nb * nb) if nnzb is not None else None
        self._check(self.lib.mpm_debug_eval(self.ctx, _p(X), _p(R), _p(Jv), int(apply_bc)),
                    "mpm_debug_eval")
        return R, Jv

    def debug_jacobian32(self, X, nnzb, form, tpb=128, apply_bc=False):
        """The mixed mode's FP32 Jacobian at X by one kernel configuration."""
        nb = self.w.dim + 1
        X = _f64(X).reshape(-1)
        Jv = np.zeros(nnzb * nb * nb, dtype=np.float32)
        self._check(self.lib.mpm_debug_jacobian32(self.ctx, _p(X), int(form), int(tpb), _p(Jv), int(apply_bc)),
                    "mpm_debug_jacobian32")
        return Jv

    def debug_precond(self, X, v):
        X = _f64(X).reshape(-1)
        v = _f64(v).reshape(-1)
        z = np.zeros_like(v)
        self._check(self.lib.mpm_debug_precond(self.ctx, _p(X), _p(v), _p(z)), "mpm_debug_precond")
        return z

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """One batched context for a list of Workloads that share dim, h, shape,
    time scheme, time step and material constants (mpm_create_batch): every
    step advances all of them with one launch per kernel."""

    def __init__(self, ws, stream: Optional[int] = None, **opts):
        lib = load()
        self.ws = list(ws)
        self.lib = lib
        m = len(self.ws)
        w0 = self.ws[0]
        self._keep = []
        grids = (mpm_grid * m)()
        parts = (mpm_particles * m)()
        mats = (mpm_material * m)()
        perms = (C.c_void_p * m)()
        for i, w in enumerate(self.ws):
            K, P, M = _point_structs(w)
            self._keep.append(K)
            grids[i], parts[i], mats[i] = _grid(w), P, M
            perms[i] = K["k"].ctypes.data
        o = _options(w0, stream, opts)
        self.options = o
        ctx = C.c_void_p()
        rc = lib.mpm_create_batch(m, grids, parts, mats, C.cast(perms, C.c_void_p), C.byref(o),
                                  C.byref(ctx))
        if rc != MPM_OK:
            raise MPMError(rc, "mpm_create_batch: " + lib.mpm_last_error(None).decode())
        self.ctx = ctx
        self.t = 0.0
        self._bcs_sent = False
        self.starts = np.concatenate([[0], np.cumsum([w.n for w in self.ws])])

    def _check(self, rc, what):
        if rc != MPM_OK:
            msg = self.lib.mpm_last_error(self.ctx)
            raise MPMError(rc, f"{what}: {msg.decode() if msg else ''}")

    def step(self, dt=None):
        """All instances t -> t + dt with each workload's traction at t + dt."""
        dt = self.ws[0].dt if dt is None else dt
        m = len(self.ws)
        loads = (mpm_loads * m)()
        self._trac = []
        for i, w in enumerate(self.ws):
            tr = np.ascontiguousarray(w.trac_full, dtype=np.float64)
            self._trac.append(tr)
            loads[i] = mpm_loads(traction=_p(tr) if w.n_surf else None, flux=None,
                                 scale=w.load_scale(self.t + dt))
        bp = None
        if not self._bcs_sent:
            bcs = (mpm_bcs * m)()
            self._bc = []
            for i, w in enumerate(self.ws):
                b = (np.ascontiguousarray(w.u_fixed, dtype=np.uint8), _f64(w.u_value),
                     np.ascontiguousarray(w.p_fixed, dtype=np.uint8), _f64(w.p_value))
                self._bc.append(b)
                bcs[i] = mpm_bcs(u_fixed=_p(b[0]), u_value=_p(b[1]), p_fixed=_p(b[2]), p_value=_p(b[3]))
            bp = C.cast(bcs, C.c_void_p)
        rc = self.lib.mpm_step_batch(self.ctx, C.c_double(dt), C.cast(loads, C.c_void_p), bp)
        self._check(rc, "mpm_step_batch")
        self._bcs_sent = True
        self.t += dt
        return self.stats()

    def stats(self):
        s = mpm_stats()
        self._check(self.lib.mpm_get_stats(self.ctx, C.byref(s)), "mpm_get_stats")
        k = s.newton_iters
        return {"newton_iters": k, "krylov_iters": list(s.krylov_iters[:k]),
                "krylov_total": s.krylov_total, "steps": s.steps, "nnzb": s.nnzb,
                "kernel_launches": s.kernel_launches,
                "jac_config": list(s.jac_config), "jac_tuned": list(s.jac_tuned),
                "jac_tune_ms": [list(r) for r in s.jac_tune_ms]}

    def read(self, fields=("x", "u", "p")):
        """Per-instance dicts of the point fields (each in its own order)."""
        n = int(self.starts[-1])
        allf = _read(self.lib, self.ctx, n, self.ws[0].dim, fields, self._check)
        return [{k: v[self.starts[i]:self.starts[i + 1]] for k, v in allf.items()}
                for i in range(len(self.ws))]

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
