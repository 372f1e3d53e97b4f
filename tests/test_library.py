"""CPU-only checks of the C-ABI library: it builds, loads, exports every entry
point include/mpm.h declares, and the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

from paper_1905_00671_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mpm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpm_create", "mpm_step", "mpm_read", "mpm_destroy", "mpm_get_stats",
                     "mpm_last_error", "mpm_default_options"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_without_gpu(lib):
    from paper_1905_00671_gb300 import mpm

    o = mpm.default_options()
    assert o.shape == mpm.MPM_SHAPE_GIMP and o.newton_rtol == 1e-8 and o.krylov_restart == 120
    assert o.precond_lag == 2
    assert o.precond_reuse == 0  # the coarse levels rebuilt at every step
    assert o.precond == mpm.MPM_PRECOND_SCHUR_MG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1905_00671_gb300 import mpm

    monkeypatch.setattr(B, "SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mpm, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        mpm.load()


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1905_00671_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).lower() or f == "inputs.py", f


@pytest.mark.parametrize("opts,model,why", [
    (dict(krylov_restart=200), None, "krylov_restart must be in 1..128"),
    (dict(model=2), None, "unknown model"),
    (dict(tau_kind=2), None, "MPM_TAU_MONFORTE needs the Newmark scheme"),
    (dict(min_volume_fraction=-1.0), None, "min_volume_fraction"),
    (dict(precond_reuse=-1), None, "precond_reuse must be in"),
])
def test_rejected_create_names_its_reason_without_gpu(lib, opts, model, why):
    """Argument checks run on the host before any device call: mpm_create
    returns MPM_ERR_BAD_ARG and mpm_last_error(NULL) says why."""
    from dataclasses import replace

    from paper_1905_00671_gb300 import inputs as I
    from paper_1905_00671_gb300 import mpm

    w = I.terzaghi_column(ncell_y=4, ncell_x=2)          # quasi-static
    if model is not None:
        w = replace(w, model=model)
    with pytest.raises(mpm.MPMError, match=why) as e:
        mpm.Simulation(w, **opts)
    assert e.value.code == -1                            # MPM_ERR_BAD_ARG


@pytest.mark.parametrize("field,value,why", [
    ("vol", -1e-3, "point volume must be positive"),
    ("vol", float("nan"), "point volume must be positive"),
    ("x", float("inf"), "non-finite point position"),
    ("E", float("nan"), "E must be positive and finite"),
    ("E", 0.0, "E must be positive and finite"),
    ("nu", 0.5, "nu must lie in"),
    ("k", -1e-12, "permeability must be non-negative"),
])
def test_bad_point_data_is_rejected_at_create_without_gpu(lib, field, value, why):
    """Host-made faults in the points' own data (a negative or NaN volume, an
    infinite position, a NaN or zero modulus, an incompressible nu, a negative
    permeability) are rejected by mpm_create before any device call."""
    from dataclasses import replace

    import numpy as np

    from paper_1905_00671_gb300 import inputs as I
    from paper_1905_00671_gb300 import mpm

    w = I.terzaghi_column(ncell_y=4, ncell_x=2)
    a = getattr(w, field).copy()
    a.reshape(-1)[3] = value
    with pytest.raises(mpm.MPMError, match=why) as e:
        mpm.Simulation(replace(w, **{field: np.ascontiguousarray(a)}))
    assert e.value.code == -1


def test_rejected_batch_create_names_its_reason_without_gpu(lib):
    from dataclasses import replace

    from paper_1905_00671_gb300 import inputs as I
    from paper_1905_00671_gb300 import mpm

    a = I.terzaghi_column(ncell_y=4, ncell_x=2)
    b = replace(I.terzaghi_column(ncell_y=6, ncell_x=2), rho_f=900.0)
    with pytest.raises(mpm.MPMError, match="material constants differ"):
        mpm.Batch([a, b])


def test_last_error_without_a_context_on_a_fresh_thread(lib):
    import threading

    from paper_1905_00671_gb300 import mpm

    m = mpm.load()
    out = []
    t = threading.Thread(target=lambda: out.append(m.mpm_last_error(None)))
    t.start()
    t.join()
    assert out == [b"null context"]


def _empty_points(w):
    import numpy as np
    d = w.dim
    return dict(x=np.zeros((0, d)), vol=np.zeros(0), lp=np.zeros((0, d)), p0=np.zeros(0), v0=None,
                E=np.zeros(0), nu=np.zeros(0), k=np.zeros(0), surf_id=np.zeros(0, np.int32),
                surf_normal=np.zeros((0, d)), surf_area=np.zeros(0), trac_full=np.zeros((0, d)))


@pytest.mark.parametrize("case,why", [
    ("no points", "need n > 0 points"),
    ("dim 4", "grid.dim must be 2 or 3"),
    ("zero cells", "grid.ncell must be at least 1"),
    ("zero spacing", "grid.h must be positive"),
    ("surface id out of range", "surf_id outside"),
    ("zero fluid viscosity", "material.mu_f must be positive"),
])
def test_degenerate_inputs_are_rejected_at_create_without_gpu(lib, case, why):
    """Degenerate problems (an empty point set, a grid of another dimension,
    of no cells or of zero spacing, a surface id past the surface count, no
    fluid viscosity) return MPM_ERR_BAD_ARG from mpm_create before any device
    call, with the reason in mpm_last_error."""
    from dataclasses import replace

    import numpy as np

    from paper_1905_00671_gb300 import inputs as I
    from paper_1905_00671_gb300 import mpm

    w = I.terzaghi_column(ncell_y=4, ncell_x=2)
    if case == "no points":
        w = replace(w, **_empty_points(w))
    elif case == "dim 4":
        w = replace(w, dim=4)
    elif case == "zero cells":
        w = replace(w, ncell=(2, 0, 0))
    elif case == "zero spacing":
        w = replace(w, h=0.0)
    elif case == "surface id out of range":
        sid = w.surf_id.copy()
        sid[np.nonzero(sid >= 0)[0][0]] = w.n_surf
        w = replace(w, surf_id=sid)
    elif case == "zero fluid viscosity":
        w = replace(w, mu_f=0.0)
    with pytest.raises(mpm.MPMError, match=why) as e:
        mpm.Simulation(w)
    assert e.value.code == -1
