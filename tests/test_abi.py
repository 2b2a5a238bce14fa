"""The C ABI library builds, loads without a GPU, and exports every declared symbol."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mto.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mto_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2301_07457_gb300.build import build
    try:
        return build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mto_create_mesh", "mto_set_design", "mto_solve", "mto_compliance_grad",
                     "mto_destroy", "mto_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mto_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(libpath):
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    assert set(_lib.SIGNATURES) == set(declared_functions())
    assert lib.mto_status_string(0) == b"ok"
    assert lib.mto_status_string(5) == b"not converged"
    o = _lib.default_opts()
    assert (o.tol, o.max_it, o.omega, o.nu1, o.nu2, o.n_coarsen) == (1e-8, 500, 0.6, 2, 2, 3)
    assert o.gamma == 1


def test_argument_validation_needs_no_gpu(libpath):
    import ctypes
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    o = _lib.default_opts()
    # Rejected before any CUDA call: bad sizes, no clamped edge, bad options.
    assert lib.mto_create_mesh(ctypes.byref(h), 0, 8, 0.3, 1, ctypes.byref(o), 0, None) == _lib.ERR_ARG
    assert lib.mto_create_mesh(ctypes.byref(h), 8, 8, 0.3, 0, ctypes.byref(o), 0, None) == _lib.ERR_ARG
    assert lib.mto_create_mesh(ctypes.byref(h), 12, 8, 0.3, 1, ctypes.byref(o), 0, None) == \
        _lib.ERR_UNSUPPORTED_MESH
    o.omega = 1.5
    assert lib.mto_create_mesh(ctypes.byref(h), 8, 8, 0.3, 1, ctypes.byref(o), 0, None) == _lib.ERR_ARG
    # Cycle index: 1..4, and at most 512 coarse-grid calls per cycle
    # (gamma = 3 with 8 coarsenings makes 1093).
    o.omega = 0.6
    for gamma, nc in ((0, 3), (5, 3), (3, 8)):
        o.gamma, o.n_coarsen = gamma, nc
        assert lib.mto_create_mesh(ctypes.byref(h), 512, 512, 0.3, 1, ctypes.byref(o), 0,
                                   None) == _lib.ERR_ARG, (gamma, nc)
    assert lib.mto_solve(None, 1, None, None, None) == _lib.ERR_ARG
    assert lib.mto_create_mesh(None, 8, 8, 0.3, 1, None, 0, None) == _lib.ERR_ARG


def test_poisson_argument_validation_needs_no_gpu(libpath):
    import ctypes
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    o = _lib.PoissonOpts()
    lib.mto_poisson_default_opts(ctypes.byref(o))
    assert (o.tol, o.max_it, o.omega, o.nu1, o.nu2, o.n_coarsen, o.cluster_ctas) == (1e-8, 500, 0.6, 2, 2, 3, 0)
    create = lambda nx, ny: lib.mto_poisson_create(ctypes.byref(h), nx, ny, ctypes.byref(o), 0, None)
    assert create(1, 8) == _lib.ERR_ARG
    assert create(12, 8) == _lib.ERR_UNSUPPORTED_MESH      # not divisible by 2^3
    assert create(8, 8) == _lib.ERR_UNSUPPORTED_MESH       # coarsest 1 x 1 has no interior node
    o.n_coarsen = 1
    assert create(128, 128) == _lib.ERR_UNSUPPORTED_MESH   # coarsest 63^2 interior nodes > 1024
    o.n_coarsen, o.cluster_ctas = 3, 3
    assert create(64, 64) == _lib.ERR_ARG                  # cluster sizes are powers of two <= 16
    o.cluster_ctas, o.omega = 0, 1.5
    assert create(64, 64) == _lib.ERR_ARG
    assert lib.mto_poisson_solve(None, 1, None, None, None) == _lib.ERR_ARG
    assert lib.mto_poisson_create(None, 8, 8, None, 0, None) == _lib.ERR_ARG


def test_memory_ledger_needs_no_gpu(libpath):
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    assert lib.mto_device_memory_in_use() == 0  # nothing allocated in this process
    lib.mto_set_device_memory_limit(1 << 20)
    lib.mto_set_device_memory_limit(0)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # No CPU fallback: without libmto.so the binding refuses to work, both
    # when loaded directly and through the public classes.
    import pytest
    from paper_2301_07457_gb300 import _lib
    import paper_2301_07457_gb300 as mto
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libmto.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError, match="libmto.so not found"):
        _lib.load()
    with pytest.raises(ImportError, match="libmto.so not found"):
        mto.Mesh(32, 32, n_coarsen=2)
