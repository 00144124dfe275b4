"""Host-side checks of the C ABI (no GPU needed): the library builds, loads, exports every
entry point that include/bsparareal.h declares, and rejects bad arguments before touching
the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bsparareal.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_02521_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bs_grid_create", "fine_propagate_batched", "coarse_propagate", "pino_load",
                     "parareal_solve"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2404_02521_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(_lib.EXPORTS) | {"bs_last_error"}


def test_grid_create_rejects_bad_sizes(lib):
    from paper_2404_02521_gb300 import _lib
    h = C.c_void_p()
    assert lib.bs_grid_create(2, 4.0, C.byref(h)) == _lib.BS_ERR_ARG
    assert "M=2" in _lib.last_error()
    assert lib.bs_grid_create(64, -1.0, C.byref(h)) == _lib.BS_ERR_ARG
    assert lib.bs_grid_create(64, 4.0, None) == _lib.BS_ERR_ARG


def test_null_handles_are_rejected(lib):
    from paper_2404_02521_gb300 import _lib
    p = _lib.bs_params(0.3, 0.2, 0.5, 0.05, 1.0, 1.0, 0.5, 0.5, 0, 0, 0.0, 1.0)
    assert lib.bs_payoff(None, C.byref(p), None, None) == _lib.BS_ERR_ARG
    assert lib.fine_propagate_batched(None, C.byref(p), None, None, None, None, 1, 1, None) == _lib.BS_ERR_ARG
    assert lib.coarse_propagate(None, 0, None, C.byref(p), None, None, 0.0, 0.1, 1, None) == _lib.BS_ERR_ARG
    k = C.c_int()
    assert lib.parareal_solve(None, C.byref(p), 8, 16, 0, 4, None, 1e-4, 8, None, C.byref(k), None, None) == _lib.BS_ERR_ARG
    assert lib.pino_physics_loss(None, C.byref(p), None, None, None, 1, None, None, None) == _lib.BS_ERR_ARG
    assert lib.bs_grid_destroy(None) == _lib.BS_OK


def test_missing_weight_file(lib, tmp_path):
    from paper_2404_02521_gb300 import _lib
    h = C.c_void_p()
    rc = lib.pino_load(str(tmp_path / "nope.bin").encode(), C.byref(h))
    assert rc == _lib.BS_ERR_FILE
    assert not h.value


def test_server_rejects_bad_arguments(lib):
    from paper_2404_02521_gb300 import _lib
    h = C.c_void_p()
    assert lib.bs_server_create(None, C.byref(h)) == _lib.BS_ERR_ARG
    cfg = _lib.bs_server_config(1024, 4)            # budget below 1 MiB
    assert lib.bs_server_create(C.byref(cfg), C.byref(h)) == _lib.BS_ERR_ARG
    cfg = _lib.bs_server_config(1 << 30, 0)         # no slots
    assert lib.bs_server_create(C.byref(cfg), C.byref(h)) == _lib.BS_ERR_ARG
    req = _lib.bs_request()
    rid = C.c_longlong(0)
    assert lib.bs_server_submit(None, C.byref(req), C.byref(rid)) == _lib.BS_ERR_ARG
    n = C.c_int(0)
    assert lib.bs_server_poll(None, None, 0, C.byref(n)) == _lib.BS_ERR_ARG
    assert lib.bs_server_progress(None, None, None) == _lib.BS_ERR_ARG
    assert lib.bs_server_destroy(None) == 0


def test_options_are_range_checked(lib):
    # the coarse (G) and fine (F) Krylov tolerances are separate options, each in (0, 1);
    # an unknown option index is rejected
    from paper_2404_02521_gb300 import _lib
    lib.bs_set_option.argtypes = [C.c_int, C.c_double]
    lib.bs_set_option.restype = C.c_int
    for opt, default in [(_lib.OPT_KRYLOV_TOL, 1e-5), (_lib.OPT_FINE_KRYLOV_TOL, 1e-6)]:
        assert lib.bs_set_option(opt, 0.0) != 0
        assert lib.bs_set_option(opt, 1.0) != 0
        assert lib.bs_set_option(opt, 3e-6) == 0
        assert lib.bs_set_option(opt, default) == 0
    for bad in (-1.0, 0.5, 3.0):
        assert lib.bs_set_option(_lib.OPT_FINE_TILE, bad) != 0
    for ok in (1.0, 2.0, 0.0):
        assert lib.bs_set_option(_lib.OPT_FINE_TILE, ok) == 0
    assert lib.bs_set_option(99, 1.0) != 0


def test_coarse_variant_info(lib):
    # host-only query of a band variant: its cluster at M = 256 and which extra planes its
    # shared memory holds (16-row bands of 256 columns: the degree-2 preconditioner's and the
    # third history plane; 32-row bands: the degree-1 preconditioner's only; strips of two
    # rows: degree 1, which needs two halo rows, not three)
    from paper_2404_02521_gb300 import _lib
    v8 = _lib.bs_coarse_variant_info(8, 256)
    assert v8 == {"ctas": 16, "threads": 256, "rows": 16, "poly": 2, "quad": True}
    v6 = _lib.bs_coarse_variant_info(6, 256)
    assert v6["ctas"] == 8 and v6["poly"] == 1 and not v6["quad"]
    assert _lib.bs_coarse_variant_info(1, 32)["poly"] == 1
    assert _lib.bs_coarse_variant_info(9, 100)["ctas"] == 7
    for bad in [(8, 100), (10, 256), (-1, 64), (0, 300)]:
        with pytest.raises(_lib.BSError):
            _lib.bs_coarse_variant_info(*bad)


def test_three_asset_arguments_are_checked(lib):
    # rejected on the host, before any device work
    import types
    from paper_2404_02521_gb300 import _lib
    ok = types.SimpleNamespace(sigma=(0.3, 0.2, 0.25), rho=(0.5, -0.3, 0.2), r=0.05, strike=1.0,
                               w=(0.4, 0.35, 0.25), payoff=0)
    fake = [1 << 20]
    bad = [
        (3, ok, 0.001), (129, ok, 0.001),
        (16, types.SimpleNamespace(**{**vars(ok), "rho": (0.9, 0.9, -0.9)}), 0.001),   # not positive definite
        (16, types.SimpleNamespace(**{**vars(ok), "payoff": 2}), 0.001),               # one-asset call
        (16, types.SimpleNamespace(**{**vars(ok), "sigma": (0.3, 0.0, 0.2)}), 0.001),
        (64, ok, 1.0),                                                                  # Jacobi bound >= 0.8
    ]
    for M, p, dtau in bad:
        with pytest.raises(_lib.BSError):
            _lib.fine_propagate3(M, 4.0, p, fake, fake, [0.0], dtau, 1, stream=0)
    with pytest.raises(_lib.BSError):
        _lib.fine_propagate3(16, 4.0, ok, [], [], [], 0.001, 1, stream=0)
    # G (BiCGSTAB) takes any step size, but not a bad grid, NULL states or an empty slice
    for M, p, u, dts, ns in [(3, ok, 1 << 20, 0.1, 1), (16, ok, 0, 0.1, 1), (16, ok, 1 << 20, 0.0, 1),
                             (16, ok, 1 << 20, 0.1, 0)]:
        with pytest.raises(_lib.BSError):
            _lib.coarse_propagate3(M, 4.0, p, u, u, 0.0, dts, ns, stream=0)


def test_missing_library_fails_loudly(tmp_path):
    # no CPU fallback: a library that cannot be loaded is an error, not a slower path
    import subprocess
    import sys
    code = ("import paper_2404_02521_gb300._lib as L\n"
            f"L.load({str(tmp_path / 'absent.so')!r})\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=str(ROOT), capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "OSError" in r.stderr
