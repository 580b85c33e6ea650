"""CPU checks of the C ABI library: it builds for sm_103a, loads without a GPU
and exports every function that include/hard_hydro.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(hard_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_08971_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hard_hydro_create", "hard_hydro_cfl_dt", "hard_hydro_step",
                     "hard_hydro_advance", "hard_hydro_totals", "hard_hydro_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_names_match_header(libpath):
    import paper_2509_08971_gb300 as hh
    missing = [n for n in declared_functions() if not callable(getattr(hh, n, None))]
    assert not missing, missing


def test_host_only_calls_without_gpu(libpath):
    import paper_2509_08971_gb300 as hh
    assert hh.hard_hydro_strerror(hh.HARD_EINVAL) == "invalid argument"
    h = hh.hard_hydro_create(16, 8, 1, 1.4, hh.HARD_BC_OUTFLOW)
    assert h
    assert hh.hard_hydro_tile_count(h) == 3            # a 2D mesh
    rc, info = hh.hard_hydro_tile_info(h, 0)
    assert rc == 0 and info[3] == info[0] * info[1]
    assert hh.hard_hydro_set(h, hh.HARD_F64, 2.0, 1.0, 1.0, None) == hh.HARD_OK
    assert hh.hard_hydro_create(4, 4, 4, 0.5, 0) is None
    # the second scheme needs three cells along every active axis
    assert hh.hard_hydro_set_scheme(h, hh.HARD_SCHEME_WENO5Z_HLL) == hh.HARD_OK
    assert hh.hard_hydro_set_scheme(h, 7) == hh.HARD_EINVAL
    assert hh.hard_hydro_set_scheme(h, hh.HARD_SCHEME_PLM_HLLC) == hh.HARD_OK
    # the exchange checks its arguments before touching the device
    assert hh.hard_hydro_rad_exchange(h, None, None, 1e-3, (1, 1, 1, 1), None) == hh.HARD_EINVAL
    assert hh.hard_hydro_rad_exchange(h, 16, 32, 1e-3, (1, 0, 1, 1), None) == hh.HARD_EINVAL
    assert hh.hard_hydro_rad_exchange(h, 16, 32, -1.0, (1, 1, 1, 1), None) == hh.HARD_EINVAL
    assert hh.hard_hydro_fld_step(h, None, None, 1.0, 1.0, 1.0, 1e-6, 10, None)[0] == hh.HARD_EINVAL
    assert hh.hard_hydro_fld_step(h, 16, 32, 1.0, 1.0, -1.0, 1e-6, 10, None)[0] == hh.HARD_EINVAL
    assert hh.hard_hydro_fld_step(h, 16, 32, 1.0, 1.0, 1.0, 1e-6, 0, None)[0] == hh.HARD_EINVAL
    # more rows than a grid dimension holds: refused before any device work
    hy = hh.hard_hydro_create(4, 70000, 1, 1.4, hh.HARD_BC_OUTFLOW)
    assert hy
    assert hh.hard_hydro_fld_step(hy, 16, 32, 1.0, 1.0, 1.0, 1e-6, 1, None)[0] == hh.HARD_EUNSUPPORTED
    hh.hard_hydro_destroy(hy)
    assert hh.hard_hydro_advect_E(h, None, None, 1.0, None) == hh.HARD_EINVAL
    assert hh.hard_hydro_advect_E(h, 16, 32, 0.0, None) == hh.HARD_EINVAL
    # the split adjoint of a slab checks its arguments before touching the device
    assert hh.hard_hydro_stage_vjp_faces(h, 3, 16, 32, 1e-3, 64, None) == hh.HARD_EINVAL
    assert hh.hard_hydro_stage_vjp_faces(h, 1, None, 32, 1e-3, 64, None) == hh.HARD_EINVAL
    assert hh.hard_hydro_stage_vjp_faces(h, 1, 16, 32, 0.0, 64, None) == hh.HARD_EINVAL
    assert hh.hard_hydro_stage_vjp_cells(h, 1, 16, 32, 48, 0, 64, 80, None) == hh.HARD_EINVAL
    assert hh.hard_hydro_stage_vjp_cells(h, 2, 16, 32, None, 0, None, 80, None) == hh.HARD_EINVAL
    assert hh.hard_hydro_add_zghost_cotangent(h, None, None, None) == hh.HARD_EINVAL  # 2D mesh
    assert hh.hard_hydro_set_zghost_adjoint(h, 17, None) == hh.HARD_EINVAL           # unaligned
    assert hh.hard_hydro_set_zghost_adjoint(h, None, None) == hh.HARD_OK
    h2 = hh.hard_hydro_create(16, 2, 1, 1.4, 0)
    assert hh.hard_hydro_advect_E(h2, 16, 32, 1.0, None) == hh.HARD_EINVAL    # 2 cells along y
    assert hh.hard_hydro_set_scheme(h2, hh.HARD_SCHEME_WENO5Z_HLL) == hh.HARD_EINVAL
    hh.hard_hydro_destroy(h2)
    hh.hard_hydro_destroy(h)


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle and fails loudly without its library."""
    src = open(os.path.join(ROOT, "paper_2509_08971_gb300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src
    assert "no CPU fallback" in src
