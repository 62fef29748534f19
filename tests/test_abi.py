"""The C-ABI library builds, loads without a GPU and exports every function include/richards.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "richards.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_05051_gb300 import build, richards
    if not os.path.exists(richards.LIB_PATH):
        build.build()
    return ctypes.CDLL(richards.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rich_create", "rich_destroy", "rich_residual", "rich_jacobian", "amg_setup",
                     "krylov_solve", "rich_step"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2112_05051_gb300 import richards
    assert set(richards.EXPORTS) <= set(_declared())


def test_host_only_calls_work_without_a_gpu(lib):
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    o = rb.default_newton_opts()
    assert o.rtol == 1e-8 and o.krylov.eta == 1e-7 and o.krylov.maxit == 200 and o.amg.theta == 0.08
    lib.rich_strerror.restype = ctypes.c_char_p
    assert lib.rich_strerror(-4) == b"Krylov solver did not converge"
    # argument validation happens before any device work
    assert lib.rich_create(None, None, 0, None, 0, None, None) == -1


def test_server_options_and_argument_checks_without_a_gpu(lib):
    import ctypes as C
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    o = rb.default_server_opts()
    assert o.slots == 8 and o.mem_budget_bytes == 0.0 and o.max_sessions == 64
    h = C.c_void_p()
    bad = rb.default_server_opts(slots=0)
    assert lib.rich_server_create(C.byref(bad), C.byref(h)) == -1 and not h.value
    assert lib.rich_server_submit(None, None, None) == -1
    assert lib.rich_server_poll(None, 1, None) == -1
    assert lib.rich_server_destroy(None) == 0
