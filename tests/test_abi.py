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


def test_autotune_table_round_trip_without_a_gpu(lib):
    """A saved tuner table loads back (host-only: no device work) and reads out the
    same; a malformed line or an unknown variant is rejected whole."""
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    before = rb.autotune_text()
    rows = ("2 8 70 32 1 513 21.376 4\n"     # l1-Jacobi sweep, FP64, SELL x8 chosen, 4 lanes the best CSR
            "0 4 90 19 1 512 213.195 8\n"    # restriction, FP32, SELL x4
            "1 8 84 3 1 1 35.509 1\n"        # prolongation, 1 lane
            "3 4 52 101 0 260 6.315 260\n")  # residual, 4 lanes x4, no SELL offered
    rb.autotune_load(rows)
    table = rb.autotune_text()
    for line in rows.splitlines():
        assert line in table.splitlines()
    again = rb.autotune_text()
    rb.autotune_load("2 8 70 32 1 2 1.0 2\n")  # an existing class keeps its choice
    assert rb.autotune_text() == again
    for bad in ("2 8 70 32 1 513 21.3\n",          # a field missing
                "2 8 71 32 1 3 1.0 2\n",           # 3 lanes is not a candidate
                "2 8 71 32 0 512 1.0 2\n",         # SELL without a SELL candidate
                "2 8 71 32 1 512 1.0 512\n",       # best CSR variant that is SELL
                "5 8 71 32 1 1 1.0 1\n",           # no such mode
                "2 2 71 32 1 1 1.0 1\n"):          # no such value size
        with pytest.raises(rb.RichError):
            rb.autotune_load(bad)
    assert rb.autotune_text() == again
    assert set(before.splitlines()) <= set(again.splitlines())


def test_sell_layout_host_logic_without_a_gpu(lib):
    """The SELL-C-sigma layout: within each 1024-row window a stable sort by
    decreasing row length, slices of 32 whose width is their first row's length,
    ragged last slice and window padded with -1, slot offsets their running sum."""
    import numpy as np
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    rng = np.random.default_rng(7)
    for n in (2048, 2500, 1, 31, 33, 1025, 3000):
        lens = rng.integers(0, 60, n)
        lens[rng.integers(0, n, max(1, n // 50))] = 0  # empty rows
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        perm, sptr, slots = rb.sell_layout(rp)
        ns = (n + 31) // 32
        assert perm.shape == (32 * ns,) and sptr.shape == (ns + 1,)
        assert np.all(perm[n:] == -1) and sorted(perm[:n]) == list(range(n))
        for w0 in range(0, n, 1024):  # each window is a permutation of its own rows ...
            w = perm[w0:min(n, w0 + 1024)]
            assert sorted(w) == list(range(w0, min(n, w0 + 1024)))
            key = [(-lens[r], r) for r in w]  # ... longest first, ties in row order
            assert key == sorted(key)
        width = [lens[perm[32 * s]] for s in range(ns)]
        assert all(lens[r] <= width[i // 32] for i, r in enumerate(perm[:n]))
        np.testing.assert_array_equal(sptr, np.concatenate([[0], np.cumsum(32 * np.array(width))]))
        assert slots == sptr[-1] >= rp[-1]
    with pytest.raises(rb.RichError):
        rb.sell_layout(np.array([0, 3, 2], dtype=np.int32))  # decreasing row pointer
