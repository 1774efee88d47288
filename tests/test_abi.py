"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol include/mbo.h and include/mbo_surface.h declare, and argument validation that happens before
any device call rejects bad input with the documented status codes."""
import os
import re

import pytest

from paper_1711_01365_gb300 import build as B
from paper_1711_01365_gb300 import mbo as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = "".join(open(os.path.join(ROOT, "include", f)).read() for f in ("mbo.h", "mbo_surface.h"))
    return sorted(set(re.findall(r"MBO_API\s+[\w\s\*]*?\b(mbo_\w+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.lib()


def test_header_declares_the_expected_entry_points():
    syms = declared_symbols()
    for name in M.EXPORTS + M.SURFACE_EXPORTS:
        assert name in syms
    assert len(syms) >= len(M.EXPORTS) + len(M.SURFACE_EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mbo_\w+)", out))
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(lib, name)


def test_status_strings(lib):
    for code in range(7):
        assert M.mbo_status_string(code)
    assert "unsupported" in M.mbo_status_string(2)


@pytest.mark.parametrize("dims", [(100, 128), (128, 5), (1, 16), (4096, 16), (7, 7, 8), (0, 8)])
def test_unsupported_sizes_rejected(lib, dims):
    with pytest.raises(M.MboError) as ei:
        M.mbo_create(dims, 2, 1e-3)
    assert ei.value.status == 2


@pytest.mark.parametrize("args", [((16, 16), 0, 1e-3), ((16, 16), 5, 1e-3), ((16, 16), 2, 0.0),
                                  ((16, 16), 2, -1.0), ((16,), 2, 1e-3), ((4, 4, 4, 4), 2, 1e-3)])
def test_invalid_arguments_rejected(lib, args):
    with pytest.raises(M.MboError) as ei:
        M.mbo_create(*args)
    assert ei.value.status == 1


def test_null_handle_rejected(lib):
    assert lib.mbo_destroy(None) == 1
    assert lib.mbo_workspace_bytes(None) == 0
    assert lib.mbo_last_error(None) == b""


def test_default_config(lib):
    c = M.mbo_default_config()
    assert c.fallback_sigma == 0.0
    assert c.check_interval == 16 and c.use_graph == 1


def test_timeout_selftest_rejects_bad_arguments_without_a_device(lib):
    # a null handle or a limit outside 1 .. 2e9 cycles is refused before any device call
    assert lib.mbo_selftest_wait_timeout(None, 1000, None) == 1
