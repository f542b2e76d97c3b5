"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/fsp.h declares (no GPU needed; only host-side calls are made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fsp.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fsp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def so():
    from paper_1810_11103_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("fsp_metrics", "fsp_rhs", "fsp_rk3_step", "fsp_line_lambda", "fsp_cfl_dt", "fsp_norms",
                 "fsp_workspace_size", "fsp_status_string"):
        assert want in names


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_host_only_calls(so):
    from paper_1810_11103_gb300 import fsp
    L = fsp.lib()
    assert L.fsp_status_string(0) == b"ok"
    assert L.fsp_status_string(1) == b"invalid argument"
    cfg = fsp.Config(scheme=2, bc=(0, 0, 0, 0))
    n = fsp.workspace_size(cfg, 256, 256)
    assert n >= 3 * 4 * 256 * 256 * 8
    b = fsp._block_shape(cfg, 10, 12)
    assert L.fsp_metrics_elems(ctypes.byref(b)) == 5 * 18 * 20
    # argument errors are caught on the host before anything is enqueued
    with pytest.raises(fsp.FspError) as e:
        fsp.workspace_size(fsp.Config(scheme=7), 16, 16)
    assert e.value.code == 1
    with pytest.raises(fsp.FspError):
        fsp.workspace_size(fsp.Config(bc=(0, 1, 0, 0)), 16, 16)   # unpaired periodic face
    with pytest.raises(fsp.FspError):
        fsp.workspace_size(fsp.Config(bc=(1, 1, 1, 1)), 8, 16)    # too few nodes to reflect
