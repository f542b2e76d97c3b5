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


def _ws_code(fsp, cfg, ni, nj, ld=None):
    b = fsp._block_shape(cfg, ni, nj, ld)
    n = ctypes.c_size_t()
    return fsp.lib().fsp_workspace_size(ctypes.byref(cfg._c()), ctypes.byref(b), ctypes.byref(n))


def test_argument_validation_on_the_host(so):
    # every case is refused before anything touches the device (no GPU needed)
    from paper_1810_11103_gb300 import fsp
    per = fsp.Config(scheme=2, bc=(0, 0, 0, 0))
    wall = fsp.Config(scheme=2, bc=(3, 3, 1, 1))
    assert _ws_code(fsp, per, 1, 1) == 0                   # a single periodic node is a valid block
    assert _ws_code(fsp, per, 0, 16) == 1                  # empty
    assert _ws_code(fsp, per, 16, 0) == 1
    assert _ws_code(fsp, per, 16, 16, ld=15) == 1          # row stride below the row length
    assert _ws_code(fsp, wall, 9, 9) == 0                  # smallest non-periodic extent
    assert _ws_code(fsp, wall, 8, 9) == 1
    assert _ws_code(fsp, wall, 9, 8) == 1
    assert _ws_code(fsp, fsp.Config(scheme=2, bc=(0, 1, 0, 0)), 16, 16) == 1   # unpaired periodic face
    assert _ws_code(fsp, per, 8 * 65535, 9) == 0           # the longest lines the sweep grids allow
    assert _ws_code(fsp, per, 8 * 65535 + 1, 9) == 1
    assert _ws_code(fsp, per, 9, 2 * 65535) == 0
    assert _ws_code(fsp, per, 9, 2 * 65535 + 1) == 1
    for bad in (dict(gamma=1.0), dict(lf_alpha=0.0), dict(eps=0.0), dict(interp=2), dict(precision=3),
                dict(bc=(6, 6, 0, 0))):
        assert _ws_code(fsp, fsp.Config(**dict(dict(scheme=2, bc=(0, 0, 0, 0)), **bad)), 16, 16) == 1, bad
    # the adjoint is FP64 only
    b = fsp._block_shape(per, 16, 16)
    n = ctypes.c_size_t()
    c32 = fsp.Config(scheme=2, bc=(0, 0, 0, 0), precision=1)
    assert fsp.lib().fsp_vjp_workspace_size(ctypes.byref(c32._c()), ctypes.byref(b), ctypes.byref(n)) == 2
    assert fsp.lib().fsp_rk3_tape_size(ctypes.byref(c32._c()), ctypes.byref(b), ctypes.byref(n)) == 2
    # ... covers WENOIU7-1MP, and refuses the options beyond the printed schemes
    c7 = fsp.Config(scheme=4, bc=(0, 0, 0, 0))
    assert _ws_code(fsp, c7, 16, 16) == 0
    assert fsp.lib().fsp_vjp_workspace_size(ctypes.byref(c7._c()), ctypes.byref(b), ctypes.byref(n)) == 0
    assert fsp.lib().fsp_rk3_tape_size(ctypes.byref(c7._c()), ctypes.byref(b), ctypes.byref(n)) == 0
    for opt in (dict(weights=1), dict(mid_split=2), dict(scheme_alpha=1.2)):
        co = fsp.Config(**dict(dict(scheme=2, bc=(0, 0, 0, 0)), **opt))
        assert _ws_code(fsp, co, 16, 16) == 0
        assert fsp.lib().fsp_vjp_workspace_size(ctypes.byref(co._c()), ctypes.byref(b), ctypes.byref(n)) == 2
    assert _ws_code(fsp, fsp.Config(scheme=6, bc=(0, 0, 0, 0)), 16, 16) == 1
    # WENOIU7-4MP: periodic blocks only, one precision
    assert _ws_code(fsp, fsp.Config(scheme=5, bc=(0, 0, 0, 0)), 16, 16) == 0
    assert _ws_code(fsp, fsp.Config(scheme=5, bc=(1, 1, 0, 0)), 16, 16) == 2
    assert _ws_code(fsp, fsp.Config(scheme=5, bc=(0, 0, 0, 0), precision=2), 16, 16) == 2
    # the state check refuses a host pointer for its result
    one = (ctypes.c_longlong * 1)()
    assert fsp.lib().fsp_check_state(ctypes.byref(per._c()), ctypes.byref(b), None, one, None) == 1
    # null and host pointers are refused
    assert fsp.lib().fsp_rhs(ctypes.byref(per._c()), ctypes.byref(b), None, None, None, None, 0, None) == 1
    host = (ctypes.c_double * 4096)()
    hp = ctypes.cast(host, ctypes.c_void_p)
    assert fsp.lib().fsp_rhs(ctypes.byref(per._c()), ctypes.byref(b), hp, hp, hp, hp, 1 << 20, None) == 1


def test_batch_argument_validation_on_the_host(so):
    from paper_1810_11103_gb300 import fsp
    L = fsp.lib()
    cfg = fsp.Config(scheme=2)
    h = ctypes.c_void_p()
    blk = (fsp._Block * 2)(fsp._block_shape(cfg, 16, 16), fsp._block_shape(cfg, 16, 16))
    links = (fsp._Link * 8)()
    ok_bc = (ctypes.c_int * 8)(1, 1, 1, 1, 1, 1, 1, 1)
    assert L.fsp_batch_create(ctypes.byref(cfg._c()), 0, blk, ok_bc, links, ctypes.byref(h)) == 1   # no blocks
    bad = (ctypes.c_int * 8)(5, 1, 1, 1, 1, 1, 1, 1)       # a link to a block that does not exist
    links[0].nbr = 7
    assert L.fsp_batch_create(ctypes.byref(cfg._c()), 2, blk, bad, links, ctypes.byref(h)) == 1
    links[0].nbr, links[0].face = 1, 1                      # a link whose faces do not match in length
    blk[1] = fsp._block_shape(cfg, 16, 12)
    assert L.fsp_batch_create(ctypes.byref(cfg._c()), 2, blk, bad, links, ctypes.byref(h)) == 1
    assert not h.value
    assert L.fsp_batch_rk3_step_host(None, None, None, 1e-3, None) == 1     # no handle


def _prototypes():
    """name -> list of parameter declarations, from the header's prototypes."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(fsp_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", text):
        params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(1)] = params
    return out


def test_binding_argument_lists_match_the_header(so):
    from paper_1810_11103_gb300 import fsp
    L = fsp.lib()
    scalar = {"int": ctypes.c_int, "double": ctypes.c_double, "long long": ctypes.c_longlong,
              "size_t": ctypes.c_size_t}
    checked = 0
    for name, params in _prototypes().items():
        f = getattr(L, name)
        if f.argtypes is None:      # not used by the binding
            continue
        assert len(f.argtypes) == len(params), (name, params, f.argtypes)
        for decl, t in zip(params, f.argtypes):
            if "*" in decl:
                assert t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer), (name, decl, t)
            else:
                base = re.sub(r"\b(const)\b", "", decl).rsplit(None, 1)[0].strip()
                if base in scalar:
                    assert t is scalar[base], (name, decl, t)
        checked += 1
    assert checked >= 30
