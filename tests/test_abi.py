"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
entry point the header declares, and its host-only calls validate arguments."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amamg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amamg_[a-z_0-9A-Z]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2608_03515_b300 import build
    build.build()
    from paper_2608_03515_b300 import amamg
    return amamg


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    cdll = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(cdll, n)]
    assert not missing, missing
    assert set(names) == set(lib.EXPORTED)


def test_default_params(lib):
    p = lib.default_params()
    assert p.nlevels == 2 and p.agg[0] == 4 and p.restart == 30 and p.post_smooth == 2
    assert p.tol == 1e-10


def test_query_bytes_scales_with_volume_and_rhs(lib):
    p = lib.make_params([4, 2])
    s1, r1 = lib.query_bytes(p, 256, 256, 1)
    s2, r2 = lib.query_bytes(p, 512, 512, 1)
    assert s1 > 0 and r1 > 0
    assert r2 > 3.5 * r1                      # per-RHS bytes grow with the volume
    # the coarsest dense inverse dominates: (2 * 32 * 32)^2 complex128, twice during setup
    assert s1 >= 2 * (2 * 32 * 32) ** 2 * 16
    pm = lib.make_params([4, 2], precision=lib.SOLVE_MIXED)
    _, rm = lib.query_bytes(pm, 256, 256, 1)
    assert rm < r1                            # FP32 flexible basis


@pytest.mark.parametrize("aggs,Nt,Nx", [
    ([3], 24, 24),          # unsupported tile side
    ([4], 12, 10),          # 4 does not divide 10
    ([4], 4, 8),            # fewer than 2 tiles per side
    ([4, 4], 32, 24),       # coarse 8x6 level not divisible by 4 for the 16-colour smoother
    ([2], 256, 256),        # coarsest 128x128 (32768 DOF) too large for the dense inverse
    ([], 16, 16),           # one level only
])
def test_invalid_configurations_are_rejected(lib, aggs, Nt, Nx):
    p = lib.make_params(aggs) if aggs else lib.default_params()
    if not aggs:
        p.nlevels = 1
    with pytest.raises(lib.AmamgError) as ei:
        lib.query_bytes(p, Nt, Nx, 1)
    assert ei.value.status == lib.ERR_INVALID_ARG


def test_status_strings(lib):
    L = lib.lib()
    assert L.amamg_status_string(0) == b"ok"
    assert b"singular" in L.amamg_status_string(lib.ERR_SINGULAR)
    assert L.amamg_launch_count(None) == -1


def test_gram_schmidt_variant_parameters_are_validated(lib):
    """gs_method: classical (default) or modified, the modified one in FP64
    arithmetic only; gs_arith double-float needs the mixed solve."""
    ok = [lib.make_params([4, 2]), lib.make_params([4, 2], gs_method="mgs"),
          lib.make_params([4, 2], precision=lib.SOLVE_MIXED, gs_method="mgs"),
          lib.make_params([4, 2], precision=lib.SOLVE_MIXED, gs="df64")]
    for p in ok:
        lib.query_bytes(p, 64, 64, 1)
    bad = [lib.make_params([4, 2], precision=lib.SOLVE_MIXED, gs="df64", gs_method="mgs"),
           lib.make_params([4, 2], gs="df64")]
    p = lib.make_params([4, 2])
    p.gs_method = 7
    bad.append(p)
    for p in bad:
        with pytest.raises(lib.AmamgError) as ei:
            lib.query_bytes(p, 64, 64, 1)
        assert ei.value.status == lib.ERR_INVALID_ARG
    assert lib.default_params().gs_method == lib.GS_CGS2
