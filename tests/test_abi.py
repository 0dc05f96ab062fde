"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point that include/lbm.h declares, and its host-only calls
validate configurations (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def P():
    from paper_1809_06735_gb300 import build
    build.build()
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_moments",
              "lbm_subvolume_balance", "lbm_adjoint_step"):
        assert s in syms


def test_library_exports_every_declared_symbol(P):
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    lib = P.load_library()
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_workspace_size_validates(P):
    ok = [P.Member(64, 64, 0.6)]
    n1 = P.workspace_size(ok, 32)
    n2 = P.workspace_size(ok * 2, 32)
    assert n2 > n1 > 0
    assert P.workspace_size(ok, 64) > n1
    with pytest.raises(P.LBMError) as e:
        P.workspace_size([P.Member(64, 64, 0.5)], 32)
    assert e.value.code == -1 and "tau" in str(e.value)
    with pytest.raises(P.LBMError):
        P.workspace_size([P.Member(0, 64, 0.6)], 32)
    with pytest.raises(P.LBMError):
        P.workspace_size(ok, 16)
    with pytest.raises(P.LBMError):
        P.workspace_size([P.Member(8, 8, 0.6, force_kind=3)], 32)
    with pytest.raises(P.LBMError):
        P.workspace_size([P.Member(8, 8, 0.6, collision=4)], 32)
    with pytest.raises(P.LBMError):
        P.workspace_size([P.Member(8, 8, 0.6, collision=1, Cs=-0.1)], 32)
    with pytest.raises(P.LBMError):
        P.workspace_size([P.Member(8, 8, 0.6, force_kind=2, FR0=float("nan"))], 32)


def test_workspace_scales_with_grid(P):
    """Population storage dominates: 2 buffers x 9 x 4 B per cell (FP32),
    plus the FP64 snapshot ring and diagnostic scratch."""
    small = P.workspace_size([P.Member(512, 512, 0.52)], 32)
    big = P.workspace_size([P.Member(1024, 1024, 0.52)], 32)
    assert 3.5 < big / small < 4.5
