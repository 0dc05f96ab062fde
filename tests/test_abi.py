"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point that include/lbm.h and include/lbm3d.h declare, and its
host-only calls validate configurations (no GPU needed)."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("lbm.h", "lbm3d.h")]


@pytest.fixture(scope="module")
def P():
    from paper_1809_06735_gb300 import build
    build.build()
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def declared_symbols():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm(?:3d)?_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_moments",
              "lbm_subvolume_balance", "lbm_adjoint_step", "lbm_subvolume_distributions",
              "lbm3d_create", "lbm3d_step", "lbm3d_subvolume_balance"):
        assert s in syms


def test_library_exports_every_declared_symbol(P):
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lbm(?:3d)?_\w+)", out))
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


def test_3d_config_checks(P):
    """Host-only validation of the 3D configuration."""
    import ctypes
    lib = P.load_library()
    n = ctypes.c_size_t()

    def size(members, precision=32, lattice=0):
        arr = (P._MemberCfg3 * len(members))(*[m.c() for m in members])
        cfg = P._Config3(len(members), arr, precision, 0, None, lattice)
        return lib.lbm3d_workspace_size(ctypes.byref(cfg), ctypes.byref(n))

    assert size([P.Member3(16, 12, 8, 0.6)]) == 0 and n.value > 19 * 4 * 2 * 16 * 12 * 8
    q19 = n.value
    assert size([P.Member3(16, 12, 8, 0.6)], lattice=19) == 0 and n.value == q19
    assert size([P.Member3(16, 12, 8, 0.6)], lattice=27) == 0
    assert n.value - q19 >= 8 * 4 * 2 * 16 * 12 * 8  # two buffers of 8 more populations
    assert size([P.Member3(16, 12, 8, 0.6)], lattice=15) == -1
    arr = (P._MemberCfg3 * 1)(P.Member3(16, 12, 8, 0.6).c())
    for dp, rc in ((0, 0), (32, 0), (64, 0), (16, -1)):
        cfg = P._Config3(1, arr, 32, 0, None, 19, dp)
        assert lib.lbm3d_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == rc, dp
    assert size([P.Member3(16, 12, 8, 0.5)]) == -1
    assert size([P.Member3(0, 12, 8, 0.6)]) == -1
    assert size([P.Member3(8, 8, 8, 0.6, force_kind=2)]) == -1
    assert size([P.Member3(8, 8, 8, 0.6)], precision=16) == -1


_NULL_SWEEP = r"""
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
import paper_1809_06735_gb300 as P
lib = P.load_library()
out = {}
for name in json.loads(sys.argv[2]):
    f = getattr(lib, name)
    if not f.argtypes:
        continue
    args = [0 if t in (ctypes.c_int, ctypes.c_size_t, ctypes.c_longlong) else
            0.0 if t is ctypes.c_double else None for t in f.argtypes]
    r = f(*args)
    out[name] = r.decode() if isinstance(r, bytes) else r
print(json.dumps(out))
"""


def test_null_handles_and_pointers_are_rejected(P):
    """Every entry point called with NULL handles and pointers and zero
    sizes (no GPU work is reached): the argument error -1 from every status
    call, -1 from the value getters, a message from the error getters, and
    destroying NULL is a no-op (0).  Run in a child process."""
    import json
    names = declared_symbols()
    r = subprocess.run([sys.executable, "-c", _NULL_SWEEP, ROOT, json.dumps(names)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(got) >= 30
    for name, v in got.items():
        if name.endswith("last_error"):
            assert v == "handle is NULL", name
        elif name in ("lbm_destroy", "lbm3d_destroy"):
            assert v == 0, name
        else:
            assert v == -1, (name, v)


_STATIC_ARGS = r"""
import ctypes, json, math, sys
sys.path.insert(0, sys.argv[1])
import paper_1809_06735_gb300 as P
lib = P.load_library()
fn = lib.lbm_global_balance_static
fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(P._MemberCfg),
               ctypes.c_void_p, ctypes.c_void_p]
lib.lbm_static_last_error.restype = ctypes.c_char_p
out = (ctypes.c_double * 7)()
fake = ctypes.c_void_p(4096)  # never dereferenced: every case fails before any CUDA call
res = {}
def call(name, f, nx, ny, m, o):
    rc = fn(f, nx, ny, ctypes.byref(m.c()) if m is not None else None, o, None)
    res[name] = [rc, lib.lbm_static_last_error().decode()]
good = P.Member(8, 8, 0.6)
call("f", None, 8, 8, good, out)
call("m", fake, 8, 8, None, out)
call("out", fake, 8, 8, good, None)
call("grid", fake, 0, 8, good, out)
call("size", fake, 1024, 512, good, out)
call("tau_inf", fake, 8, 8, P.Member(8, 8, math.inf), out)
call("tau_half", fake, 8, 8, P.Member(8, 8, 0.5), out)
call("F0_nan", fake, 8, 8, P.Member(8, 8, 0.6, 1.0, 1, 1, math.nan), out)
call("kind2", fake, 8, 8, P.Member(8, 8, 0.6, 1.0, 2), out)
print(json.dumps(res))
"""


def test_static_entry_point_rejects_bad_arguments_before_any_cuda_call(P):
    """lbm_global_balance_static: each NULL pointer, an empty or oversized
    grid and invalid member parameters (tau infinite or not above 1/2, a
    non-finite F0, force kind 2) return -1 with a message naming the fault,
    before any CUDA call (runs without a GPU).  Run in a child process."""
    import json
    r = subprocess.run([sys.executable, "-c", _STATIC_ARGS, ROOT],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    for name, (rc, msg) in got.items():
        assert rc == -1, (name, rc, msg)
    assert got["f"][1] == "f is NULL" and got["m"][1] == "m is NULL"
    assert got["out"][1] == "out is NULL"
    assert "LBM_STATIC_MAX_CELLS" in got["size"][1]
    for name in ("tau_inf", "tau_half", "F0_nan", "kind2"):
        assert got[name][1] == "invalid member parameters", name
