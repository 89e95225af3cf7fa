"""C-ABI checks that need no GPU: the library loads, exports every entry
point that include/nekgb.h declares, and rejects bad arguments before doing
any device work.  Host-side fault injection (NEKGB_FAIL_ALLOC) exercises the
out-of-memory path without touching a GPU."""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nekgb.h")


@pytest.fixture(scope="module")
def nek():
    from paper_2005_13425_gb300 import build as b
    b.build()
    from paper_2005_13425_gb300 import nekgb
    nekgb.load()
    return nekgb


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_are_exported(nek):
    lib = nek.load()
    decl = declared_functions()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib, name), f"{name} declared in nekgb.h but not exported"
    # and the binding covers every declared entry point
    assert set(decl) == set(nek.exported_symbols())


def test_status_strings(nek):
    assert nek.nb_status_str(0) == "NB_OK"
    assert nek.nb_status_str(5) == "NB_ERR_BREAKDOWN"
    assert nek.nb_status_str(99) == "NB_UNKNOWN"


@pytest.mark.parametrize("mesh,n", [((2, 2, 2), 1), ((2, 2, 2), 17), ((0, 2, 2), 4), ((2, -1, 2), 4)])
def test_setup_rejects_bad_sizes(nek, mesh, n):
    D = np.zeros((max(n, 1), max(n, 1)))
    g = np.zeros(10)
    with pytest.raises(nek.NekgbError) as ei:
        nek.nb_setup(mesh, n, D, g)
    assert ei.value.status == nek.NB_ERR_ARG
    assert nek.nb_last_error()


def test_setup_rejects_missing_arrays(nek):
    lib = nek.load()
    import ctypes
    ctx = ctypes.c_void_p()
    st = lib.nb_setup(ctypes.byref(ctx), nek.nb_box(2, 2, 2), 4, None, None, None, 0, None)
    assert st == nek.NB_ERR_ARG and not ctx.value
    st = lib.nb_setup_box(ctypes.byref(ctx), nek.nb_box(2, 2, 2), 4, 0.05, None, 0, None)
    assert st == nek.NB_ERR_ARG
    st = lib.nb_setup(ctypes.byref(ctx), nek.nb_box(2, 2, 2), 4, np.zeros(16).ctypes.data,
                      np.zeros(8 * 6 * 64).ctypes.data, None, 7, None)
    assert st == nek.NB_ERR_ARG            # unknown precision


def test_null_context_calls(nek):
    lib = nek.load()
    assert lib.nb_ax(None, None, None) == nek.NB_ERR_ARG
    assert lib.nb_dssum(None, None) == nek.NB_ERR_ARG
    assert lib.nb_cg_solve(None, None, None, 0.0, 1, None, None) == nek.NB_ERR_ARG
    assert lib.nb_destroy(None) == nek.NB_OK


def test_injected_allocation_failure_is_reported():
    """NEKGB_FAIL_ALLOC=1 fails the first device allocation of the process
    on the host, before any CUDA call: nb_setup must return NB_ERR_OOM and
    leave no context behind."""
    code = (
        "import numpy as np, ctypes\n"
        "from paper_2005_13425_gb300 import nekgb as k\n"
        "lib = k.load(); ctx = ctypes.c_void_p()\n"
        "D = np.zeros((4, 4)); g = np.zeros(8 * 6 * 64)\n"
        "st = lib.nb_setup(ctypes.byref(ctx), k.nb_box(2, 2, 2), 4, D.ctypes.data, g.ctypes.data, None, 0, None)\n"
        "print(st, ctx.value, lib.nb_last_error().decode())\n"
    )
    env = dict(os.environ, NEKGB_FAIL_ALLOC="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    st, ctxv, msg = r.stdout.strip().split(" ", 2)
    assert int(st) == 3 and ctxv == "None" and "alloc" in msg


def test_engine_footprint_host_arithmetic(nek):
    """Admission footprint (host-only): gxyz pairs and four FP64 CG vectors
    (80 B per local point) for FP64 requests; FP64 and FP32 gxyz, three FP64
    and four FP32 vectors (112 B per point) for mixed ones; plus the tile
    partials, a small remainder.  Bad arguments are rejected."""
    for dims, n in [((16, 16, 16), 10), ((4, 4, 4), 8), ((8, 4, 2), 6), ((1, 1, 1), 2)]:
        E = dims[0] * dims[1] * dims[2]
        npts = E * n ** 3
        f64 = nek.nb_engine_footprint(dims, n, nek.NB_FP64)
        mix = nek.nb_engine_footprint(dims, n, nek.NB_MIXED)
        assert 80 * npts <= f64 <= 80 * npts + 16 * E + 4096
        assert 112 * npts <= mix <= 112 * npts + 16 * E + 4096
    small = nek.nb_engine_footprint((8, 8, 8), 10, nek.NB_FP64)
    assert nek.nb_engine_footprint((16, 8, 8), 10, nek.NB_FP64) > small
    for bad in [((0, 1, 1), 10, nek.NB_FP64), ((2, 2, 2), 1, nek.NB_FP64), ((2, 2, 2), 17, nek.NB_FP64),
                ((2, 2, 2), 8, 7)]:
        with pytest.raises(nek.NekgbError) as ei:
            nek.nb_engine_footprint(*bad)
        assert ei.value.status == nek.NB_ERR_ARG
