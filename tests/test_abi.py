"""CPU checks of the C ABI: the library loads, exports every symbol include/fwi.h declares,
and its host-side planning (workspace sizes) behaves.  No compute call needs a GPU here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fwi.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fwi_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_1804_01184_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:   # no nvcc on this machine
        pytest.skip(str(e))
    return C.CDLL(path)


def test_header_declares_the_operations():
    names = declared()
    for n in ("fwi_model", "fwi_born", "fwi_adjoint", "fwi_gradient", "fwi_workspace_bytes", "fwi_status",
              "fwi_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for n in declared():
        assert hasattr(L, n), n


def test_workspace_planning(L):
    from paper_1804_01184_gb300 import fwi
    fwi._lib = None
    g = fwi.make_grid(601, 601, 5.0, 5e-4, 3000, order=8, sponge=40)
    mn = fwi.fwi_workspace_bytes(g, 64, 256, fwi.OP_GRADIENT, 0)
    big = fwi.fwi_workspace_bytes(g, 64, 256, fwi.OP_GRADIENT, 1 << 50)
    assert mn < big
    Np = 704 * 681 * 4
    # the whole history of all 64 shots: 3001 snapshot slots of 64 fields
    assert big >= 3001 * 64 * Np
    mid = fwi.fwi_workspace_bytes(g, 64, 256, fwi.OP_GRADIENT, 150 << 30)
    assert mn <= mid <= 150 << 30
    # forward only needs the model and the ping-ponged state (2 x p, vx, vz) of every shot
    m = fwi.fwi_workspace_bytes(g, 64, 256, fwi.OP_MODEL, 1 << 50)
    assert 6 * 64 * Np <= m <= 7 * 64 * Np + (64 << 20)
    # invalid arguments -> 0 -> error
    bad = fwi.make_grid(601, 601, 5.0, 5e-4, 3000, order=6)
    with pytest.raises(fwi.FwiError):
        fwi.fwi_workspace_bytes(bad, 1, 1, fwi.OP_MODEL, 0)


def test_fborn_workspace_planning(L):
    from paper_1804_01184_gb300 import fborn, fwi
    fwi._lib = None
    fborn._bound = False
    fg = fborn.make_fgrid(121, 121, 60, 5.0, -300.0, -300.0)
    n = fborn.fwi_fborn_workspace_bytes(fg, 10, 100)
    rows = (121 * 121 + 127) // 128 * 128      # table rows padded to 128 nodes
    tables = 2 * 60 * 110 * rows * 8
    chunks = (121 * 121 + 255) // 256
    freq_partials = 60 * 6 * 121 * 121 * 8      # gradient [nf][2][N], Hessian [nf][4][N]
    contrasts = 2 * rows * 4                   # FP32 contrasts of the data contraction
    assert tables <= n <= tables + (chunks + 3) * 60 * 10 * 100 * 8 + freq_partials + contrasts + (1 << 16)
    with pytest.raises(fwi.FwiError):
        fborn.fwi_fborn_workspace_bytes(fborn.make_fgrid(121, 121, 0, 5.0, 0.0, 0.0), 10, 100)
    with pytest.raises(fwi.FwiError):
        fborn.fwi_fborn_workspace_bytes(fg, 0, 100)
