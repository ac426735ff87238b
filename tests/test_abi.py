"""The C-ABI library builds, loads and exports what include/*.h declares, and
rejects bad arguments on the host before touching a GPU (CPU only)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_2004_13653_gb300 as kde
from paper_2004_13653_gb300 import build as kbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return kde.load()


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(kde_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_binding_exports():
    declared = _declared_functions()
    assert set(kde.EXPORTS) <= declared


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", kbuild.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = _declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_built_for_sm_103a_only():
    src = open(kbuild.__file__).read()
    assert "arch=compute_103a,code=sm_103a" in src
    assert kbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version(lib):
    assert "sm_103a" in kde.version()


def _args(**kw):
    base = dict(points=None, weights=None, n=0, origin_x=0.0, origin_y=0.0, cell=1.0, nx=4, ny=4,
                h=1.0, kernel_id=6, out=None)
    base.update(kw)
    return kde.KdeArgs(**base)


BAD = [
    ("negative n", dict(n=-1, out=8)),
    ("null points", dict(n=5, out=8)),
    ("null out", dict(n=0)),
    ("empty grid", dict(nx=0, out=8)),
    ("grid overflow", dict(nx=65536, ny=32768, out=8)),
    ("zero h", dict(h=0.0, out=8)),
    ("nan h", dict(h=float("nan"), out=8)),
    ("inf h", dict(h=float("inf"), out=8)),
    ("zero cell", dict(cell=0.0, out=8)),
    ("nan origin", dict(origin_x=float("nan"), out=8)),
    ("kernel id", dict(kernel_id=16, out=8)),
    ("negative kernel id", dict(kernel_id=-1, out=8)),
]


@pytest.mark.parametrize("name,kw", BAD, ids=[b[0] for b in BAD])
def test_invalid_arguments_rejected_on_host(lib, name, kw):
    a = _args(**kw)
    rc = lib.kde_grid_ex(ctypes.byref(a), None)
    assert rc == kde.KDE_EINVAL, (name, rc)
    assert lib.kde_last_error().decode()


def test_tensor_path_needs_gaussian(lib):
    a = _args(kernel_id=2, out=8)
    for path in ("tc_fp16", "tc_split16"):
        o = kde.make_opts(path=path)
        assert lib.kde_grid_ex(ctypes.byref(a), ctypes.byref(o)) == kde.KDE_ENOTSUP


@pytest.mark.parametrize("field,value", [("path", 9), ("split_k", -1), ("k_chunk", 100),
                                         ("k_chunk", 64), ("tile_n", 96)])
def test_invalid_options_rejected(lib, field, value):
    a = _args(out=8)
    o = kde.make_opts()
    setattr(o, field, value)
    assert lib.kde_grid_ex(ctypes.byref(a), ctypes.byref(o)) == kde.KDE_EINVAL


def test_plain_entry_rejects_null_origin(lib):
    rc = lib.kde_grid(None, None, 0, None, 1.0, 4, 4, 1.0, 6, 8)
    assert rc == kde.KDE_EINVAL


def test_mercator_rejects_bad_arguments(lib):
    assert lib.kde_project_mercator(None, -1, 0.0, None, None) == kde.KDE_EINVAL
    assert lib.kde_project_mercator(8, 1, 95.0, 8, None) == kde.KDE_EINVAL
    assert lib.kde_project_mercator(None, 0, 30.0, None, None) == kde.KDE_OK


def _noalloc(lib, n, kernel_id=6, nx=4, ny=4):
    org = (ctypes.c_double * 2)(0.0, 0.0)
    # fake, aligned non-null addresses: the call must refuse before it touches them
    return lib.kde_grid_noalloc(4096, None, n, ctypes.byref(org), 1.0, nx, ny, 1.0, kernel_id,
                                4096, None)


@pytest.mark.parametrize("n", [2 ** 62, 2 ** 60 + 1, (8 << 20) // 20 + 1])
def test_noalloc_rejects_point_counts_beyond_its_scratch_on_host(lib, n):
    # 2^62 points: 16 n and 4 n are 0 modulo 2^64, so a size computed before the
    # count is bounded would wrap around to a small number and pass
    assert _noalloc(lib, n) == kde.KDE_EINVAL
    assert "static maximum" in lib.kde_last_error().decode()


def test_noalloc_rejects_a_grid_that_leaves_no_room_on_host(lib):
    assert _noalloc(lib, 1000, nx=1 << 20, ny=1) == kde.KDE_EINVAL
    assert "static maximum" in lib.kde_last_error().decode()


def test_noalloc_kernel_ids_on_host(lib):
    # the radial Gaussian (14) is the product Gaussian and passes the kernel
    # check (the oversized count stops it next); radial compact kernels do not
    assert _noalloc(lib, 2 ** 62, kernel_id=14) == kde.KDE_EINVAL
    assert "static maximum" in lib.kde_last_error().decode()
    for kid in (10, 15, 16, -1):
        assert _noalloc(lib, 10, kernel_id=kid) == kde.KDE_EINVAL
        assert "kernel_id" in lib.kde_last_error().decode()
