"""The C ABI library loads and exports every symbol declared in
include/pecann.h; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2312_03940_gb300 import build as pbuild
from paper_2312_03940_gb300 import pecann as pc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    try:
        path = pbuild.build()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    return pc.load_library(path)


def declared_symbols():
    with open(os.path.join(ROOT, "include", "pecann.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"PECANN_API[^;]*?\b(pecann_\w+)\s*\(", text, re.S)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == sorted(pc.EXPORTS)


def test_params_default_and_strings(lib):
    p = pc.params()
    assert (p.k, p.R, p.L_search, p.dep_threshold, p.max_dep_beam) == (16, 32, 64, 300, 8192)
    assert abs(p.alpha - 1.1) < 1e-6 and abs(p.batch_frac - 0.02) < 1e-7
    assert lib.pecann_status_string(pc.EINVAL) == b"invalid argument"
    assert lib.pecann_version() >= 100


def test_struct_layout_matches_header(lib):
    # pecann_params: 24 four-byte fields, then a uint64 -> 104 bytes
    assert ctypes.sizeof(pc.PecannParams) == 104
    assert ctypes.sizeof(pc.PecannDataset) == 48
    assert ctypes.sizeof(pc.PecannClusterSetting) == 16


def test_invalid_arguments_rejected_on_host(lib):
    p = pc.params()
    ds = pc.PecannDataset(None, 100, 32, pc.F32, pc.L2, 0, None, None)
    st = lib.pecann_density(ctypes.byref(ds), None, ctypes.byref(p), None, None, None, None, None, 0, None)
    assert st == pc.EINVAL
    assert b"NULL" in lib.pecann_last_error()
    # misaligned rows, bad d, bad dtype: all caught before any GPU work
    ds = pc.PecannDataset(8, 100, 32, pc.F32, pc.L2, 0, None, None)
    assert lib.pecann_density(ctypes.byref(ds), None, ctypes.byref(p), None, None, None, None, None, 0,
                              None) == pc.EINVAL
    ds = pc.PecannDataset(256, 100, 30, pc.F32, pc.L2, 0, None, None)
    assert lib.pecann_search(ctypes.byref(ds), None, 8, None, 0, None, 0, 8, 4, None, None, None, None, None, 0,
                             None) == pc.EINVAL
    ds = pc.PecannDataset(256, 100, 512, pc.U8, pc.L2, 0, None, None)
    g = ctypes.c_void_p(256)
    st = lib.pecann_search(ctypes.byref(ds), g, 8, g, 1, None, 0, 8, 4, g, g, g, None, g, 1 << 20, None)
    assert st == pc.EUNSUPPORTED


def test_workspace_size_is_host_only(lib):
    p = pc.params(R=64, L_build=128)
    ds = pc.PecannDataset(256, 1_000_000, 128, pc.U8, pc.L2, 0, None, None)
    b = ctypes.c_size_t(0)
    assert lib.pecann_workspace_size(ctypes.byref(ds), ctypes.byref(p), ctypes.byref(b)) == pc.OK
    assert 16 * 1_000_000 < b.value < 1 << 31


def test_cluster_sweep_checks_on_host(lib):
    """Workspace sizing and every setting check answer on the host (the fake
    device pointers below are never dereferenced)."""
    b = ctypes.c_size_t(0)
    assert lib.pecann_cluster_workspace_size(1000, 3, ctypes.byref(b)) == pc.OK and b.value >= 1000 * 8 + 3 * 8
    assert lib.pecann_cluster_workspace_size(0, 3, ctypes.byref(b)) == pc.EINVAL
    assert lib.pecann_cluster_workspace_size(1000, 0, ctypes.byref(b)) == pc.EINVAL
    fake = ctypes.c_void_p(256)

    def sweep(settings, knn=None, k=0, rk=None):
        arr = (pc.PecannClusterSetting * len(settings))(*settings)
        return lib.pecann_cluster_sweep(1000, fake, fake, fake, knn, k, rk, len(settings), arr, fake, None, fake,
                                        1 << 30, None)

    S = pc.PecannClusterSetting
    assert sweep([S(7, 0.0, 0.0, 1)]) == pc.EINVAL                      # unknown center function
    assert sweep([S(pc.CENTER_PRODUCT, 0.0, 0.0, 0)]) == pc.EINVAL      # n_clusters < 1
    assert sweep([S(pc.CENTER_LOCAL, 0.0, 0.0, 1)]) == pc.EINVAL        # local center without k-NN lists
    assert b"local center" in lib.pecann_last_error()


def test_small_workspace_is_enomem_on_host(lib):
    """A workspace below what the call needs is PECANN_ENOMEM, answered on the
    host before any GPU work (this machine has no GPU: a CUDA call would turn
    the status into ECUDA)."""
    p = pc.params(k=4, R=8, L_search=8, L_dep=8, n_clusters=2)
    ds = pc.PecannDataset(256, 1000, 32, pc.F32, pc.L2, 0, None, None)
    g = ctypes.c_void_p(256)
    assert lib.pecann_density(ctypes.byref(ds), g, ctypes.byref(p), g, g, g, g, g, 64, None) == pc.ENOMEM
    assert lib.pecann_dependent_points(ctypes.byref(ds), g, ctypes.byref(p), g, g, g, g, g, None, g, 64,
                                       None) == pc.ENOMEM
    assert lib.pecann_cluster(1000, g, g, g, ctypes.byref(p), g, None, g, 64, None) == pc.ENOMEM
    S = pc.PecannClusterSetting
    arr = (S * 1)(S(pc.CENTER_THRESHOLD, 0.0, 1.0, 1))
    assert lib.pecann_cluster_sweep(1000, g, g, g, None, 0, None, 1, arr, g, None, g, 64, None) == pc.ENOMEM
    assert b"workspace too small" in lib.pecann_last_error()


def test_header_is_plain_c_and_links(lib, tmp_path):
    """tests/c_abi_example.c includes include/pecann.h as C99 (-Wall -Werror),
    links the shared library and calls host-only entry points."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(pbuild.LIB)
    exe = str(tmp_path / "c_abi_example")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_example.c"), "-L", libdir, "-lpecann",
                        "-Wl,-rpath," + libdir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "workspace ok" in r.stdout and "bad center function" in r.stdout


def test_nndescent_checks_on_host(lib):
    """NN-Descent workspace sizing, argument checks and a short workspace
    answer on the host (fake device pointers, never dereferenced)."""
    p = pc.params(R=24, alpha=1.2)
    ds = pc.PecannDataset(256, 100_000, 128, pc.U8, pc.L2, 0, None, None)
    b = ctypes.c_size_t(0)
    assert lib.pecann_nndescent_workspace_size(ctypes.byref(ds), ctypes.byref(p), 16, 2, ctypes.byref(b)) == pc.OK
    # at least the two list buffers, the reverse keys and both repeats' lists
    assert b.value >= 100_000 * 16 * (4 * 4 + 8 + 2 * 4 * 2)
    for K, reps in ((0, 1), (65, 1), (16, 0), (16, 65)):
        assert lib.pecann_nndescent_workspace_size(ctypes.byref(ds), ctypes.byref(p), K, reps,
                                                   ctypes.byref(b)) == pc.EINVAL
    g = ctypes.c_void_p(256)
    call = lib.pecann_build_nndescent
    assert call(ctypes.byref(ds), ctypes.byref(p), 16, 1, None, 5, g, None, None, None, g, 1 << 40, None) == pc.EINVAL
    assert call(ctypes.byref(ds), ctypes.byref(p), 16, 1, g, -1, g, None, None, None, g, 1 << 40, None) == pc.EINVAL
    bad = pc.params(R=24, alpha=0.9)
    assert call(ctypes.byref(ds), ctypes.byref(bad), 16, 1, g, 5, g, None, None, None, g, 1 << 40, None) == pc.EINVAL
    assert call(ctypes.byref(ds), ctypes.byref(p), 16, 1, g, 5, g, None, None, None, g, 64, None) == pc.ENOMEM


def test_hcnng_checks_on_host(lib):
    """HCNNG workspace sizing and argument checks answer on the host."""
    p = pc.params(R=32, alpha=1.2)
    ds = pc.PecannDataset(256, 100_000, 128, pc.U8, pc.L2, 0, None, None)
    b = ctypes.c_size_t(0)
    assert lib.pecann_hcnng_workspace_size(ctypes.byref(ds), ctypes.byref(p), 3, 200, 3, ctypes.byref(b)) == pc.OK
    assert b.value >= 100_000 * (4 * 4 + 2 * 9 * 4)  # orders, flags and both candidate arrays
    for reps, leaf, deg in ((0, 200, 3), (3, 201, 3), (3, 1, 3), (3, 200, 17)):
        assert lib.pecann_hcnng_workspace_size(ctypes.byref(ds), ctypes.byref(p), reps, leaf, deg,
                                               ctypes.byref(b)) == pc.EINVAL
    g = ctypes.c_void_p(256)
    call = lib.pecann_build_hcnng
    assert call(ctypes.byref(ds), ctypes.byref(p), 3, 200, 3, None, None, None, g, 1 << 40, None) == pc.EINVAL
    assert call(ctypes.byref(ds), ctypes.byref(p), 3, 200, 3, g, None, None, g, 64, None) == pc.ENOMEM


def test_cluster_workspace_size_covers_the_single_setting_call(lib):
    """pecann_cluster accepts a workspace of pecann_cluster_workspace_size(n, 1)
    bytes (answered on the host: past the size check the call needs a GPU)."""
    p = pc.params(n_clusters=3)
    g = ctypes.c_void_p(256)
    for n in (10, 1000, 1_000_000):
        b = ctypes.c_size_t(0)
        assert lib.pecann_cluster_workspace_size(n, 1, ctypes.byref(b)) == pc.OK
        assert lib.pecann_cluster(n, g, g, g, ctypes.byref(p), g, None, g, b.value, None) != pc.ENOMEM
        assert lib.pecann_cluster(n, g, g, g, ctypes.byref(p), g, None, g, 64, None) == pc.ENOMEM
