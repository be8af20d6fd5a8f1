"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no GPU needed: only host-side calls are made)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2403_12820_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|size_t|int32_t|int64_t)\s*\*?\s*(\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cloth_create", "cloth_step_plain", "cloth_rollout_plain", "cloth_forces",
                     "cloth_set_state", "cloth_get_state", "cloth_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_workspace_size_host_only():
    lib = _lib.load()
    g = (_lib.ClothGrid * 2)(_lib.ClothGrid(32, 32, 0.02, 1e-3), _lib.ClothGrid(5, 7, 0.02, 1e-3))
    n = ctypes.c_size_t()
    assert lib.cloth_workspace_size(2, g, ctypes.byref(n)) == 0
    # two double-buffered copies of 6 float planes per node at least
    assert n.value >= 2 * 6 * 4 * (32 * 32 + 5 * 7)
    bad = (_lib.ClothGrid * 1)(_lib.ClothGrid(0, 7, 0.02, 1e-3))
    assert lib.cloth_workspace_size(1, bad, ctypes.byref(n)) == -1
    assert lib.cloth_workspace_size(0, g, ctypes.byref(n)) == -1


def test_strerror_and_codes():
    lib = _lib.load()
    assert lib.cloth_strerror(0) == b"ok"
    assert b"workspace" in lib.cloth_strerror(-2)


def test_create_rejects_bad_arguments_before_touching_the_device():
    lib = _lib.load()
    g = (_lib.ClothGrid * 1)(_lib.ClothGrid(4, 4, 0.02, 1e-3))
    p = (_lib.ClothParams * 1)()
    h = ctypes.c_void_p()
    # NULL workspace, non-positive dt, too-small workspace are refused on the host
    assert lib.cloth_create(ctypes.byref(h), 1, g, p, None, None, ctypes.c_float(1e-4), None, 0, None) == -1
    assert lib.cloth_create(ctypes.byref(h), 1, g, p, None, None, ctypes.c_float(0.0), ctypes.c_void_p(256), 1 << 20, None) == -1
    assert lib.cloth_create(ctypes.byref(h), 1, g, p, None, None, ctypes.c_float(1e-4), ctypes.c_void_p(256), 16, None) == -2


def test_missing_library_and_toolchain_fail_loudly(tmp_path, monkeypatch):
    """No CPU fallback: with no built library and no nvcc, loading raises."""
    from paper_2403_12820_gb300 import build as bld

    def no_nvcc():
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcloth")

    monkeypatch.setattr(bld, "LIB", str(tmp_path / "libcloth.so"))
    monkeypatch.setattr(bld, "_nvcc", no_nvcc)
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="nvcc not found"):
        _lib.load()
    with pytest.raises(RuntimeError, match="not found"):
        _lib.load(build_if_needed=False)


def test_static_forward_cuda_failure_is_reported_by_cloth_last_cuda_error():
    """With no CUDA device visible, net_forward_static fails in its device
    look-up (before any launch: the pointers are never dereferenced) and
    cloth_last_cuda_error reports the cudaError_t.  Run in a child process
    with CUDA_VISIBLE_DEVICES empty, so it behaves the same on a GPU machine."""
    import subprocess
    import sys
    code = (
        "import ctypes, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_2403_12820_gb300 import _lib\n"
        "lib = _lib.load(build_if_needed=False)\n"
        "p = ctypes.c_void_p\n"
        "rc = lib.net_forward_static(p(256), p(512), p(768), 1, 4, 4, p(0))\n"
        "print(rc, lib.cloth_last_cuda_error())\n"
    )
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    rc, err = (int(t) for t in out.stdout.split())
    assert rc == -3 and err != 0, (rc, err)
