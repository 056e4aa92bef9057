"""CPU-side checks of the C ABI: the library builds, loads, exports every entry
point include/cosenu.h declares, and rejects bad arguments before any device
work.  No compute calls are made here (there may be no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2203_12866_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cosenu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cosenu_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == names


def test_workspace_bytes(lib):
    nz, nv = 1000, 32
    n = 8 * nz * nv
    fp64 = binding.cosenu_workspace_bytes(nz, nv, binding.COSENU_FDKO, binding.COSENU_FP64)
    mixed = binding.cosenu_workspace_bytes(nz, nv, binding.COSENU_FDKO, binding.COSENU_MIXED)
    # fp64: two state buffers + three increments; mixed: state, its float copy, three increments
    assert fp64 >= 5 * n * 8 and mixed >= n * 8 + n * 4 + 3 * n * 4
    assert mixed < fp64
    for bad in [(0, 32), (16, 6), (16, 0), (16, 512), (-1, 32)]:
        assert binding.cosenu_workspace_bytes(*bad, 0, 0) == 0


@pytest.mark.parametrize("args", [(0, 32, 1.0, 0, 0), (16, 30, 1.0, 0, 0), (16, 32, -1.0, 0, 0),
                                  (16, 32, 1.0, 3, 0), (16, 32, 1.0, 0, 7), (16, 512, 1.0, 0, 0)])
def test_create_rejects_bad_sizes_without_device_work(lib, args):
    with pytest.raises(binding.CosenuError) as e:
        binding.cosenu_create(*args)
    assert e.value.code == binding.COSENU_EINVAL
    assert "invalid grid" in binding.cosenu_last_error(None)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.cosenu_step(None, 1) == binding.COSENU_EINVAL
    assert lib.cosenu_sync(None) == binding.COSENU_EINVAL
    assert lib.cosenu_steps_taken(None) == -1
    lib.cosenu_destroy(None)
    assert lib.cosenu_create_external(16, 32, 1.0, 0, 0, None, 0) is None


def test_header_constants_match_binding():
    """Every COSENU_* enumerator of include/cosenu.h has the same value in the
    Python binding (the binding only marshals; a stale constant would pass a
    different scheme, precision or status across the ABI)."""
    import re
    text = open(os.path.join(ROOT, "include", "cosenu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    found = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"(COSENU_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            found[name] = int(val)
    assert len(found) >= 16, found  # schemes, precisions, status codes, quadratures
    for name, val in found.items():
        assert getattr(binding, name) == val, name
