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


def _ctype_of(decl):
    """ctypes class expected for one C parameter or return declaration of the header."""
    import ctypes
    d = " ".join(decl.replace("const ", "").split())
    if "*" in d or d.split()[0] in ("cosenu_t", "cosenu_batch_t", "cosenu_server_t"):
        return "pointer"
    base = d.split()[0]
    return {"int64_t": ctypes.c_int64, "int32_t": ctypes.c_int32, "int": ctypes.c_int,
            "size_t": ctypes.c_size_t, "double": ctypes.c_double, "uint64_t": ctypes.c_uint64,
            "void": None}[base]


def test_header_prototypes_match_binding(lib):
    """Each function of include/cosenu.h is bound with the header's parameter count
    and the same integer widths, floating types and pointer positions."""
    import ctypes
    text = open(os.path.join(ROOT, "include", "cosenu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = re.findall(r"([A-Za-z_][A-Za-z0-9_ \*]*?)\b(cosenu_\w+)\s*\(([^;{]*?)\)\s*;", text)
    assert len(protos) >= 50
    for ret, name, params in protos:
        f = getattr(lib, name)
        params = " ".join(params.split())
        args = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        assert len(f.argtypes) == len(args), name
        for want, got in zip([_ctype_of(a) for a in args], f.argtypes):
            if want == "pointer":
                assert got is ctypes.c_void_p or got is ctypes.c_char_p or \
                    issubclass(got, ctypes._Pointer), (name, got)
            else:
                assert got is want, (name, want, got)
        want_ret = _ctype_of(ret.strip())
        if want_ret == "pointer":
            assert f.restype in (ctypes.c_void_p, ctypes.c_char_p), name
        else:
            assert f.restype is want_ret, (name, want_ret, f.restype)


def test_struct_layouts_match_binding(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's size and
    field offsets (compiled with gcc against include/cosenu.h)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {
        "cosenu_params": ["mu", "omega", "theta", ("lambda", "lambda_"), "ko_eps", "weno_eps", "dt"],
        "cosenu_conserved_t": ["tr_nu", "tr_nubar", "M", "M_vac", "dP_max", "dP_mean", "step"],
        "cosenu_batch_class": ["scheme", "precision", "nv", "members", "rows", "rows_per_slot",
                               "ring", "grid", "smem", "occupancy", "concurrent", "kernel_ms"],
        "cosenu_request": ["nz", "nv", "L", "scheme", "precision", "params", "nsteps", "state",
                           "alpha", "sigma_nu", "sigma_nubar", "eps0", "seed", "out_state"],
        "cosenu_result": ["status", "steps", "conserved", "t_submit", "t_admit", "t_done"],
        "cosenu_server_stats": ["submitted", "admitted", "finished", "rounds", "steps", "queued",
                                "running", "bytes_in_use", "peak_bytes", "budget"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cosenu.h"', "int main(void) {"]
    for s, fields in structs.items():
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f in fields:
            c = f[0] if isinstance(f, tuple) else f
            lines.append(f'  printf("{s} {c} %zu\\n", offsetof({s}, {c}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if ln:
            s, k, v = ln.split()
            got[(s, k)] = int(v)
    for s, fields in structs.items():
        py = getattr(binding, s)
        assert ctypes.sizeof(py) == got[(s, "size")], s
        for f in fields:
            c, p = (f if isinstance(f, tuple) else (f, f))
            assert getattr(py, p).offset == got[(s, c)], (s, c)


@pytest.mark.parametrize("y,nz,nv,L,out", [(None, 16, 8, 1.0, 64), (64, 16, 8, 1.0, None),
                                           (64, 0, 8, 1.0, 64), (64, 16, 0, 1.0, 64),
                                           (64, 16, 8, 0.0, 64), (64, 16, 8, -2.0, 64)])
def test_conserved_noalloc_rejects_bad_arguments_without_device_work(lib, y, nz, nv, L, out):
    """The argument checks return before any CUDA call (the pointers are never
    dereferenced on this path, so placeholder addresses are safe)."""
    rc = lib.cosenu_conserved_noalloc(y, nz, nv, L, 0.0, out, None)
    assert rc == binding.COSENU_EINVAL
    assert "NULL pointer, nz < 1, nv < 1 or L <= 0" in binding.cosenu_last_error(None)


def test_conserved_noalloc_rejects_grids_beyond_its_static_scratch(lib):
    rc = lib.cosenu_conserved_noalloc(64, (1 << 28) // 256 + 1, 256, 1.0, 0.0, 64, None)
    assert rc == binding.COSENU_EINVAL
    assert "exceeds the static scratch limit" in binding.cosenu_last_error(None)
    assert "268435456" in binding.cosenu_last_error(None)
