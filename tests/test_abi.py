"""The C-ABI library builds, loads and exports every function include/trw.h
declares, and a plain C99 program compiles and links against it (CPU only: no
compute calls)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2107_11983_gb300 as trw
from paper_2107_11983_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "trw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(trw_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_functions():
    assert sorted(trw._SIGS) == declared_functions()


def test_binding_loads_without_gpu():
    lib = trw.load_library()
    assert lib.trw_last_error() is not None


def test_plain_c_consumer(tmp_path):
    """tests/abi_consumer.c: strict C99 against trw.h, linked with libtrw.so;
    argument errors, NULL handles and per-thread error messages need no GPU."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = _build.build()
    src = os.path.join(ROOT, "tests", "abi_consumer.c")
    inc = os.path.join(ROOT, "include")
    exe = str(tmp_path / "abi_consumer")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-pthread", "-I", inc, src, lib,
           "-Wl,-rpath," + os.path.dirname(lib), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    gxx = shutil.which("g++")
    if gxx is not None:  # the same program is valid C++ (the header's extern "C" guard)
        r = subprocess.run([gxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-x", "c++", "-fsyntax-only",
                            "-I", inc, src], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    load = int(re.search(r"load=(-?\d+)", r.stdout).group(1))
    import torch
    assert load == (0 if torch.cuda.is_available() else -4), r.stdout  # TRW_OK, or TRW_ERR_CUDA without a GPU


def test_no_fallback_without_gpu():
    """The product path has no CPU fallback: without a GPU, loading a graph
    fails with TRW_ERR_CUDA, importing the package pulls in nothing from
    oracle/, and no package source imports or includes it."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    import numpy as np
    rp = np.array([0, 2, 4, 6], np.int64)
    col = np.array([1, 2, 0, 2, 0, 1], np.int32)
    with pytest.raises(trw.TRWError) as e:
        trw.Graph(rp, col)
    assert e.value.status == -4
    code = ("import sys, paper_2107_11983_gb300, paper_2107_11983_gb300.shard; "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "assert not bad, bad")
    r = subprocess.run([os.sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    pkg = os.path.join(ROOT, "paper_2107_11983_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|#include\s+\"oracle", text, re.M), f


def test_readme_c_example(tmp_path):
    """The README's C quick start compiles as strict C99, links against
    libtrw.so and runs: it walks on a GPU, and without one it reports the
    CUDA error through trw_last_error() and exits 1."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    text = open(os.path.join(ROOT, "README.md")).read()
    m = re.search(r"## Quick start \(C\)\s*```c\n(.*?)```", text, re.S)
    assert m, "README has no C quick start"
    src = tmp_path / "example.c"
    src.write_text(m.group(1))
    lib = _build.build()
    exe = str(tmp_path / "example")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                        os.path.join(ROOT, "include"), str(src), lib, "-Wl,-rpath," + os.path.dirname(lib), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    import torch
    if torch.cuda.is_available():
        assert r.returncode == 0 and r.stdout.startswith("walk 0: "), r.stdout + r.stderr
    else:
        assert r.returncode == 1 and r.stderr.startswith("trw: ") and "cudaGetDevice" in r.stderr, r.stderr


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the size, field offsets and field
    sizes of their C counterparts in trw.h (compiled and measured by gcc)."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"trw_params": trw._Params, "trw_tuning": trw.Tuning, "trw_stats": trw.Stats,
               "trw_serve_config": trw.ServeConfig}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "trw.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu %zu\\n", offsetof({cname}, {f}), sizeof((({cname}*)0)->{f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for ln in out:
        parts = ln.split()
        if not parts:
            continue
        py = structs[parts[0]]
        if parts[1] == "sizeof":
            assert ctypes.sizeof(py) == int(parts[2]), ln
        else:
            fd = getattr(py, parts[1])
            assert (fd.offset, fd.size) == (int(parts[2]), int(parts[3])), ln
        seen += 1
    assert seen == sum(len(py._fields_) + 1 for py in structs.values())


def _c_kind(t: str) -> str:
    t = " ".join(t.split())
    if "*" in t or t.startswith("trw_stream_fn"):
        return "ptr"
    base = t.replace("const ", "").split()[0]
    return {"int64_t": "i64", "int32_t": "i32", "int": "i32", "trw_algo": "i32", "trw_kernel": "i32",
            "trw_status": "i32", "uint32_t": "u32", "uint64_t": "u64", "double": "f64", "void": "void"}[base]


def _ctypes_kind(c) -> str:
    if c is None:
        return "void"
    if c in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(c, (ctypes._Pointer, ctypes._CFuncPtr)):
        return "ptr"
    if c is ctypes.c_double:
        return "f64"
    return ("i" if c(-1).value < 0 else "u") + str(8 * ctypes.sizeof(c))


def test_binding_signatures_match_header():
    """Every ctypes signature has the header prototype's return kind and the
    same number, order, width and signedness of arguments (a mismatch would
    pass garbage through the ABI without any error)."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "trw.h")).read(), flags=re.S)
    protos = re.findall(r"([A-Za-z_][A-Za-z_0-9 \*]*?)\b(trw_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text, re.S)
    assert sorted(name for _, name, _ in protos) == declared_functions()
    for ret, name, args in protos:
        args = " ".join(args.split())
        want_args = [] if args in ("void", "") else [
            _c_kind(re.sub(r"\b[A-Za-z_0-9]+$", "", a.strip())) for a in args.split(",")]
        pr, pa = trw._SIGS[name]
        assert _ctypes_kind(pr) == _c_kind(ret), name
        assert [_ctypes_kind(a) for a in pa] == want_args, name
