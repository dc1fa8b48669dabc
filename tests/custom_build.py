"""Builds tests/custom_walks.cu (walk types written against
include/trw_custom.cuh) into a shared library linked with libtrw.so."""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = os.path.join(ROOT, "paper_2107_11983_gb300")


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(out_dir: str, link: bool = True) -> str:
    """Compile (and, with link, link against libtrw.so) into out_dir; returns the path."""
    src = os.path.join(HERE, "custom_walks.cu")
    out = os.path.join(out_dir, "libcustom_walks.so" if link else "custom_walks.o")
    cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), src, "-o", out]
    if link:
        cmd[1:1] = ["-shared"]
        cmd += ["-L", PKG, "-ltrw", "-Xlinker", "-rpath=" + PKG]
    else:
        cmd[1:1] = ["-c"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed:\n{r.stdout}\n{r.stderr}")
    return out
