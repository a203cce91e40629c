"""Builds the CUDA library libstencil_gb300.so in-tree for sm_103a.

Every ``csrc/*.cu`` file is compiled by nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a``) and linked into
``paper_2103_08825_gb300/_build/libstencil_gb300.so``.  ptxas register and
shared-memory reports go to ``_build/ptxas.log``.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libstencil_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the GB300 stencil library needs the CUDA toolkit to build")


_INCLUDE_RE = None


def _local_deps(path: str, seen=None) -> set:
    """The quoted #include files a source pulls in, transitively (the headers
    of csrc/ and include/ it depends on)."""
    global _INCLUDE_RE
    import re
    if _INCLUDE_RE is None:
        _INCLUDE_RE = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)
    seen = set() if seen is None else seen
    with open(path) as f:
        text = f.read()
    for name in _INCLUDE_RE.findall(text):
        dep = os.path.normpath(os.path.join(os.path.dirname(path), name))
        if os.path.exists(dep) and dep not in seen:
            seen.add(dep)
            _local_deps(dep, seen)
    return seen


def _stale(obj: str, src: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src, *deps])


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                    "-I", INCLUDE, "--expt-relaxed-constexpr"]

    def one(src):
        obj = os.path.join(OUT, "obj", os.path.basename(src)[:-3] + ".o")
        if not force and not _stale(obj, src, _local_deps(src)):
            return obj, ""
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc, *flags, "-c", src, "-o", tmp]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{p.stderr[-6000:]}")
        os.replace(tmp, obj)
        return obj, p.stderr

    # compile the longest translation units first (they set the build's length)
    srcs.sort(key=lambda f: -os.path.getsize(f) - sum(os.path.getsize(d) for d in _local_deps(f)))
    n = jobs or max(1, min(len(srcs), os.cpu_count() or 4))
    logs = []
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        objs = []
        for obj, log in ex.map(one, srcs):
            objs.append(obj)
            if log:
                logs.append(f"== {os.path.basename(obj)}\n{log}")
    if logs:
        with open(os.path.join(OUT, "ptxas.log"), "w") as f:
            f.write("\n".join(logs))
    need_link = force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs)
    if need_link:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed:\n{p.stderr[-4000:]}")
        os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
