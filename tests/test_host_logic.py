"""Host-side logic of the CUDA library that needs no GPU, compiled by nvcc as
host code: the dependency sets of the persistent multi-pass kernels
(tile_span in common.cuh) against brute force, and the tile geometry of the
fused kernels (f2_tiling, f3_lz, f3_axis with the TMA path's x halo f3_hx)
against its covering, halo, minimum-length and 16-byte alignment rules."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_08825_gb300", "csrc")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not available")


def test_tile_span_matches_brute_force(tmp_path):
    exe = tmp_path / "tile_span_check"
    src = os.path.join(ROOT, "tests", "host", "tile_span_check.cu")
    subprocess.run([_nvcc(), "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), src, "-o",
                    str(exe)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")


def test_tile_geometry_covers_each_axis(tmp_path):
    exe = tmp_path / "tiling_check"
    src = os.path.join(ROOT, "tests", "host", "tiling_check.cu")
    subprocess.run([_nvcc(), "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include"), src, "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")
