"""The device-resident driver's one-game kernels (one terminal per product item, and items
merged per opponent column) fit their 512-thread CTA without register spills (a spill on this path has cost several percent of the iteration rate every time it
appeared): compile engine.cu for sm_103a with ptxas statistics and read them."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_one_game_engine_kernel_has_no_spills(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    csrc = os.path.join(ROOT, "paper_1810_03063_b300", "csrc")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c",
                        os.path.join(csrc, "engine.cu"), "-o", str(tmp_path / "engine.o")],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stderr.splitlines()
    idx = [i for i, l in enumerate(lines) if "Compiling entry function" in l and "engine_kernel_one" in l]
    assert len(idx) == 2, "engine_kernel_one / engine_kernel_one_merged not found in the ptxas output"
    for i in idx:
        block = " ".join(lines[i:i + 4])
        spills = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", block)
        regs = re.search(r"Used (\d+) registers", block)
        assert spills and regs, block
        assert int(spills.group(1)) == 0 and int(spills.group(2)) == 0, block
        assert int(regs.group(1)) <= 128, block
