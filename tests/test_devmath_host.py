"""The FP64 sincos of the CUDA path keeps only its two final sums in FP64; the
reduction, the corrections and the join back to FP64 run in integer and FP32
arithmetic (csrc/devmath.cuh).  Those building blocks are host-compilable, so
this CPU test builds them with nvcc for the host and checks them against exact
references and long-double libm: the join is exact for normalised pairs, the
split loses < 2^-46 relative, the integer reduction equals the FP64 one, and
sin/cos stay within 1.5e-16 absolute (the device test holds the GPU build to
5e-16), with sin x relatively accurate near 0 (elsewhere the bound is
absolute: ~1e-17 from the double-float corrections plus the final FP64
rounding)."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_devmath_building_blocks_on_host(tmp_path):
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    if not (os.path.exists(nvcc) or shutil.which(nvcc)):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "devmath_host_check")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                           "-Xcompiler", "-ffp-contract=off", "-o", exe, os.path.join(HERE, "devmath_host_check.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, check=True, timeout=300).stdout
    r = json.loads(out.strip().splitlines()[-1])
    assert r["pair_to_f64_rel"] == 0.0, r
    assert r["split_f64_rel"] <= 2.0 ** -46, r
    assert r["reduce_pair_mismatch"] == 0, r
    assert r["sin_abs"] < 1.5e-16 and r["cos_abs"] < 1.5e-16, r
    # table index 0 (x < D/2): sin x = x + (sin x - x) keeps ~1 ulp relative accuracy
    assert r["tiny_sin_rel"] < 5e-16, r
