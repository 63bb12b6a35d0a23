"""The C ABI used from plain C (no Python binding, no PyTorch): the example
program is compiled against include/morph.h and the built library, run on an
image and SE written here, and its dilation / erosion (values and counts) are
compared with the oracle."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import morph as M
from paper_2305_03018_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_matches_oracle(tmp_path):
    lib = M.load_library()._name
    exe = tmp_path / "c_api_example"
    src = os.path.join(ROOT, "paper_2305_03018_gb300", "examples", "c_api_example.c")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    subprocess.run(["gcc", "-O2", "-std=c99", src, "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), "-o", str(exe), lib,
                    "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{os.path.dirname(lib)}",
                    f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"], check=True)
    g = wl.rng(70)
    n, h, w, L = 2, 45, 77, 64
    f = g.integers(0, L, size=(n, h, w)).astype(np.uint8)
    se = wl.se_random(g, 7, 5, 0.6, 5, origin=(2, 3))
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as fh:
        fh.write(np.array([n, h, w, L, 7, 5, 2, 3], np.int32).tobytes())
        fh.write(f.tobytes())
        fh.write(se.mask.astype(np.uint8).tobytes())
        fh.write(se.offset.astype(np.int32).tobytes())
    out = tmp_path / "out.bin"
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    res = np.fromfile(out, dtype=np.int32).reshape(4, n, h, w)
    D, cD = oracle.dilate(f, L, se.mask, se.offset, se.origin)
    E, cE = oracle.erode(f, L, se.mask, se.offset, se.origin)
    assert np.array_equal(res[0], D) and np.array_equal(res[1], cD)
    assert np.array_equal(res[2], E) and np.array_equal(res[3], cE)
