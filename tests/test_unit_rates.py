"""Measured throughput of the arithmetic units an FP64 panel update could use
(SIMT FP64, the FP64 tensor-core instruction, the INT8 tensor-core
instruction that integer-slice emulation of FP64 products is built from),
beside SIMT FP32 and BF16 tensor-core yardsticks, from tests/rates_probe.cu
timed with CUDA events.  The numbers decide whether FP64 panels should move
to tensor cores by Ozaki-style integer slicing: the test asserts only that
every unit runs and that the yardsticks come out in a plausible order."""
import ctypes
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
KINDS = {"dfma_fp64": 0, "ffma_fp32": 1, "dmma_fp64": 2, "imma_int8": 3, "hmma_bf16": 4}


def measured_rates(tmpdir):
    lib = os.path.join(str(tmpdir), "rates_probe.so")
    subprocess.run(["nvcc", "-shared", "-Xcompiler", "-fPIC", "-O3", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-o", lib, os.path.join(HERE, "rates_probe.cu")], check=True)
    L = ctypes.CDLL(lib)
    L.rates_probe.restype = ctypes.c_double
    L.rates_probe.argtypes = [ctypes.c_int, ctypes.c_int]
    return {k: L.rates_probe(v, 5) for k, v in KINDS.items()}


def test_arithmetic_unit_rates(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = measured_rates(tmp_path)
    print({k: round(v, 2) for k, v in r.items()}, "T(FL)OP/s")
    assert all(v > 0 for v in r.values()), r
    assert r["hmma_bf16"] > r["ffma_fp32"] > r["dfma_fp64"], r
