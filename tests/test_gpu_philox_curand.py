"""Philox-4x32-10 against cuRAND's device generator, all four counter words.

cuRAND's host generator only reaches counter words 0-2 (the CPU pins in
test_oracle_rng_exp.py).  Its device API reaches word 3 as well: a Philox
state initialised with curand_init(seed, subsequence, offset) produces, as its
first curand4(), the block of counter (offset/4 lo, offset/4 hi,
subsequence lo, subsequence hi) under key (seed lo, seed hi).  The probe
tests/curand_philox_probe.cu calls exactly that for a list of counters and
keys; its blocks must equal the oracle's (the counter word 3 that carries the
replica index in every draw of the chain) and the library's device Philox.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("curand_probe") / "libprobe.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "curand_philox_probe.cu")], check=True)
    lib = ctypes.CDLL(out)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib.probe_philox.argtypes = [p, p, p, ctypes.c_int]
    lib.probe_philox.restype = ctypes.c_int

    def run(ctr, key):
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
        key = np.ascontiguousarray(key, dtype=np.uint32)
        res = np.zeros_like(ctr)
        rc = lib.probe_philox(ctr.ctypes.data_as(p), key.ctypes.data_as(p),
                              res.ctypes.data_as(p), len(ctr))
        assert rc == 0, rc
        return res
    return run


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] &= (1 << 30) - 1          # the probe's offset must fit in 64 bits
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # the counters the chain draws: label k of round r of replica c
    # (k, r lo, r hi, c), the disorder domains (s, 1 or 2, 0xFFFFFFFF, c) and
    # the random-site positions (s, 3, 0xFFFFFFFF, c)
    special = np.array([[0, 0, 0, 1], [5, 7, 0, 303], [4095, 123456, 0, 0xFFFFFFFF],
                        [17, 1, 0xFFFFFFFF, 12], [9, 2, 0xFFFFFFFF, 65535],
                        [3, 3, 0xFFFFFFFF, 0x80000000], [1, 0, 0xFFFFFFFE, 7]],
                       dtype=np.uint32)
    ctr[:len(special)] = special
    return ctr, key


def test_oracle_philox_equals_curand_device_on_all_counter_words(probe):
    ctr, key = _cases(512, 11)
    ref = probe(ctr, key)
    for t in range(len(ctr)):
        np.testing.assert_array_equal(oracle.philox(ctr[t], key[t]), ref[t], err_msg=str(t))


def test_library_philox_equals_curand_device(probe):
    from paper_1407_5026_gb300 import build, binding
    build.build()
    binding.load()
    ctr, key = _cases(4096, 12)
    np.testing.assert_array_equal(binding.cg_debug_philox(ctr, key), probe(ctr, key))
