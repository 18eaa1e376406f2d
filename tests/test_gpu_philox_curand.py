"""Pin of the oracle's Philox4x32-10 against an implementation it shares
nothing with: cuRAND's Philox4_32_10 device generator, run as a black box
(tests/curand_philox_probe.cu).  cuRAND's documented use of its arguments --
the seed as the two key words, the subsequence as the high half of the
128-bit counter and the offset (in 32-bit outputs, four per block) as the
low half -- is the mapping tested; every sample must give the same four
words as the oracle's Philox at that counter and key."""

import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _probe():
    src = os.path.join(HERE, "curand_philox_probe.cu")
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libcurand_philox_probe.so")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                        "-Xcompiler", "-fPIC", src, "-o", lib], check=True)
    return ctypes.CDLL(lib)


def test_oracle_philox_equals_curand_philox(cuda):
    torch = cuda
    fn = _probe().curand_philox_raw
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int]
    rng = np.random.default_rng(42)
    n = 256
    seeds = rng.integers(0, 2**63, size=n, dtype=np.uint64) * 2 + rng.integers(0, 2, size=n, dtype=np.uint64)
    subseq = rng.integers(0, 2**63, size=n, dtype=np.uint64)
    blocks = rng.integers(0, 2**40, size=n, dtype=np.uint64)
    blocks[:8] = 0
    offsets = blocks * np.uint64(4)
    dev = [torch.from_numpy(a.view(np.int64).copy()).cuda() for a in (seeds, subseq, offsets)]
    out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    assert fn(*(t.data_ptr() for t in dev), out.data_ptr(), n) == 0
    got = out.cpu().numpy().view(np.uint32)
    M = 0xFFFFFFFF
    for i in range(n):
        s, q, b = int(seeds[i]), int(subseq[i]), int(blocks[i])
        ctr = [b & M, b >> 32, q & M, q >> 32]
        ref = oracle.philox(ctr, [s & M, s >> 32])
        assert [int(v) for v in got[i]] == [int(v) for v in ref], (i, s, q, b)
