"""A second independent pin of the oracle's Philox4x32-10: cuRAND's device
implementation.  curand_init(seed, subsequence, 0) followed by curand4()
calls yields the blocks of counter (i, 0, subsequence lo, subsequence hi)
under key (seed lo, seed hi), i = 0, 1, ..."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import chain

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_philox_matches_curand(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "curand_philox")
    subprocess.run([nvcc, "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "gpu_ref", "curand_philox.cu"), "-o", exe], check=True)
    for seed, sub in ((0, 0), (12345, 7), (2**40 + 17, 2**33 + 5)):
        n = 64
        out = subprocess.run([exe, str(seed), str(sub), str(n)], check=True, capture_output=True,
                             text=True).stdout
        ref = np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()],
                       dtype=np.uint64).astype(np.uint32)
        ctr = np.zeros((n, 4), dtype=np.uint32)
        ctr[:, 0] = np.arange(n, dtype=np.uint32)
        ctr[:, 2] = sub & 0xFFFFFFFF
        ctr[:, 3] = sub >> 32
        key = np.tile(np.array([[seed & 0xFFFFFFFF, seed >> 32]], dtype=np.uint64), (n, 1))
        np.testing.assert_array_equal(chain.philox(ctr, key.astype(np.uint32)), ref)
