"""Independent Philox4x32-10: Triton's own implementation, run by its CPU interpreter.

Used only by the oracle's Philox pin (run as a subprocess so that the
interpreter flag is set before Triton is imported).  Usage:
    python philox_triton_ref.py counters.npy keys.npy out.npy
counters uint32[n,4], keys uint32[n,2] -> out uint32[n,4].
"""
import os
import sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np
import torch
import triton
import triton.language as tl

@triton.jit
def _k(c_ptr, k_ptr, o_ptr, n, BLOCK: tl.constexpr):
    i = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    msk = i < n
    c0 = tl.load(c_ptr + 4 * i + 0, mask=msk).to(tl.uint32)
    c1 = tl.load(c_ptr + 4 * i + 1, mask=msk).to(tl.uint32)
    c2 = tl.load(c_ptr + 4 * i + 2, mask=msk).to(tl.uint32)
    c3 = tl.load(c_ptr + 4 * i + 3, mask=msk).to(tl.uint32)
    k0 = tl.load(k_ptr + 2 * i + 0, mask=msk).to(tl.uint32)
    k1 = tl.load(k_ptr + 2 * i + 1, mask=msk).to(tl.uint32)
    o0, o1, o2, o3 = tl.philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(o_ptr + 4 * i + 0, o0.to(tl.int64), mask=msk)
    tl.store(o_ptr + 4 * i + 1, o1.to(tl.int64), mask=msk)
    tl.store(o_ptr + 4 * i + 2, o2.to(tl.int64), mask=msk)
    tl.store(o_ptr + 4 * i + 3, o3.to(tl.int64), mask=msk)

c = np.load(sys.argv[1]); k = np.load(sys.argv[2])
n = c.shape[0]
ct = torch.from_numpy(c.astype(np.int64)); kt = torch.from_numpy(k.astype(np.int64))
o = torch.zeros((n, 4), dtype=torch.int64)
_k[(triton.cdiv(n, 64),)](ct, kt, o, n, BLOCK=64)
np.save(sys.argv[3], o.numpy().astype(np.uint32))
