"""Pins for the oracle's Philox4x32-10 (Salmon et al., SC'11).

The oracle's generator is checked against an independent implementation:
Triton's ``tl.philox`` (open Python source, run on the CPU through Triton's
interpreter), which takes 32-bit counters (c0..c3) and the key
(seed lo, seed hi).  A statistical check guards the output distribution.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _k(c_ptr, seed_lo_ptr, seed_hi_ptr, out_ptr, n, BLOCK: tl.constexpr):
    off = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    msk = off < n
    c0 = tl.load(c_ptr + off * 4 + 0, mask=msk).to(tl.uint32, bitcast=True)
    c1 = tl.load(c_ptr + off * 4 + 1, mask=msk).to(tl.uint32, bitcast=True)
    c2 = tl.load(c_ptr + off * 4 + 2, mask=msk).to(tl.uint32, bitcast=True)
    c3 = tl.load(c_ptr + off * 4 + 3, mask=msk).to(tl.uint32, bitcast=True)
    lo = tl.load(seed_lo_ptr + off, mask=msk).to(tl.uint32, bitcast=True).to(tl.uint64)
    hi = tl.load(seed_hi_ptr + off, mask=msk).to(tl.uint32, bitcast=True).to(tl.uint64)
    seed = (hi << 32) | lo
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + off * 4 + 0, r0.to(tl.int32, bitcast=True), mask=msk)
    tl.store(out_ptr + off * 4 + 1, r1.to(tl.int32, bitcast=True), mask=msk)
    tl.store(out_ptr + off * 4 + 2, r2.to(tl.int32, bitcast=True), mask=msk)
    tl.store(out_ptr + off * 4 + 3, r3.to(tl.int32, bitcast=True), mask=msk)

d = np.load(sys.argv[1])
ctr = torch.from_numpy(d["ctr"].view(np.int32).copy())
key = d["key"].view(np.int32)
lo = torch.from_numpy(key[:, 0].copy()); hi = torch.from_numpy(key[:, 1].copy())
n = ctr.shape[0]
out = torch.zeros((n, 4), dtype=torch.int32)
_k[(triton.cdiv(n, 256),)](ctr, lo, hi, out, n, BLOCK=256)
np.save(sys.argv[2], out.numpy().view(np.uint32))
"""


def _cases(n, rng):
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # edge counters and keys: zeros, all-ones, the layouts the annealer uses
    ctr[0] = 0; key[0] = 0
    ctr[1] = 0xFFFFFFFF; key[1] = 0xFFFFFFFF
    ctr[2] = [5, 7, 3, (0 << 24) | 1]; key[2] = [42, 0]
    ctr[3] = [11, 0, 9, (1 << 24) | 0]; key[3] = [1, 0]
    ctr[4] = [2, 1, 0, (2 << 24)]; key[4] = [7, 0]
    return ctr, key


def test_philox_matches_triton(orc, tmp_path):
    pytest.importorskip("triton")
    rng = np.random.default_rng(2510)
    ctr, key = _cases(4096, rng)
    inp = tmp_path / "in.npz"
    out = tmp_path / "out.npy"
    np.savez(inp, ctr=ctr, key=key)
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, str(script), str(inp), str(out)], env=env,
                         capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
    ref = np.load(out)
    got = orc.philox(ctr, key)
    assert ref.shape == got.shape
    mism = np.nonzero((ref != got).any(axis=1))[0]
    assert mism.size == 0, f"{mism.size} mismatches, first at {mism[:5]}"


def test_philox_word_indexing(orc):
    # rand_word(seed, ctr, idx) is word idx of Philox(ctr, key=(seed lo, seed hi))
    seed = (123 << 32) | 456
    full = orc.philox(np.array([[9, 8, 7, 6]], np.uint32), np.array([[456, 123]], np.uint32))[0]
    for idx in range(4):
        assert orc.rand_word(seed, 9, 8, 7, 6, idx) == int(full[idx])


def test_philox_uniform_bits(orc):
    # 2^16 counters x 4 words: top byte uniform (chi-square), every bit balanced
    n = 1 << 16
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    key = np.tile(np.array([[2025, 0]], np.uint32), (n, 1))
    w = orc.philox(ctr, key).reshape(-1)
    counts = np.bincount(w >> 24, minlength=256)
    _, p = stats.chisquare(counts)
    assert p > 1e-4
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    sigma = 0.5 / np.sqrt(w.size)
    assert np.all(np.abs(bits - 0.5) < 5 * sigma)
