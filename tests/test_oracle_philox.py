"""Pins the oracle's Philox4x32-10 against an implementation it shares nothing with:
Triton's ``tl.philox`` run by Triton's CPU interpreter (third-party source, written from the
same published definition, Salmon et al. SC'11)."""
import os

import numpy as np
import pytest


def _triton_philox(ctrs: np.ndarray, seed: int) -> np.ndarray:
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    import torch
    import triton.language as tl

    @triton.jit
    def kern(out_ptr, c_ptr, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(c_ptr + 4 * i + 0)
        c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2)
        c3 = tl.load(c_ptr + 4 * i + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a)
        tl.store(out_ptr + 4 * i + 1, b)
        tl.store(out_ptr + 4 * i + 2, c)
        tl.store(out_ptr + 4 * i + 3, d)

    n = ctrs.shape[0]
    c = torch.from_numpy(ctrs.astype(np.uint32).view(np.int32).reshape(-1).copy())
    out = torch.zeros(4 * n, dtype=torch.int32)
    kern[(1,)](out, c, seed, N=n)
    return out.numpy().view(np.uint32).reshape(n, 4)


def test_philox_matches_triton_interpreter(oracle_mod):
    rng = np.random.default_rng(12345)
    n = 256
    ctrs = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    # include structured counters of the kind the method uses
    ctrs[:8] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
                [0xFFFFFFFF] * 4, [341, 6005, 1, 8], [0, 3, 0, 1 << 28]]
    for seed in (0, 1, 0x0123456789ABCDEF, 2**64 - 1):
        ref = _triton_philox(ctrs, seed)
        got = oracle_mod.philox(ctrs, seed)
        np.testing.assert_array_equal(got, ref)


def test_philox_key_and_counter_sensitivity(oracle_mod):
    base = np.array([[5, 6, 7, 8]], dtype=np.uint32)
    a = oracle_mod.philox(base, 1)
    for i in range(4):
        c = base.copy()
        c[0, i] ^= 1
        assert not np.array_equal(oracle_mod.philox(c, 1), a)
    assert not np.array_equal(oracle_mod.philox(base, 1 + (1 << 32)), a)  # high key word used


def test_philox_bit_balance(oracle_mod):
    # 2^16 blocks: every output bit is set with frequency 1/2 within 5 sigma
    n = 1 << 16
    ctrs = np.zeros((n, 4), dtype=np.uint32)
    ctrs[:, 0] = np.arange(n)
    ctrs[:, 1] = 77
    out = oracle_mod.philox(ctrs, 1)
    bits = np.unpackbits(out.view(np.uint8), bitorder="little").reshape(n, 128)
    freq = bits.mean(0)
    assert np.all(np.abs(freq - 0.5) < 5 * 0.5 / np.sqrt(n))
