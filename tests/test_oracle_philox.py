"""Pins for the oracle's Philox4x32-10 (Salmon et al., SC'11) and its uniform mapping.

The pin is an independent implementation: cuRAND's host generator for PHILOX4_32_10,
called as a black box through its public C API.  With the default ordering it emits, for
block j of four words, Philox(counter = (j // 65536, 0, j % 65536, 0), key = (seed_lo,
seed_hi)); a generator offset of 4 * 65536 * (x + 2^32 y) words starts it at counter
(x, y, 0, 0).  Matching it over more than one 65536-block wrap and at large offsets pins the
round function, the key schedule, the key words and counter words 0, 1 and 2.  Counter word 3
is the draw's tag, always 0 in this method.  The device implementation is compared with the
oracle bit for bit on the GPU (tests/test_gpu_parity.py, the sampler cases).
"""
import ctypes
import os

import numpy as np
import pytest

CURAND = "/usr/local/cuda/lib64/libcurand.so"
PHILOX4_32_10 = 161          # curandRngType_t value for CURAND_RNG_PSEUDO_PHILOX4_32_10
ORDERING_DEFAULT = 101


def _curand_host_words(seed: int, nwords: int, offset: int = 0) -> np.ndarray:
    if not os.path.exists(CURAND):
        pytest.skip("libcurand not present")
    lib = ctypes.CDLL(CURAND)
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOrdering(gen, ORDERING_DEFAULT) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(nwords, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(nwords)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(oracle_mod, seed):
    blocks = 65536 * 2 + 4096
    ref = _curand_host_words(seed, 4 * blocks)
    j = np.arange(blocks, dtype=np.int64)
    ctr = np.zeros((blocks, 4), np.uint32)
    ctr[:, 0] = (j // 65536).astype(np.uint32)
    ctr[:, 2] = (j % 65536).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    got = oracle_mod.philox(ctr, key)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("x,y", [(0, 1), (7, 3), (123, 4095), (2**32 - 2, 8191)])  # offset < 2^64
def test_philox_counter_words_0_and_1_via_offset(oracle_mod, x, y):
    seed = 0x243F6A8885A308D3
    blocks = 4096
    ref = _curand_host_words(seed, 4 * blocks, offset=4 * 65536 * (x + (y << 32)))
    ctr = np.zeros((blocks, 4), np.uint32)
    ctr[:, 0] = x
    ctr[:, 1] = y
    ctr[:, 2] = np.arange(blocks, dtype=np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    assert np.array_equal(oracle_mod.philox(ctr, key), ref)


def test_uniform_mapping_is_exact_and_open(oracle_mod):
    # u = ((w >> 9) + 0.5) * 2^-23 lies strictly inside (0, 1) and is exact in FP32 and FP64.
    w = np.concatenate([np.array([0, 511, 512, 0xFFFFFFFF, 0x80000000, 0xFFFFFE00], np.uint32),
                        np.random.default_rng(0).integers(0, 2 ** 32, 100000, dtype=np.uint64).astype(np.uint32)])
    u64 = ((w >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
    u32 = ((w >> 9).astype(np.float32) + np.float32(0.5)) * np.float32(2.0 ** -23)
    assert np.all(u64 > 0) and np.all(u64 < 1)
    assert np.array_equal(u32.astype(np.float64), u64)
    # The sampler's directions use these values: theta = 2 pi u1 covers [0, 2 pi).
    assert u64.min() == 2.0 ** -24 and u64.max() == 1.0 - 2.0 ** -24


def test_sampler_words_follow_the_counter_layout(oracle_mod):
    from paper_2304_08052_gb300 import scenes
    sc = scenes.tiny(seed=3, B=3, S=2, M=2, images=17)
    p = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    seed = 0xDEADBEEF12345678
    out = oracle_mod.sample(sc, p, seed)
    ctr = []
    for b in range(sc.B):
        for s in range(sc.S):
            for i in range(int(sc.n_vs[b])):
                ctr.append((i, s, b, 0))
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    assert np.array_equal(out.words, oracle_mod.philox(np.array(ctr, np.uint32), key))
