"""Pins of the oracle's random-number contract.

Philox4x32-10 is pinned against cuRAND's host-side PHILOX4_32_10 generator (a library run on
the CPU; only its outputs are compared).  With the default ordering the generator's output at
offset o is word o%4 of Philox(counter = (pos_lo, pos_hi, subseq, 0), key = seed), where
block b = o/4 = pos * 2^16 + subseq; the offsets below walk counter words 0, 1 and 2 and both
key words.  Box-Muller is pinned by its distribution.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest
from scipy import stats

import oracle


def _curand():
    for name in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if name and os.path.exists(name) or (name and not name.startswith("/")):
            try:
                return ctypes.CDLL(name)
            except OSError:
                continue
    return None


def _curand_host_words(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = (ctypes.c_uint * n)()
        assert lib.curandGenerate(gen, out, ctypes.c_size_t(n)) == 0
        return list(out)
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 987654321987])
@pytest.mark.parametrize("block", [0, 1, 7, 65535, 65536, 3 * 65536 + 5, (1 << 48) + (9 << 16) + 2])
def test_philox_matches_curand_host_generator(seed, block):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    words = _curand_host_words(lib, seed, 4 * block, 4)
    pos, sub = block >> 16, block & 0xFFFF
    ctr = [pos & 0xFFFFFFFF, pos >> 32, sub, 0]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    assert oracle.philox4x32_10(ctr, key) == words
    assert oracle.philox4x32_10(ctr, key, precision="f32") == words


def test_box_muller_distribution():
    z = oracle.normals_bulk(seed=7, purpose=1, m=3, w1=11, step=2, d=8, count=200_000)
    flat = z.ravel()
    n = flat.size
    assert abs(flat.mean()) < 5.0 / np.sqrt(n)
    assert abs(flat.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert stats.kstest(flat, "norm").pvalue > 1e-4
    # the 8 normals of one counter are uncorrelated
    c = np.corrcoef(z.T)
    off = c[~np.eye(8, dtype=bool)]
    assert np.abs(off).max() < 5.0 / np.sqrt(z.shape[0])
    # truncation of the 23-bit uniforms: |z| <= sqrt(-2 ln 2^-23)
    assert np.abs(flat).max() <= np.sqrt(-2.0 * np.log(2.0 ** -23)) + 1e-12
    # the cos and sin members of a pair are independent: E[z0^2 z1^2] = 1
    assert abs(np.mean(z[:, 0] ** 2 * z[:, 1] ** 2) - 1.0) < 0.05


def test_streams_differ_by_purpose_date_item_step():
    base = oracle.normals(5, 1, 2, 0, 0, 3, 4)
    for args in [(5, 2, 2, 0, 0, 3), (5, 1, 3, 0, 0, 3), (5, 1, 2, 1, 0, 3), (5, 1, 2, 0, 1, 3),
                 (5, 1, 2, 0, 0, 4), (6, 1, 2, 0, 0, 3)]:
        assert not np.allclose(base, oracle.normals(*args, 4))


def test_single_precision_normals_close_to_double():
    z64 = oracle.normals_bulk(3, 1, 1, 0, 1, 5, 20000)
    z32 = oracle.normals_bulk(3, 1, 1, 0, 1, 5, 20000, precision="f32")
    assert np.max(np.abs(z64 - z32)) < 2e-5
