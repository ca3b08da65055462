"""Pins of the oracle's random stream (CPU only).

Philox4x32-10 is pinned to the generator's published known-answer vectors
and to an independent implementation (cuRAND's host generator); the uniform
recipes are pinned to their exact end points; the normal/exponential draws are
checked against their laws.
"""
import ctypes
import glob
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat_rows())
def test_philox_known_answers(orc, ctr, key, want):
    assert orc.philox4x32_10(ctr, key) == want


def _curand_host():
    cands = sorted(glob.glob("/usr/local/cuda/lib64/libcurand.so*"))
    if not cands:
        return None
    try:
        lib = ctypes.CDLL(cands[0])
    except OSError:
        return None
    return lib


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF])
def test_philox_matches_curand_host_generator(orc, seed):
    """cuRAND's host PHILOX4_32_10 generator, seeded with s, emits the blocks
    philox(ctr=(0,0,j,0), key=(s_lo, s_hi)) for consecutive j (its
    subsequence layout).  Every oracle block j = 1..64 must appear in that
    output, in order and contiguous."""
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    rc = lib.curandCreateGeneratorHost(ctypes.byref(gen), 161)  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    if rc != 0:
        pytest.skip("curand host generator unavailable (status %d)" % rc)
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4096
        buf = (ctypes.c_uint32 * n)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        words = list(buf)
    finally:
        lib.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    blocks = [orc.philox4x32_10([0, 0, j, 0], key) for j in range(1, 65)]
    first = blocks[0]
    pos = next(i for i in range(len(words) - 4) if words[i:i + 4] == first)
    flat = [w for b in blocks for w in b]
    assert words[pos:pos + len(flat)] == flat


def test_uniform_recipes_end_points(orc):
    L = orc.lib()
    assert L.orc_uniform24(0) == 2.0 ** -24
    assert L.orc_uniform24(0xFFFFFFFF) == 1.0
    assert L.orc_uniform24(0x000000FF) == 2.0 ** -24          # low 8 bits dropped
    assert L.orc_uniform53(0, 0) == 2.0 ** -53
    assert L.orc_uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0
    # 32 bits of the first word land in bits 21..52, 21 bits of the second in 0..20
    assert L.orc_uniform53(1, 0) == (2.0 ** 21 + 1) * 2.0 ** -53
    assert L.orc_uniform53(0, 1 << 11) == 2.0 * 2.0 ** -53


@pytest.mark.parametrize("recipe", [0, 1])
def test_stream_draws_follow_their_laws(orc, recipe):
    """nu ~ N(0,1), chi ~ N(0,1), E ~ Exp(1) over many counters; nu and chi
    from one Box-Muller pair are uncorrelated."""
    p = orc.Problem(eps=1.0, T=1.0, dt0=1.0, recipe=recipe, seed=7)
    nus, Es, chis = [], [], []
    for pair in range(400):
        _, nu, E, chi = orc.stream_draws(p, 1, pair, 50)
        nus.append(nu); Es.append(E); chis.append(chi)
    nu, E, chi = np.concatenate(nus), np.concatenate(Es), np.concatenate(chis)
    assert stats.kstest(nu, "norm").pvalue > 1e-3
    assert stats.kstest(chi, "norm").pvalue > 1e-3
    assert stats.kstest(E, "expon").pvalue > 1e-3
    assert abs(np.corrcoef(nu, chi)[0, 1]) < 4.0 / np.sqrt(len(nu))


def test_streams_differ_by_level_pair_request_seed(orc):
    base = orc.Problem(eps=1.0, T=1.0, dt0=1.0, seed=3)
    ref = orc.stream_draws(base, 2, 5, 4)[1]
    for kw, lev, pair in [({}, 3, 5), ({}, 2, 6), ({"request": 1}, 2, 5), ({"seed": 4}, 2, 5)]:
        p = orc.Problem(eps=1.0, T=1.0, dt0=1.0, seed=kw.get("seed", 3), request=kw.get("request", 0))
        other = orc.stream_draws(p, lev, pair, 4)[1]
        assert not np.array_equal(ref, other)
    # same counter, same draws
    assert np.array_equal(ref, orc.stream_draws(base, 2, 5, 4)[1])


def test_uniformity_chi_square(orc):
    """Top byte of 2^18 Philox words over a counter sweep: chi-square over 256 cells."""
    words = []
    for j in range(1 << 16):
        words.extend(orc.philox4x32_10([j, 11, 0, 0], [1, 2]))
    top = np.array(words, np.uint64) >> 24
    counts = np.bincount(top.astype(np.int64), minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4
