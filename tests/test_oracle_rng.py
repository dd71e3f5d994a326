"""Pins of the oracle's random-number path (Sec. 3 random walk: xi_i standard
normal; the generator itself is this project's reading, the paper names none).

Pinned to things other than the oracle: a third-party Philox4x32-10 (PyTorch's
host-side engine, called as a library routine) word for word over random and
edge-case counters and keys; numpy's float64 log/sin/cos (library routines)
over every input the walk can produce; the float64 Box-Muller formula on the
library's words; the N(0,1) distribution (Kolmogorov-Smirnov and moments);
and the avalanche / uniformity properties of a correct 10-round Philox.
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from philox_library import philox4x32_10 as library_philox

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_log_f32_matches_library_log_on_every_uniform():
    k = np.arange(1, 2 ** 24 + 1, dtype=np.uint32)
    u = k.astype(np.float32) * np.float32(2.0 ** -24)
    assert np.all(u.astype(np.float64) == k.astype(np.float64) * 2.0 ** -24)  # exact uniforms
    got = O.log_f32(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    assert got[-1] == 0.0                       # ln 1 = 0 exactly
    nz = ref != 0
    ulp = np.spacing(np.abs(ref[nz]).astype(np.float32)).astype(np.float64)
    err_ulp = np.abs(got[nz] - ref[nz]) / ulp
    assert err_ulp.max() <= 2.0, err_ulp.max()


def test_sincos_matches_library_on_every_angle():
    k = np.arange(0, 2 ** 24 + 1, dtype=np.uint32)
    s, c = O.sincos_2pi_f32(k)
    th = 2.0 * np.pi * k.astype(np.float64) / 2.0 ** 24
    assert np.abs(s - np.sin(th)).max() <= 2.0 * 2.0 ** -24
    assert np.abs(c - np.cos(th)).max() <= 2.0 * 2.0 ** -24
    # quadrant points are exact
    for kk, (es, ec) in {0: (0.0, 1.0), 2 ** 22: (1.0, 0.0), 2 ** 23: (0.0, -1.0),
                         3 * 2 ** 22: (-1.0, 0.0), 2 ** 24: (0.0, 1.0)}.items():
        ss, cc = O.sincos_2pi_f32([kk])
        assert abs(ss[0]) == abs(es) and abs(cc[0]) == abs(ec)
        assert np.sign(ss[0]) * abs(es) == es and np.sign(cc[0]) * abs(ec) == ec


def test_normals_are_standard_normal():
    z = O.normals(2204037561, np.arange(500_000), 3)
    assert z.dtype == np.float32 and z.shape == (500_000, 4)
    flat = z.astype(np.float64).ravel()
    ks = stats.kstest(flat, "norm")
    assert ks.pvalue > 1e-4, ks
    n = flat.size
    assert abs(flat.mean()) < 5 / np.sqrt(n)
    assert abs(flat.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(stats.skew(flat)) < 5 * np.sqrt(6.0 / n)
    assert abs(stats.kurtosis(flat)) < 5 * np.sqrt(24.0 / n)
    # the four draws of one counter are uncorrelated, and so are steps
    cc = np.corrcoef(z.astype(np.float64).T)
    assert np.abs(cc - np.eye(4)).max() < 5 / np.sqrt(500_000)
    z2 = O.normals(2204037561, np.arange(500_000), 4)
    assert abs(np.corrcoef(z[:, 0], z2[:, 0])[0, 1]) < 5 / np.sqrt(500_000)
    # Box-Muller with 24-bit uniforms: |z| <= sqrt(-2 ln 2^-24)
    assert np.abs(flat).max() <= np.sqrt(-2.0 * np.log(2.0 ** -24)) + 1e-5


def test_normals_are_a_pure_function_of_seed_id_step():
    a = O.normals(7, np.array([5, 9, 5]), 11)
    assert np.array_equal(a[0], a[2])
    assert not np.array_equal(a[0], a[1])
    b = O.normals(8, np.array([5]), 11)
    assert not np.array_equal(a[0], b[0])
    c = O.normals(7, np.array([5]), 11 + (1 << 32))   # high half of the step is in the counter
    assert not np.array_equal(a[0], c[0])


def _bits(words):
    return np.unpackbits(words.view(np.uint8), axis=-1)


def test_philox_avalanche_and_uniformity():
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([0x12345678, 0x9ABCDEF0], dtype=np.uint32)
    base = O.philox4x32_10(ctr, key)
    # flipping any one counter bit flips each output bit with probability 1/2
    for word in range(4):
        for bit in (0, 13, 31):
            c2 = ctr.copy()
            c2[:, word] ^= np.uint32(1 << bit)
            flips = _bits(base ^ O.philox4x32_10(c2, key)).mean()
            assert abs(flips - 0.5) < 0.01, (word, bit, flips)
    # and so does flipping a key bit
    for kw in range(2):
        k2 = key.copy()
        k2[kw] ^= np.uint32(1 << 7)
        flips = _bits(base ^ O.philox4x32_10(ctr, k2)).mean()
        assert abs(flips - 0.5) < 0.01
    # byte histogram of sequential counters is uniform (chi-square)
    seq = np.zeros((1 << 16, 4), dtype=np.uint32)
    seq[:, 0] = np.arange(1 << 16, dtype=np.uint32)
    out = O.philox4x32_10(seq, key)
    counts = np.bincount(out.view(np.uint8).ravel(), minlength=256)
    chi = stats.chisquare(counts)
    assert chi.pvalue > 1e-4
    # distinct counters give distinct blocks
    assert len({tuple(r) for r in out[:20000].tolist()}) == 20000


def _edge_counters():
    """Counters whose words sit at 0, 1 and 2^32 - 1 in every combination
    (the carries and wrap-arounds of the round arithmetic)."""
    vals = np.array([0, 1, 0xFFFFFFFF], dtype=np.uint64)
    grid = np.stack(np.meshgrid(vals, vals, vals, vals, indexing="ij"), axis=-1)
    return grid.reshape(-1, 4).astype(np.uint32)


def test_philox_matches_an_independent_library_implementation():
    rng = np.random.default_rng(2204)
    keys = [np.array([0, 0], np.uint32), np.array([0xFFFFFFFF, 0xFFFFFFFF], np.uint32),
            np.array([0x243F6A88, 0x85A308D3], np.uint32)]
    keys += [rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
             for _ in range(5)]
    rand_ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    for key in keys:
        for ctr in (_edge_counters(), rand_ctr):
            got = O.philox4x32_10(ctr, key)
            ref = library_philox(ctr, key)
            assert np.array_equal(got, ref), (key, np.argwhere(got != ref)[:4])
    # the walk's counters: (id, step low word, step high word, 0) under the seed
    ids = np.arange(64, dtype=np.uint32)
    for seed, step in ((0, 0), (2204037561, 3), (2 ** 64 - 1, 2 ** 64 - 1), (7, 2 ** 32 + 5)):
        ctr = np.stack([ids, np.full_like(ids, step & 0xFFFFFFFF),
                        np.full_like(ids, step >> 32), np.zeros_like(ids)], axis=1)
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
        assert np.array_equal(O.philox4x32_10(ctr, key), library_philox(ctr, key))


def test_walk_normals_are_box_muller_of_the_library_words():
    ids = np.arange(0, 5000, 7, dtype=np.uint32)
    for seed, step in ((0, 0), (2204037561, 41), (2 ** 64 - 1, 2 ** 64 - 1)):
        ctr = np.stack([ids, np.full_like(ids, step & 0xFFFFFFFF),
                        np.full_like(ids, step >> 32), np.zeros_like(ids)], axis=1)
        words = library_philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        z = O.normals(seed, ids, step)
        assert np.array_equal(z, O.box_muller(words))
        # the word -> normal map against the Box-Muller formula in float64:
        # u = ((w >> 8) + 1) 2^-24, radius from words 0 and 2, angle from 1 and 3
        u = ((words >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0 ** -24
        rad = np.sqrt(-2.0 * np.log(u[:, [0, 2]]))
        th = 2.0 * np.pi * u[:, [1, 3]]
        ref = np.empty((ids.size, 4))
        ref[:, 0], ref[:, 1] = rad[:, 0] * np.cos(th[:, 0]), rad[:, 0] * np.sin(th[:, 0])
        ref[:, 2], ref[:, 3] = rad[:, 1] * np.cos(th[:, 1]), rad[:, 1] * np.sin(th[:, 1])
        assert np.abs(z - ref).max() <= 2e-6 * np.maximum(1.0, np.abs(ref)).max()
