"""Pins of the oracle's mass-transfer update (Sec. 3: K_ij Gaussian of
variance h^2 = 2 D_MT dt / beta, W_ij = K_ij / (1/2 (sum_i K_ij + sum_j K_ij)),
delta_i = sum_j beta (M_j - M_i) W_ij, explicit update).  The expected
values are hand-derived closed forms, invariants and special cases."""
import numpy as np
import pytest

import oracle as O


def _p(dim=2, D=1.0, kappa=0.5, dt=0.1, beta=1.0, lam=3.0, hi=100.0):
    return O.OracleParams(dim=dim, D=D, kappa=kappa, dt=dt, beta=beta, lam=lam,
                          lo=(0.0, 0.0, 0.0), hi=(hi, hi, hi), seed=1)


def test_derived_parameters():
    d = O.derived(_p(D=1.0, kappa=0.5, dt=0.1))
    assert d["D_RW"] == 0.5 and d["D_MT"] == 0.5
    assert abs(d["h2"] - 0.1) < 1e-17
    assert abs(d["psi"] - 3.0 * np.sqrt(4 * 0.5 * 0.1)) < 1e-15    # 6 sqrt(D_MT dt)
    assert abs(d["sigma"] - np.sqrt(0.1)) < 1e-16
    assert abs(d["kernel_norm"] - 1.0 / (2 * np.pi * 0.1)) < 1e-14
    d3 = O.derived(_p(dim=3, D=1.0, dt=0.05))
    assert abs(d3["kernel_norm"] - (2 * np.pi * 0.05) ** -1.5) < 1e-12


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("method", ["brute", "kdtree"])
def test_two_particle_closed_form(dim, method):
    # r_1 = r_2 = c (1 + e) with e = exp(-r^2 / (2 h^2)), so W_12 = e / (1 + e)
    # and delta_1 = beta (M_2 - M_1) e / (1 + e) = -delta_2.
    p = _p(dim=dim, beta=0.8)
    h2 = O.derived(p)["h2"]
    r = 0.7
    pos = np.zeros((dim, 2)) + 50.0
    pos[0, 1] += r
    M = np.array([0.2, 1.3])
    new, rs, cs, npairs = O.mass_transfer(p, pos, M, method)
    assert npairs == 2
    e = np.exp(-r * r / (2 * h2))
    c = (2 * np.pi * h2) ** (-dim / 2)
    np.testing.assert_allclose(rs, c * (1 + e), rtol=1e-14)
    np.testing.assert_allclose(cs, c * (1 + e), rtol=1e-14)
    d1 = 0.8 * (M[1] - M[0]) * e / (1 + e)
    np.testing.assert_allclose(new, [M[0] + d1, M[1] - d1], rtol=1e-14)


def test_three_collinear_particles_hand_case():
    # spacing s with s <= psi < 2 s: pairs (1,2), (2,3) only.
    # r_1 = r_3 = c (1 + e), r_2 = c (1 + 2 e); W_12 = W_23 = 2 e / (2 + 3 e).
    p = _p()
    d = O.derived(p)
    s = 0.9
    assert s <= d["psi"] < 2 * s
    pos = np.array([[10.0, 10.0 + s, 10.0 + 2 * s], [5.0, 5.0, 5.0]])
    M = np.array([1.0, 0.25, -0.5])
    new, rs, cs, npairs = O.mass_transfer(p, pos, M)
    assert npairs == 4
    e = np.exp(-s * s / (2 * d["h2"]))
    w = 2 * e / (2 + 3 * e)
    expect = [M[0] + (M[1] - M[0]) * w,
              M[1] + ((M[0] - M[1]) + (M[2] - M[1])) * w,
              M[2] + (M[1] - M[2]) * w]
    np.testing.assert_allclose(new, expect, rtol=1e-14, atol=1e-16)


def _random_case(dim, n, L, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, size=(dim, n))
    M = rng.uniform(0, 1, size=n)
    return pos, M


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_uniform_masses_are_invariant_bit_exactly(dim):
    pos, _ = _random_case(dim, 800, {1: 200.0, 2: 20.0, 3: 8.0}[dim], 3)
    M = np.full(800, 0.625)
    new, _, _, npairs = O.mass_transfer(_p(dim=dim), pos, M)
    assert npairs > 0
    assert np.array_equal(new, M)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_conservation_symmetry_and_maximum_principle(dim):
    pos, M = _random_case(dim, 1500, {1: 150.0, 2: 12.0, 3: 5.0}[dim], 4)
    new, rs, cs, npairs = O.mass_transfer(_p(dim=dim), pos, M)
    assert npairs > 0
    # K symmetric => row sums equal column sums (up to summation order)
    np.testing.assert_allclose(rs, cs, rtol=1e-14)
    # W symmetric => sum_i delta_i = 0 up to rounding
    assert abs(new.sum() - M.sum()) <= 1e-13 * np.abs(M).sum()
    # beta = 1, sum_j W_ij <= 1 here => convex combination => maximum principle
    assert new.min() >= M.min() - 1e-15 and new.max() <= M.max() + 1e-15
    assert np.any(new != M)


def test_brute_and_kdtree_transfer_agree():
    pos, M = _random_case(2, 1200, 15.0, 5)
    a = O.mass_transfer(_p(), pos, M, "brute")
    b = O.mass_transfer(_p(), pos, M, "kdtree")
    assert a[3] == b[3]
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-15)


def test_no_transfer_without_mass_transfer_diffusion():
    pos, M = _random_case(2, 500, 10.0, 6)
    new, rs, cs, npairs = O.mass_transfer(_p(kappa=1.0), pos, M)
    assert npairs == 0 and np.array_equal(new, M)


def test_isolated_particles_keep_their_mass():
    pos = np.array([[0.0, 50.0, 99.0], [0.0, 50.0, 99.0]])
    M = np.array([1.0, 2.0, 3.0])
    new, rs, cs, npairs = O.mass_transfer(_p(), pos, M)
    assert npairs == 0 and np.array_equal(new, M)
    np.testing.assert_allclose(rs, O.derived(_p())["kernel_norm"], rtol=0)
