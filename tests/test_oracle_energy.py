"""Pins of the oracle's energy-conserving replacement (VAR_CONSERVE_ENERGY):
every final set of m >= 3 particles becomes two particles of weight W/2 at
the centroid X with momenta P + d, P - d that keep W, W P and the total
energy sum w sqrt(1 + |p|^2).  Checked against the conservation laws, a
hand-worked set, a numerical root of the one-axis equation, the literal
run's partition, and the rule for the direction of d."""
import math

import numpy as np
import pytest

import oracle
from paper_1504_00636_gb300 import synth

EC = oracle.VAR_CONSERVE_ENERGY


def gamma(mom):
    return np.sqrt(1.0 + np.sum(np.atleast_2d(mom) ** 2, axis=0))


def test_hand_worked_three_particles():
    # p_x = 0.75, 2.4, 0 (gamma 5/4, 13/5, 1), w = 1: W = 3, P = (1.05, 0, 0),
    # E = 4.85, g = 97/60, |d|^2 = g^2 - 1 - P^2 = 23/45.  Every
    # sigma_k^2 (1 - Phat_k^2) is 0 (the spread is along P), so d takes the
    # first axis with the smallest |P_k|: y
    mom = np.array([[0.75, 2.4, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    pos = np.array([[0.2, 0.5, 0.8]])
    r = oracle.merge(np.zeros(3, np.int32), pos, mom, np.ones(3), 1, tol_x=1.0, tol_p=1.0,
                     variant=EC)
    assert r.count == 2
    np.testing.assert_array_equal(r.w, [1.5, 1.5])
    np.testing.assert_allclose(r.pos[0], [0.5, 0.5], rtol=1e-15)
    d = math.sqrt(23.0 / 45.0)
    np.testing.assert_allclose(r.mom[0], [1.05, 1.05], rtol=1e-14)
    np.testing.assert_allclose(r.mom[1], [d, -d], rtol=1e-13)
    np.testing.assert_array_equal(r.mom[2], [0.0, 0.0])
    assert list(r.index) == [0, 0, 0]


@pytest.mark.parametrize("make", [lambda: synth.counter_beams(cells=6),
                                  lambda: synth.two_stream(cells=12),
                                  lambda: synth.shower(grid=(10, 10), cap=3000)],
                         ids=["counter_beams", "two_stream", "shower"])
def test_conservation_per_cell(make):
    p = make()
    r = oracle.merge_particles(p, variant=EC)
    for c in np.unique(p.cell):
        mi, mo = p.cell == c, r.cell == c
        W = p.w[mi].sum()
        assert abs(r.w[mo].sum() - W) <= 1e-12 * W
        A = np.sum(p.w[mi] * np.abs(p.mom[:, mi]), axis=1)
        err = np.abs(np.sum(r.w[mo] * r.mom[:, mo], axis=1) - np.sum(p.w[mi] * p.mom[:, mi], axis=1))
        assert np.all(err <= 1e-12 * A + 1e-300)
        E_in = np.sum(p.w[mi] * gamma(p.mom[:, mi]))
        E_out = np.sum(r.w[mo] * gamma(r.mom[:, mo]))
        assert abs(E_out - E_in) <= 1e-12 * E_in
    # kinetic bookkeeping of the oracle agrees (W is conserved too)
    assert r.stats["energy_out"] == pytest.approx(r.stats["energy_in"], rel=1e-10)


def test_structure_against_the_literal_run():
    # Step 7 is the only change: the same final sets; a set of m >= 3 gives
    # two outputs of weight W/2 at X, with (p_a + p_b)/2 = P, p_a - P
    # orthogonal to P and |p_a| = |p_b| = sqrt(g^2 - 1); sets of 1 or 2 are
    # copied verbatim
    p = synth.two_stream(cells=8)
    lit = oracle.merge_particles(p)
    ec = oracle.merge_particles(p, variant=EC)
    n = p.n
    members = {}
    for i in range(n):
        members.setdefault(int(lit.index[i]), []).append(i)
    k = 0
    seen3 = 0
    for j in range(lit.count):
        mem = members[j]
        if len(mem) == 1:
            assert ec.w[k] == lit.w[j]
            k += 1
        elif len(mem) == 2:
            np.testing.assert_array_equal(np.sort(ec.w[k:k + 2]), np.sort(p.w[mem]))
            k += 2
        else:
            seen3 += 1
            W = lit.w[j]
            P = lit.mom[:, j]
            np.testing.assert_allclose(ec.w[k:k + 2], [W / 2, W / 2], rtol=1e-15)
            np.testing.assert_allclose(ec.pos[:, k], lit.pos[:, j], rtol=1e-15)
            pa, pb = ec.mom[:, k], ec.mom[:, k + 1]
            np.testing.assert_allclose((pa + pb) / 2, P, rtol=1e-12, atol=1e-15)
            g = np.sum(p.w[mem] * gamma(p.mom[:, mem])) / W
            assert np.dot(pa, pa) == pytest.approx(g * g - 1, rel=1e-10)
            assert np.dot(pb, pb) == pytest.approx(g * g - 1, rel=1e-10)
            assert abs(np.dot(pa - P, P)) <= 1e-9 * (np.dot(P, P) + 1e-300) ** 0.5 * np.linalg.norm(pa - P) + 1e-15
            assert ec.index[mem[0]] == k and all(ec.index[i] == k for i in mem)
            k += 2
    assert k == ec.count and seen3 > 0


def test_one_momentum_axis_matches_a_numerical_root():
    # dp = 1: P +- u with sqrt(1 + (P+u)^2) + sqrt(1 + (P-u)^2) = 2 g
    scipy = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(5)
    m = 7
    mom = rng.normal(0.4, 0.3, size=(1, m))
    w = rng.uniform(0.5, 2.0, m)
    r = oracle.merge(np.zeros(m, np.int32), rng.random((1, m)), mom, w, 1,
                     tol_x=1.0, tol_p=1e9, variant=EC)
    assert r.count == 2
    W = w.sum()
    P = np.sum(w * mom[0]) / W
    g = np.sum(w * gamma(mom)) / W
    f = lambda u: math.sqrt(1 + (P + u) ** 2) + math.sqrt(1 + (P - u) ** 2) - 2 * g
    u = scipy.brentq(f, 0.0, 10.0, xtol=1e-15)
    np.testing.assert_allclose(r.mom[0], [P + u, P - u], rtol=1e-12)


def test_direction_is_the_spread_axis_orthogonal_to_p():
    # P mostly along x; the largest raw variance is along x (the direction of
    # P), but the largest variance across P is along z: d points along z
    # (P_z != 0 so that the set is not split: Delta_z would be infinite)
    mom = np.array([[1.0, 2.0, 1.5, 1.5], [0.2, 0.2, 0.2, 0.2], [0.05, 0.05, 0.2, -0.1]])
    r = oracle.merge(np.zeros(4, np.int32), np.full((1, 4), 0.5), mom, np.ones(4), 1,
                     tol_x=1.0, tol_p=1e9, variant=EC)
    assert r.count == 2
    P = mom.mean(axis=1)
    d = r.mom[:, 0] - P
    d /= np.linalg.norm(d)
    assert abs(d[2]) > 0.99


def test_identical_momenta_give_d_zero():
    mom = np.tile([[0.3], [0.1], [-0.2]], (1, 5))
    r = oracle.merge(np.zeros(5, np.int32), np.full((1, 5), 0.5), mom, np.ones(5), 1,
                     tol_x=1.0, tol_p=0.1, variant=EC)
    assert r.count == 2
    np.testing.assert_allclose(r.mom[:, 0], mom[:, 0], rtol=1e-7)
    np.testing.assert_allclose(r.mom[:, 1], mom[:, 0], rtol=1e-7)


def test_energy_mode_changes_only_step7():
    p = synth.shower(grid=(8, 8))
    lit = oracle.merge_particles(p)
    ec = oracle.merge_particles(p, variant=EC)
    assert ec.stats["splits"] == lit.stats["splits"]
    assert ec.stats["leaves"] == lit.stats["leaves"]
    assert ec.count >= lit.count


def test_copied_pair_comes_out_in_input_order():
    # x = 0.9, 0.1, 0.8: the cut on x leaves {1} and the pair {0, 2}, which
    # stays whole (tol_x 0.1 > its Delta_x 0.05); the pair is copied with the
    # lower input index first
    pos = np.array([[0.9, 0.1, 0.8]])
    mom = np.full((1, 3), 1.0)
    w = np.array([1.0, 2.0, 3.0])
    r = oracle.merge(np.zeros(3, np.int32), pos, mom, w, 1, tol_x=0.1, tol_p=0.1, variant=EC)
    assert r.count == 3
    assert list(r.index) == [1, 0, 2]
    np.testing.assert_array_equal(r.w, [2.0, 1.0, 3.0])
    np.testing.assert_array_equal(r.pos[0], [0.1, 0.9, 0.8])
