"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle (Sec. 3, Steps 1-7 of the paper) against one of:
numpy's weighted mean / covariance (library routines), closed forms derived by
hand from the paper's definitions, exact rational arithmetic, brute force over
permutations, and invariants of the method (partition, conservation, the
stop/argmax/cut rules at every node, Jensen's inequality for the energy).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1504_00636_gb300 import synth


def np_stats(pos, mom, w, L=(1.0, 1.0, 1.0)):
    """W, Q, sigma, Delta of one set via numpy's weighted average/covariance."""
    q = np.concatenate([np.atleast_2d(pos), np.atleast_2d(mom)])
    dx = np.atleast_2d(pos).shape[0]
    W = float(np.sum(w))
    Q = np.average(q, axis=1, weights=w)
    sig = np.array([math.sqrt(max(0.0, float(np.cov(q[l], aweights=w, bias=True))))
                    if q.shape[1] > 1 else 0.0 for l in range(q.shape[0])])
    delta = np.empty_like(sig)
    for l in range(q.shape[0]):
        if l < dx:
            delta[l] = sig[l] / L[l]
        elif sig[l] == 0.0:
            delta[l] = 0.0
        elif Q[l] == 0.0:
            delta[l] = math.inf
        else:
            delta[l] = sig[l] / abs(Q[l])
    return W, Q, sig, delta


# ---------------------------------------------------------------- Steps 1-2

@pytest.mark.parametrize("dx,dp,weights", [(1, 3, "uniform"), (2, 3, "lognormal"),
                                           (3, 3, "lognormal"), (1, 1, "uniform")])
def test_moments_match_numpy(dx, dp, weights):
    rng = np.random.default_rng(11)
    for m in (1, 2, 3, 17, 400):
        p = synth.random_cell(rng, m, dx, dp, weights=weights, drift=(-0.4, 0.2, 0.05))
        L = (0.5, 2.0, 1.0)
        W, Q, S, Dl = oracle.subset_moments(p.pos, p.mom, p.w, L)
        W2, Q2, S2, D2 = np_stats(p.pos, p.mom, p.w, L)
        assert W == pytest.approx(W2, rel=1e-14)
        np.testing.assert_allclose(Q, Q2, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(S, S2, rtol=1e-10, atol=1e-15)
        np.testing.assert_allclose(Dl, D2, rtol=1e-10, atol=1e-15)


def test_momentum_cv_uses_magnitude_of_mean():
    # Eq. cv_p with a negative mean momentum: the CV is sigma / |P|
    w = np.array([1.0, 1.0])
    pos = np.array([[0.5, 0.5]])
    mom = np.array([[-1.0, -3.0]])
    _, Q, S, Dl = oracle.subset_moments(pos, mom, w)
    assert Q[1] == -2.0 and S[1] == 1.0 and Dl[1] == 0.5


def test_identical_values_have_zero_sigma():
    w = np.array([0.3, 0.7, 1.9])
    pos = np.full((1, 3), 0.1)
    mom = np.full((3, 3), 0.1)
    _, _, S, Dl = oracle.subset_moments(pos, mom, w)
    assert np.all(S == 0.0) and np.all(Dl == 0.0)


# ------------------------------------------------- closed forms, two particles

def _pair(a, b, axis, w=(1.0, 1.0), dx=1):
    pos = np.full((dx, 2), 0.5)
    mom = np.full((3, 2), 1.0)
    if axis < dx:
        pos[axis] = (a, b)
    else:
        mom[axis - dx] = (a, b)
    return np.zeros(2, np.int32), pos, mom, np.array(w, dtype=float)


@pytest.mark.parametrize("a,b,tol", [(1.0, 1.2, 0.1), (1.0, 1.2, 0.05), (-2.0, -2.5, 0.12),
                                     (-2.0, -2.5, 0.1), (0.3, -0.1, 1.9), (0.3, -0.1, 2.1)])
def test_two_particles_momentum_closed_form(a, b, tol):
    # equal weights: sigma = |a-b|/2, P = (a+b)/2, so Delta = |a-b|/|a+b|
    cv = abs(a - b) / abs(a + b)
    cell, pos, mom, w = _pair(a, b, axis=1)
    r = oracle.merge(cell, pos, mom, w, 1, tol_x=1.0, tol_p=tol)
    if cv <= tol:
        assert r.count == 1
        assert r.w[0] == 2.0
        assert r.mom[0, 0] == pytest.approx((a + b) / 2, rel=1e-15)
    else:
        assert r.count == 2
        # V1 = {q <= Q} first
        assert list(r.mom[0]) == sorted([a, b])


@pytest.mark.parametrize("w1,w2", [(1.0, 3.0), (0.25, 2.0)])
def test_two_particles_weighted_closed_form(w1, w2):
    # sigma = sqrt(w1 w2)|a-b|/W and P = (w1 a + w2 b)/W
    a, b = 1.0, 1.5
    cv = math.sqrt(w1 * w2) * abs(a - b) / abs(w1 * a + w2 * b)
    cell, pos, mom, w = _pair(a, b, axis=1, w=(w1, w2))
    for tol, expect in ((cv * 1.001, 1), (cv * 0.999, 2)):
        r = oracle.merge(cell, pos, mom, w, 1, tol_x=1.0, tol_p=tol)
        assert r.count == expect
    r = oracle.merge(cell, pos, mom, w, 1, tol_x=1.0, tol_p=cv * 1.001)
    assert r.w[0] == w1 + w2
    assert r.mom[0, 0] == pytest.approx((w1 * a + w2 * b) / (w1 + w2), rel=1e-15)


@pytest.mark.parametrize("L", [1.0, 0.25])
def test_two_particles_position_closed_form(L):
    # Eq. cv_x: sigma/L with sigma = |a-b|/2 for equal weights
    a, b = 0.2 * L, 0.6 * L
    cv = abs(a - b) / (2 * L)
    cell, pos, mom, w = _pair(a, b, axis=0)
    for tol, expect in ((cv * 1.001, 1), (cv * 0.999, 2)):
        r = oracle.merge(cell, pos, mom, w, 1, cell_size=(L,), tol_x=tol, tol_p=1.0)
        assert r.count == expect


def test_stop_test_is_less_or_equal():
    # Step 3 "less than or equal": p = 1 and 3 give Delta = 0.5 exactly
    cell, pos, mom, w = _pair(1.0, 3.0, axis=1)
    assert oracle.merge(cell, pos, mom, w, 1, tol_x=1.0, tol_p=0.5).count == 1
    assert oracle.merge(cell, pos, mom, w, 1, tol_x=1.0, tol_p=np.nextafter(0.5, 0)).count == 2


# --------------------------------------------------- hand-worked small cases

def test_hand_worked_four_particles():
    # x = 0.1, 0.2, 0.8, 0.9 (L = 1), p = 1, w = 1, T_X = 0.2, T_P = 0.1.
    # Root: X = 0.5, sigma_x = sqrt((.16+.09+.09+.16)/4) = 0.35355 > 0.2 and
    # sigma_p = 0, so the cut is on x at 0.5: V1 = {0.1, 0.2}, V2 = {0.8, 0.9}.
    # Each child has sigma_x = 0.05 <= 0.2: two leaves, X = 0.15 and 0.85.
    order = [3, 0, 2, 1]  # input order 0.9, 0.1, 0.8, 0.2
    xs = np.array([[0.1, 0.2, 0.8, 0.9]])[:, order]
    mom = np.ones((1, 4))
    w = np.ones(4)
    cell = np.zeros(4, np.int32)
    r = oracle.merge(cell, xs, mom, w, 1, tol_x=0.2, tol_p=0.1)
    assert r.count == 2
    np.testing.assert_allclose(r.pos[0], [0.15, 0.85], rtol=1e-15)
    assert list(r.w) == [2.0, 2.0]
    assert list(r.index) == [1, 0, 1, 0]
    # T_X = 0.04 < 0.05: both children split again into singletons, in x order
    r = oracle.merge(cell, xs, mom, w, 1, tol_x=0.04, tol_p=0.1)
    assert r.count == 4
    assert list(r.pos[0]) == [0.1, 0.2, 0.8, 0.9]
    assert list(r.index) == [3, 0, 2, 1]


def test_argmax_picks_largest_cv_axis():
    # Delta_x = 0.3/1 (x = 0.2, 0.8) and Delta_p = 0.5 (p = 1, 3): p is cut first.
    # The p-children {p=1}, {p=3} are singletons whatever x is.
    pos = np.array([[0.2, 0.8, 0.2, 0.8]])
    mom = np.array([[1.0, 1.0, 3.0, 3.0]])
    w = np.ones(4)
    t = oracle.trace(pos, mom, w, tol_x=0.1, tol_p=0.1)
    assert t.axis[0] == 1 and t.Q[0] == 2.0
    # children: {p = 1} then {p = 3}; each then cut on x
    assert set(t.perm[t.begin[1]:t.end[1]]) == {0, 1}
    assert t.axis[1] == 0


def test_identical_particles_never_split():
    m = 7
    cell = np.zeros(m, np.int32)
    pos = np.full((2, m), 0.37)
    mom = np.full((3, m), -0.21)
    w = np.linspace(0.5, 2.0, m)
    r = oracle.merge(cell, pos, mom, w, 1, tol_x=0.0, tol_p=0.0)
    assert r.count == 1
    assert r.w[0] == pytest.approx(w.sum(), rel=1e-15)
    assert np.all(r.index == 0)


def test_passthrough_at_or_below_n_min():
    rng = np.random.default_rng(3)
    cells = np.array([0, 1, 1, 0, 1, 2, 2, 1], np.int32)
    pos = rng.random((1, 8)) + cells
    mom = rng.normal(0.3, 0.1, (3, 8))
    w = rng.random(8) + 0.5
    r = oracle.merge(cells, pos, mom, w, 3, n_min=4, tol_x=0.01, tol_p=0.01)
    # every cell has <= 4 particles: verbatim copies, cells ascending, input order
    order = np.argsort(cells, kind="stable")
    assert r.count == 8
    np.testing.assert_array_equal(r.pos[0], pos[0, order])
    np.testing.assert_array_equal(r.w, w[order])
    np.testing.assert_array_equal(r.cell, cells[order])
    assert list(r.index[order]) == list(range(8))


# ------------------------------------------------------ invariants per node

def _check_tree(p, tol_x, tol_p, L=(1.0, 1.0, 1.0)):
    t = oracle.trace(p.pos, p.mom, p.w, L, tol_x, tol_p)
    D = p.dx + p.dp
    q = np.concatenate([p.pos, p.mom])
    tol = [tol_x] * p.dx + [tol_p] * p.dp
    m = p.w.shape[0]
    assert sorted(t.perm) == list(range(m))
    leaves = []
    for j in range(len(t.begin)):
        b, e = t.begin[j], t.end[j]
        mem = t.perm[b:e]
        assert e > b
        W, Q, S, Dl = np_stats(p.pos[:, mem], p.mom[:, mem], p.w[mem], L)
        ok = all(Dl[l] <= tol[l] for l in range(D))
        if t.axis[j] < 0:
            assert ok or t.near
            leaves.append((b, e))
            continue
        assert (not ok) or t.near
        k = t.axis[j]
        assert Dl[k] == pytest.approx(np.max(Dl), rel=1e-9) or t.near
        assert t.Q[j] == pytest.approx(Q[k], rel=1e-12, abs=1e-15)
        # children: V1 = {q <= Q} then V2 = {q > Q}, both contiguous and non-empty
        kids = [i for i in range(len(t.begin))
                if t.depth[i] == t.depth[j] + 1 and b <= t.begin[i] < e]
        assert len(kids) == 2
        v1, v2 = sorted(kids, key=lambda i: t.begin[i])
        assert t.begin[v1] == b and t.end[v2] == e and t.end[v1] == t.begin[v2]
        assert np.all(q[k, t.perm[t.begin[v1]:t.end[v1]]] <= t.Q[j])
        assert np.all(q[k, t.perm[t.begin[v2]:t.end[v2]]] > t.Q[j])
    # leaves tile the set in order (V1-first depth-first)
    leaves.sort()
    assert leaves[0][0] == 0 and leaves[-1][1] == m
    assert all(leaves[i][1] == leaves[i + 1][0] for i in range(len(leaves) - 1))
    return t


@pytest.mark.parametrize("seed", range(6))
def test_tree_invariants_random_cells(seed):
    rng = np.random.default_rng(100 + seed)
    dx = 1 + seed % 3
    p = synth.random_cell(rng, 60 + 40 * seed, dx, 3, drift=(0.3, -0.2, 0.1),
                          weights="lognormal" if seed % 2 else "uniform")
    _check_tree(p, 0.3, 0.15)


def test_tree_invariants_counter_beams_cell():
    p = synth.counter_beams(cells=1)
    t = _check_tree(p, 0.1, 0.1)
    assert t.near == 0


# ------------------------------------------------------- merge-level checks

def _conservation(p, r):
    for c in range(p.n_cells):
        mi = p.cell == c
        mo = r.cell == c
        W_in, W_out = p.w[mi].sum(), r.w[mo].sum()
        assert abs(W_out - W_in) <= 1e-12 * W_in
        for l in range(p.dp):
            s_in = np.sum(p.w[mi] * p.mom[l, mi])
            s_out = np.sum(r.w[mo] * r.mom[l, mo])
            scale = np.sum(p.w[mi] * np.abs(p.mom[l, mi]))
            assert abs(s_out - s_in) <= 1e-12 * scale


def test_conservation_and_partition_counter_beams():
    p = synth.counter_beams()
    r = oracle.merge_particles(p)
    _conservation(p, r)
    # index maps every particle into its own cell's outputs
    assert np.all(r.cell[r.index] == p.cell)
    assert np.all(np.diff(r.cell) >= 0)
    # every output slot is used
    assert np.array_equal(np.unique(r.index), np.arange(r.count))


def test_energy_does_not_increase():
    # Jensen: sqrt(1+|p|^2) is convex, so a centroid never carries more energy
    p = synth.counter_beams()
    for tol in (0.1, 0.3, 1.0):
        r = oracle.merge_particles(p, tol_x=tol, tol_p=tol)
        e_in = np.sum(p.w * (np.sqrt(1 + np.sum(p.mom ** 2, axis=0)) - 1))
        e_out = np.sum(r.w * (np.sqrt(1 + np.sum(r.mom ** 2, axis=0)) - 1))
        assert e_out <= e_in * (1 + 1e-14)
        assert r.stats["energy_in"] == pytest.approx(e_in, rel=1e-12)
        assert r.stats["energy_out"] == pytest.approx(e_out, rel=1e-12)


def test_position_cv_bounded_so_tx_half_equals_one():
    # in-cell positions give Delta_x <= 1/2, so T_X = 0.5 and T_X = 1.0 run the
    # same algorithm (the two curves of the tolerance scan coincide, Sec. 4.3)
    p = synth.shower(grid=(8, 8))
    a = oracle.merge_particles(p, tol_x=0.5, tol_p=0.05)
    b = oracle.merge_particles(p, tol_x=1.0, tol_p=0.05)
    assert a.count == b.count
    np.testing.assert_array_equal(a.index, b.index)
    np.testing.assert_array_equal(a.mom, b.mom)


def test_threads_do_not_change_result():
    p = synth.two_stream(cells=64)
    a = oracle.merge_particles(p, threads=1)
    b = oracle.merge_particles(p, threads=4)
    assert a.count == b.count
    np.testing.assert_array_equal(a.index, b.index)
    np.testing.assert_array_equal(a.mom, b.mom)
    np.testing.assert_array_equal(a.w, b.w)


# ------------------------------------------------------------- metamorphic

def _partition(r, n):
    groups = {}
    for i in range(n):
        groups.setdefault(int(r.index[i]), set()).add(i)
    return sorted(tuple(sorted(g)) for g in groups.values())


def test_permutation_invariance_brute_force():
    rng = np.random.default_rng(5)
    p = synth.random_cell(rng, 6, 1, 3, drift=(0.3, 0.1, -0.2), spread=0.1)
    base = oracle.merge_particles(p, tol_x=0.3, tol_p=0.2)
    ref = _partition(base, 6)
    for perm in itertools.permutations(range(6)):
        perm = np.array(perm)
        r = oracle.merge(p.cell, p.pos[:, perm], p.mom[:, perm], p.w[perm], 1,
                         tol_x=0.3, tol_p=0.2)
        got = sorted(tuple(sorted(int(perm[i]) for i in g)) for g in _partition(r, 6))
        assert got == ref
        assert r.count == base.count


def test_scaling_by_powers_of_two_is_exact():
    p = synth.two_stream(cells=8)
    r0 = oracle.merge_particles(p)
    for k in (-3, 5):
        s = 2.0 ** k
        r = oracle.merge(p.cell, p.pos, p.mom * s, p.w * s, p.n_cells, tol_x=p.tol_x,
                         tol_p=p.tol_p)
        np.testing.assert_array_equal(r.index, r0.index)
        np.testing.assert_array_equal(r.mom, r0.mom * s)
        np.testing.assert_array_equal(r.w, r0.w * s)


def test_reflection_of_momentum_axis():
    p = synth.two_stream(cells=8)
    r0 = oracle.merge_particles(p)
    mom = p.mom.copy()
    mom[0] = -mom[0]
    r = oracle.merge(p.cell, p.pos, mom, p.w, p.n_cells, tol_x=p.tol_x, tol_p=p.tol_p)
    # same partition into sets (the order of the two sides of a p_x cut flips)
    assert r.count == r0.count
    assert _partition(r, p.n) == _partition(r0, p.n)


# ------------------------------------------------------------ exact rational

@pytest.mark.parametrize("seed", range(8))
def test_fp64_oracle_equals_exact_rational(seed):
    rng = np.random.default_rng(200 + seed)
    dx = 1 + seed % 3
    p = synth.random_cell(rng, 8 + 4 * seed, dx, 3, drift=(0.25, -0.1, 0.05),
                          weights="lognormal" if seed % 2 else "uniform")
    r = oracle.merge_particles(p, tol_x=0.2, tol_p=0.15)
    idx, out = exact.merge(p.cell, p.pos, p.mom, p.w, 1, tol_x=0.2, tol_p=0.15)
    if r.flags[0]:
        pytest.skip("near tie")
    assert r.count == len(out)
    assert list(r.index) == idx
    for j, (c, W, coords) in enumerate(out):
        assert r.w[j] == pytest.approx(float(W), rel=1e-14)
        got = np.concatenate([r.pos[:, j], r.mom[:, j]])
        np.testing.assert_allclose(got, [float(x) for x in coords], rtol=1e-13, atol=1e-15)


def test_exact_rational_on_counter_beams_cells():
    p = synth.counter_beams(cells=2, per_cell=24)
    r = oracle.merge_particles(p)
    idx, out = exact.merge(p.cell, p.pos, p.mom, p.w, p.n_cells, tol_x=p.tol_x,
                           tol_p=p.tol_p)
    assert not r.flags.any()
    assert list(r.index) == idx


def test_particle_on_the_centroid_goes_to_v1():
    # Step 5: V1 = {q <= Q}.  x = 0.25, 0.5, 0.75 gives Q = 0.5 exactly.
    pos = np.array([[0.75, 0.5, 0.25]])
    mom = np.ones((1, 3))
    t = oracle.trace(pos, mom, np.ones(3), tol_x=0.1, tol_p=0.1)
    assert t.axis[0] == 0 and t.Q[0] == 0.5
    assert set(t.perm[t.begin[1]:t.end[1]]) == {1, 2}
