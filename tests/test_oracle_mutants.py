"""The oracle's pins are sharp: plant plausible mistakes in a copy of the
oracle's C source (on the CPU) and check that the pins catch every one."""
import math
import multiprocessing
import os

import numpy as np
import pytest

import oracle
from paper_1504_00636_gb300 import synth


def pin_failures(lib):
    """Run a compact set of pins against ``lib``; return the names that fail."""
    fails = []

    def check(name, cond):
        if not cond:
            fails.append(name)

    z2 = np.zeros(2, np.int32)
    # two particles, momentum axis, negative mean: Delta = |a-b|/|a+b| = 0.2
    pos = np.full((1, 2), 0.5)
    mom = np.array([[-1.0, -1.5]])
    r = oracle.merge(z2, pos, mom, np.ones(2), 1, tol_x=1.0, tol_p=0.21, lib=lib)
    check("pair_merge", r.count == 1)
    r = oracle.merge(z2, pos, mom, np.ones(2), 1, tol_x=1.0, tol_p=0.19, lib=lib)
    check("pair_split", r.count == 2 and list(r.mom[0]) == [-1.5, -1.0])
    # weighted pair: Delta = sqrt(w1 w2)|a-b|/|w1 a + w2 b|
    w = np.array([1.0, 3.0])
    mom = np.array([[1.0, 1.5]])
    cv = math.sqrt(3.0) * 0.5 / 5.5
    r = oracle.merge(z2, pos, mom, w, 1, tol_x=1.0, tol_p=cv * 1.001, lib=lib)
    check("weighted_pair_merge", r.count == 1 and abs(r.mom[0, 0] - 5.5 / 4) < 1e-15
          and r.w[0] == 4.0)
    r = oracle.merge(z2, pos, mom, w, 1, tol_x=1.0, tol_p=cv * 0.999, lib=lib)
    check("weighted_pair_split", r.count == 2)
    # exact tie on the stop test: p = 1, 3 gives Delta = 0.5
    mom = np.array([[1.0, 3.0]])
    r = oracle.merge(z2, pos, mom, np.ones(2), 1, tol_x=1.0, tol_p=0.5, lib=lib)
    check("stop_le", r.count == 1)
    # particle on the centroid goes to V1, V1 comes out first
    t = oracle.trace(np.array([[0.75, 0.5, 0.25]]), np.ones((1, 3)), np.ones(3),
                     tol_x=0.1, tol_p=0.1, lib=lib)
    check("cut_le", t.axis[0] == 0 and set(t.perm[t.begin[1]:t.end[1]]) == {1, 2})
    # argmax: Delta_p = 0.5 beats Delta_x = 0.3
    t = oracle.trace(np.array([[0.2, 0.8, 0.2, 0.8]]), np.array([[1.0, 1.0, 3.0, 3.0]]),
                     np.ones(4), tol_x=0.1, tol_p=0.1, lib=lib)
    check("argmax", t.axis[0] == 1)
    # hand-worked order
    xs = np.array([[0.9, 0.1, 0.8, 0.2]])
    r = oracle.merge(np.zeros(4, np.int32), xs, np.ones((1, 4)), np.ones(4), 1,
                     tol_x=0.2, tol_p=0.1, lib=lib)
    check("order", list(r.index) == [1, 0, 1, 0])
    # numpy moments on a weighted random set
    rng = np.random.default_rng(1)
    p = synth.random_cell(rng, 50, 2, 3, weights="lognormal", drift=(-0.3, 0.2, 0.1))
    W, Q, S, Dl = oracle.subset_moments(p.pos, p.mom, p.w, lib=lib)
    q = np.concatenate([p.pos, p.mom])
    Qn = np.average(q, axis=1, weights=p.w)
    Sn = np.sqrt([np.cov(q[l], aweights=p.w, bias=True) for l in range(5)])
    check("moments", np.allclose(Q, Qn, rtol=1e-12) and np.allclose(S, Sn, rtol=1e-10))
    # conservation on a real workload
    p = synth.counter_beams(cells=4)
    r = oracle.merge_particles(p, lib=lib)
    ok = abs(r.w.sum() - p.w.sum()) < 1e-9 and all(
        abs(np.sum(r.w * r.mom[l]) - np.sum(p.w * p.mom[l])) < 1e-9 for l in range(3))
    check("conservation", ok)
    # momentum-norm variant: p = (0.6, 0.7, 0), (0.6, 0.9, 0); mean (0.6, 0.8, 0),
    # |P| = 1, sigma_y = 0.1, so Delta_y = 0.1 (the literal rule: 0.1/0.8)
    pos = np.full((1, 2), 0.5)
    mom = np.array([[0.6, 0.6], [0.7, 0.9], [0.0, 0.0]])
    r = oracle.merge(z2, pos, mom, np.ones(2), 1, tol_x=1.0, tol_p=0.11, lib=lib,
                     variant=oracle.VAR_PNORM)
    check("pnorm_merge", r.count == 1)
    r = oracle.merge(z2, pos, mom, np.ones(2), 1, tol_x=1.0, tol_p=0.09, lib=lib,
                     variant=oracle.VAR_PNORM)
    check("pnorm_split", r.count == 2)
    # normalised split axis: Delta_x = 0.3, Delta_p = 0.5; with T_X = 0.1 and
    # T_P = 0.25 the ratios are 3 and 2, so x is cut (the literal rule cuts p)
    xs, ps = np.array([[0.2, 0.8, 0.2, 0.8]]), np.array([[1.0, 1.0, 3.0, 3.0]])
    t = oracle.trace(xs, ps, np.ones(4), tol_x=0.1, tol_p=0.25, lib=lib,
                     variant=oracle.VAR_NORMALIZED)
    check("normalized_axis", t.axis[0] == 0)
    # T_X = 0: any position spread is an infinite ratio
    t = oracle.trace(xs, ps, np.ones(4), tol_x=0.0, tol_p=1.0, lib=lib,
                     variant=oracle.VAR_NORMALIZED)
    check("normalized_zero_tol", t.axis[0] == 0)
    # energy-conserving replacement: hand-worked set (|d|^2 = 23/45 along y)
    EC = oracle.VAR_CONSERVE_ENERGY
    z3 = np.zeros(3, np.int32)
    mom = np.array([[0.75, 2.4, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    r = oracle.merge(z3, np.array([[0.2, 0.5, 0.8]]), mom, np.ones(3), 1, tol_x=1.0,
                     tol_p=1.0, lib=lib, variant=EC)
    d = math.sqrt(23.0 / 45.0)
    check("ec_hand", r.count == 2 and np.allclose(r.mom[1], [d, -d], rtol=1e-13))

    def total_energy(w_, m_):
        return float(np.sum(w_ * np.sqrt(1.0 + np.sum(m_ ** 2, axis=0))))

    p = synth.two_stream(cells=4)
    r = oracle.merge_particles(p, lib=lib, variant=EC)
    e_in, e_out = total_energy(p.w, p.mom), total_energy(r.w, r.mom)
    check("ec_energy", abs(e_out - e_in) <= 1e-12 * e_in and r.count > 0)
    rng = np.random.default_rng(3)
    m1 = rng.normal(0.5, 0.2, size=(1, 9))
    w1 = rng.uniform(0.5, 1.5, 9)
    r = oracle.merge(np.zeros(9, np.int32), rng.random((1, 9)), m1, w1, 1, tol_x=1.0,
                     tol_p=1e9, lib=lib, variant=EC)
    check("ec_one_axis", r.count == 2 and
          abs(total_energy(r.w, r.mom) - total_energy(w1, m1)) <= 1e-12 * total_energy(w1, m1))
    mom = np.array([[1.0, 2.0, 1.5, 1.5], [0.2, 0.2, 0.2, 0.2], [0.05, 0.05, 0.2, -0.1]])
    r = oracle.merge(np.zeros(4, np.int32), np.full((1, 4), 0.5), mom, np.ones(4), 1,
                     tol_x=1.0, tol_p=1e9, lib=lib, variant=EC)
    dd = r.mom[:, 0] - mom.mean(axis=1) if r.count == 2 else np.zeros(3)
    check("ec_direction", r.count == 2 and abs(dd[2]) > 0.99 * np.linalg.norm(dd))
    return fails


def test_real_oracle_passes_compact_pins():
    assert pin_failures(None) == []


MUTANTS = {
    "drop_abs_of_mean": ("fabs(M->Q[l])", "M->Q[l]"),
    "bessel_variance": ("sqrt(v / W)", "sqrt(v / (W - 1.0))"),
    "unweighted_mean": ("s += P->w[idx[i]] * q[idx[i]];", "s += q[idx[i]];"),
    "stop_strict": ("if (!(M->delta[l] <= T))", "if (!(M->delta[l] < T))"),
    "argmin": ("if (score[l] > score[k])", "if (score[l] < score[k])"),
    "cut_strict": ("q[sub[i]] <= Qk", "q[sub[i]] < Qk"),
    "v2_first": ("        S->stack[sp++] = (orc_range){r.begin + n1, r.end, r.depth + 1};\n"
                 "        S->stack[sp++] = (orc_range){r.begin, r.begin + n1, r.depth + 1};",
                 "        S->stack[sp++] = (orc_range){r.begin, r.begin + n1, r.depth + 1};\n"
                 "        S->stack[sp++] = (orc_range){r.begin + n1, r.end, r.depth + 1};"),
    "leaf_weight_count": ("L->W = M.W;", "L->W = (double)ms;"),
    "pnorm_sum_abs": ("s2 += M->Q[l] * M->Q[l];", "s2 += fabs(M->Q[l]);"),
    "pnorm_ignored": ("double scale = (P->variant & ORC_VAR_PNORM) ? pnorm : fabs(M->Q[l]);",
                      "double scale = fabs(M->Q[l]);"),
    "normalized_ignores_T": ("return d / T;", "return d;"),
    "normalized_zero_tol": ("return d > 0.0 ? INFINITY : 0.0;", "return 0.0;"),
    "ec_no_orthogonalization": ("dir[l] = (l == k ? 1.0 : 0.0) - ph[k] * ph[l];",
                                "dir[l] = (l == k ? 1.0 : 0.0);"),
    "ec_kinetic_mean": ("E += P->w[ids[i]] * sqrt(1.0 + p2);",
                        "E += P->w[ids[i]] * (sqrt(1.0 + p2) - 1.0);"),
    "ec_raw_variance": ("double score = (v / W) * (1.0 - ph[l] * ph[l]);",
                        "double score = (v / W);"),
    "ec_one_axis_sign": ("(g * g - 1.0 - P2) / (g * g - P2)", "(g * g - 1.0 - P2) / (g * g + P2)"),
}


def _run_mutant(so_path, queue):
    try:
        queue.put(pin_failures(oracle.load_library(so_path)))
    except Exception as exc:  # a mutant that errors out is caught too
        queue.put(["error: %r" % (exc,)])


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pma_oracle.c")).read()
    assert src.count(old) >= 1, "mutation anchor missing"
    path = tmp_path / ("mut_%s.c" % name)
    path.write_text(src.replace(old, new))
    so = oracle.compile_source(str(path), str(tmp_path / "mut.so"))
    # run in a separate process: a planted mistake may also crash the C code
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    proc = ctx.Process(target=_run_mutant, args=(so, q))
    proc.start()
    proc.join(120)
    if proc.is_alive():
        proc.kill()
        proc.join()
    fails = q.get() if not q.empty() else ["crashed or hung (exit %s)" % proc.exitcode]
    assert fails, "planted mistake %s not caught" % name
