"""Pins for the oracle's wavefunction cut (Methods section: after a factor, if
more than N_MAX determinants remain, keep the N_CUT of largest |c|) and for
its adjoint gradient under that cut.

The reference here is the dense state vector (oracle/dense.py: Taylor-series
matrix exponentials, no 2x2 closed form) carried factor by factor with the
truncation rules written out on the full vector:

* the stored set grows by the determinants the factor links to a stored one
  (tau and tau^+ applied to the indicator of the set, read off structurally);
* with eps > 0, stored determinants with |c| < eps are dropped;
* then, if more than N_MAX are stored, they are ranked by |c| descending with
  ties to the smaller determinant key, and all but the first N_CUT dropped.

Each case also checks that the test can tell the rule from its plausible
mistakes (the cut taken before the eps rule, N_MAX kept instead of N_CUT, ties
broken towards the larger key): each mistaken variant of the dense reference
must disagree with the oracle somewhere.
"""
import numpy as np
import pytest

from paper_2301_05726_gb300 import synth
from oracle import Oracle
from oracle.dense import Dense


def dense_truncated(d, prob, theta, eps, n_max, n_cut, variant="paper"):
    """Dense propagation with the eps rule and the cut after every factor.

    Returns (v, stored mask, per-factor stored-set digests, total cut, smallest
    |c| gap at any cut threshold between a kept and a dropped determinant
    whose magnitudes differ, number of cuts whose threshold fell inside a run
    of exactly equal magnitudes)."""
    v = d.reference()
    stored = np.zeros(d.dim, bool)
    stored[prob.hf_key] = True
    digests, cut_total, min_gap, tie_cuts = [], 0, np.inf, 0
    idx = np.arange(d.dim)

    def cut(v, stored):
        nonlocal cut_total, min_gap, tie_cuts
        keep_n = n_max if variant == "keep_n_max" else n_cut
        if n_max <= 0 or stored.sum() <= n_max:
            return v, stored
        s_idx = idx[stored]
        mag = np.abs(v[s_idx])
        tie_key = -s_idx if variant == "ties_to_larger" else s_idx
        order = np.lexsort((tie_key, -mag))  # |c| descending, then the tie key ascending
        kept, dropped = s_idx[order[:keep_n]], s_idx[order[keep_n:]]
        if len(dropped):
            a, b = np.abs(v[kept[-1]]), np.abs(v[dropped[0]])
            if a == b:
                tie_cuts += 1
            else:
                min_gap = min(min_gap, a - b)
        stored = stored.copy()
        stored[dropped] = False
        v = np.where(stored, v, 0.0)
        cut_total += len(dropped)
        return v, stored

    def eps_rule(v, stored):
        if eps <= 0:
            return v, stored
        stored = stored & ~(np.abs(v) < eps)
        return np.where(stored, v, 0.0), stored

    for k in range(len(theta)):
        row = prob.exc[k]
        ind = stored.astype(np.float64)
        linked = (d.tau(row, ind) != 0) | (d.tau_dagger(row, ind) != 0)
        v = d.expm_factor(row, theta[k], v)
        stored = stored | linked
        v = np.where(stored, v, 0.0)
        if variant == "cut_before_eps":
            v, stored = cut(v, stored)
            v, stored = eps_rule(v, stored)
        else:
            v, stored = eps_rule(v, stored)
            v, stored = cut(v, stored)
        digests.append(hash(np.packbits(stored).tobytes()))
    return v, stored, digests, cut_total, min_gap, tie_cuts


def assert_matches(prob, o_keys, o_amps, o_cnt, ref):
    v, stored, _, cut_total, _, _ = ref
    d_keys = np.flatnonzero(stored).astype(np.uint64)
    assert np.array_equal(o_keys, d_keys)
    assert np.max(np.abs(o_amps - v[d_keys.astype(np.int64)])) < 1e-13
    assert o_cnt["cut"] == cut_total


def disagrees(o_keys, o_amps, o_cnt, ref):
    v, stored, _, cut_total, _, _ = ref
    d_keys = np.flatnonzero(stored).astype(np.uint64)
    if not np.array_equal(o_keys, d_keys) or o_cnt["cut"] != cut_total:
        return True
    return np.max(np.abs(o_amps - v[d_keys.astype(np.int64)])) > 1e-10


@pytest.fixture(scope="module")
def cfg1():
    return synth.config_problem(1)


@pytest.fixture(scope="module")
def fourteen():
    # 14 spin-orbitals, 6 electrons, 204 factors, with pruning.
    return synth.make_problem(21, 7, 3, 3, 0.1)


@pytest.mark.parametrize("n_max,n_cut", [(60, 40), (150, 90)])
def test_cut_vs_dense_eps0(cfg1, n_max, n_cut):
    o, d = Oracle(cfg1), Dense(cfg1)
    keys, amps, cnt = o.apply(eps=0.0, n_max=n_max, n_cut=n_cut)
    ref = dense_truncated(d, cfg1, cfg1.theta, 0.0, n_max, n_cut)
    assert ref[3] > 0 and ref[4] > 1e-9  # cuts happened, no near-ties at their thresholds
    assert_matches(cfg1, keys, amps, cnt, ref)
    for variant in ("keep_n_max",):
        assert disagrees(keys, amps, cnt, dense_truncated(d, cfg1, cfg1.theta, 0.0, n_max, n_cut, variant))


def test_cut_vs_dense_with_eps(fourteen):
    # eps and the cut together: the eps rule comes first.  With these values
    # the order matters (the cut-first variant disagrees).
    eps, n_max, n_cut = 1e-4, 200, 120
    o, d = Oracle(fourteen), Dense(fourteen)
    keys, amps, cnt = o.apply(eps=eps, n_max=n_max, n_cut=n_cut)
    ref = dense_truncated(d, fourteen, fourteen.theta, eps, n_max, n_cut)
    assert ref[3] > 0 and ref[4] > 1e-9
    assert cnt["dropped_new"] > 0 and cnt["dropped_old"] > 0
    assert_matches(fourteen, keys, amps, cnt, ref)
    for variant in ("cut_before_eps", "keep_n_max"):
        assert disagrees(keys, amps, cnt, dense_truncated(d, fourteen, fourteen.theta, eps, n_max, n_cut, variant))


def test_cut_tie_rule_vs_dense(cfg1):
    # Angles of exactly zero create partners with amplitude exactly 0 (eps = 0
    # keeps them), so the cut threshold can fall inside a run of equal |c|;
    # then the smaller keys are kept.
    theta = cfg1.theta.copy()
    theta[::2] = 0.0
    o, d = Oracle(cfg1), Dense(cfg1)
    n_max, n_cut = 70, 55
    keys, amps, cnt = o.apply(theta, eps=0.0, n_max=n_max, n_cut=n_cut)
    ref = dense_truncated(d, cfg1, theta, 0.0, n_max, n_cut)
    assert ref[5] > 0  # some cut decided among exact ties
    assert_matches(cfg1, keys, amps, cnt, ref)
    assert disagrees(keys, amps, cnt, dense_truncated(d, cfg1, theta, 0.0, n_max, n_cut, "ties_to_larger"))


def test_cut_gradient_vs_dense_central_differences(cfg1):
    # With the cut, the adjoint gives the derivative of the truncated map with
    # every kept set held fixed.  Central differences of the dense truncated
    # energy agree wherever a +-h change of theta_k keeps every per-factor
    # kept set (compared factor by factor).
    n_max, n_cut = 60, 40
    o, d = Oracle(cfg1), Dense(cfg1)
    E, g = o.gradient(eps=0.0, n_max=n_max, n_cut=n_cut)
    th = cfg1.theta
    ref = dense_truncated(d, cfg1, th, 0.0, n_max, n_cut)
    assert E == pytest.approx(d.energy(ref[0]), abs=1e-11)
    h = 1e-6
    checked = 0
    for k in range(0, cfg1.n_exc, 3):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        rp = dense_truncated(d, cfg1, tp, 0.0, n_max, n_cut)
        rm = dense_truncated(d, cfg1, tm, 0.0, n_max, n_cut)
        if rp[2] != ref[2] or rm[2] != ref[2]:
            continue
        fd = (d.energy(rp[0]) - d.energy(rm[0])) / (2 * h)
        assert abs(g[k] - fd) < max(1e-8, 5e-9 * abs(E)), (k, g[k], fd)
        checked += 1
    assert checked >= 20
    # The cut gradient is not the uncut one (the test sees the truncation).
    _, g_full = o.gradient(eps=0.0, n_max=0, n_cut=0)
    assert np.max(np.abs(g - g_full)) > 1e-4


def test_cut_gradient_with_eps_vs_dense(fourteen):
    eps, n_max, n_cut = 1e-4, 200, 120
    prob = fourteen.prefix(90)
    o, d = Oracle(prob), Dense(prob)
    E, g = o.gradient(eps=eps, n_max=n_max, n_cut=n_cut)
    th = prob.theta
    ref = dense_truncated(d, prob, th, eps, n_max, n_cut)
    assert ref[3] > 0
    assert E == pytest.approx(d.energy(ref[0]), abs=1e-11)
    h = 1e-6
    checked = 0
    for k in range(0, prob.n_exc, 9):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        rp = dense_truncated(d, prob, tp, eps, n_max, n_cut)
        rm = dense_truncated(d, prob, tm, eps, n_max, n_cut)
        if rp[2] != ref[2] or rm[2] != ref[2]:
            continue
        fd = (d.energy(rp[0]) - d.energy(rm[0])) / (2 * h)
        assert abs(g[k] - fd) < max(1e-8, 5e-9 * abs(E)), (k, g[k], fd)
        checked += 1
    assert checked >= 6
