"""Oracle pins above 64 spin-orbitals (test infrastructure; no GPU).

The paper stops at 64 spin-orbitals only because of its key width and says
the limit could be removed (Conclusions; its CH2O/cc-pVDZ frozen-core case
has 72).  The oracle's 128-bit build is the same source as the 64-bit one
with a wider key type, and is pinned to it two ways:

* the same problems through both builds give the same determinants,
  amplitudes (bit for bit) and counts, and the same energies and gradients;
* a problem embedded in a larger orbital space -- its virtual orbitals moved
  above spin-orbital 64, the orbitals in between given zero integrals and no
  excitations -- is the same physical problem: every occupation-number count
  below an occupied or touched orbital is unchanged, so the Jordan-Wigner
  signs, amplitudes, energy and gradient are those of the original, with each
  determinant key relabelled.  This exercises the keys' high word.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2301_05726_gb300 import synth

E_TOL = 1e-12
G_TOL = 1e-11


def embed(prob, first_virtual_so=64):
    """prob with its virtual spatial orbitals moved so that the first one
    starts at spin-orbital `first_virtual_so`; returns (embedded, spatial map)."""
    n = prob.n_spatial
    n_occ = max(prob.n_alpha, prob.n_beta)
    gap = first_virtual_so // 2 - n_occ
    assert gap > 0
    m = np.array([i if i < n_occ else i + gap for i in range(n)])
    n2 = n + gap
    h = np.zeros((n2, n2))
    h[np.ix_(m, m)] = prob.h
    g = np.zeros((n2,) * 4)
    g[np.ix_(m, m, m, m)] = prob.g
    so = 2 * m[np.arange(2 * n) // 2] + (np.arange(2 * n) % 2)  # spin-orbital map
    exc = prob.exc.copy()
    exc[exc >= 0] = so[exc[exc >= 0]]
    emb = dataclasses.replace(prob, n_spatial=n2, h=h, g=g, exc=np.ascontiguousarray(exc, dtype=np.int32),
                              name=prob.name + f"_embedded{2 * n2}so")
    return emb, so


def relabel(key, so):
    out = 0
    p = 0
    while key:
        if key & 1:
            out |= 1 << int(so[p])
        key >>= 1
        p += 1
    return out


def small_pruned():
    prob = synth.config_problem(2).prefix(150)
    return dataclasses.replace(prob, eps=1e-7, n_max=1500, n_cut=1000)


@pytest.mark.parametrize("case", ["cfg1", "pruned_cut"])
def test_128_bit_build_matches_64_bit(case):
    prob = synth.config_problem(1) if case == "cfg1" else small_pruned()
    a, b = oracle.Oracle(prob), oracle.Oracle(prob, key_bits=128)
    ka, aa, ca = a.apply()
    kb, ab, cb = b.apply()
    assert oracle.key_ints(ka) == oracle.key_ints(kb)
    assert np.array_equal(aa, ab) and ca == cb
    if case == "pruned_cut":
        assert ca["cut"] > 0 and ca["dropped_new"] > 0  # both rules were exercised
    Ea, Eb = a.energy(ka, aa)[0], b.energy(kb, ab)[0]
    assert abs(Ea - Eb) <= E_TOL
    _, sa = a.sigma(ka, aa)
    _, sb = b.sigma(kb, ab)
    assert np.max(np.abs(sa - sb)) <= E_TOL
    Ga, ga = a.gradient()
    Gb, gb = b.gradient()
    assert abs(Ga - Gb) <= E_TOL and np.max(np.abs(ga - gb)) <= G_TOL


@pytest.mark.parametrize("case", ["cfg1", "pruned_cut"])
def test_embedding_past_64_spin_orbitals(case):
    prob = synth.config_problem(1) if case == "cfg1" else small_pruned()
    emb, so = embed(prob)
    assert emb.n_so > 64
    base, wide = oracle.Oracle(prob), oracle.Oracle(emb)
    assert wide.key_bits == 128
    kb, ab, cb = base.apply()
    kw, aw, cw = wide.apply()
    assert cb == cw
    wide_keys = oracle.key_ints(kw)
    assert any(k >> 64 for k in wide_keys)  # determinants with bits in the high word
    mapped = {relabel(k, so): a for k, a in zip(oracle.key_ints(kb), ab)}
    assert set(mapped) == set(wide_keys)
    assert all(mapped[k] == a for k, a in zip(wide_keys, aw))  # bit for bit
    Eb, Ew = base.energy(kb, ab)[0], wide.energy(kw, aw)[0]
    assert abs(Eb - Ew) <= E_TOL
    Gb, gb = base.gradient()
    Gw, gw = wide.gradient()
    assert abs(Gb - Gw) <= E_TOL and np.max(np.abs(gb - gw)) <= G_TOL


def test_wide_operators_and_matrix_elements():
    prob = synth.config_problem(1)
    emb, so = embed(prob)
    base, wide = oracle.Oracle(prob), oracle.Oracle(emb)
    hf, hf_w = prob.hf_key, emb.hf_key
    assert relabel(hf, so) == hf_w
    for k in range(prob.n_exc):
        s, d = base.tau(k, hf)
        sw, dw = wide.tau(k, hf_w)
        assert s == sw and (d is None) == (dw is None)
        if d is not None:
            assert relabel(d, so) == dw and dw >> 64  # the excitation reaches the high word
            assert wide.hmat(hf_w, dw) == base.hmat(hf, d)
    assert wide.hmat(hf_w, hf_w) == base.hmat(hf, hf)


def test_key_width_is_checked():
    emb, _ = embed(synth.config_problem(1))
    with pytest.raises(ValueError):
        oracle.Oracle(emb, key_bits=64)
