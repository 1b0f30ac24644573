"""Pins of the oracle's score alternatives (Sec. 6): the general l_p norm
(i), Burkoff's D_ij (ii, Eqs. burkoffscore1-2), gap exclusion (iii), the
average sum correction (iv, Eq. corr_normsum), and the reweighted site
frequencies Burkoff's score needs.

The pins are closed forms on planted blocks (a rank-one block u v^T with
zero-sum u, v is already in the Ising gauge, so its norms factor), a
symbolic evaluation of Burkoff's score for two states, its information
inequalities, and exact rational arithmetic for the correction.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

Q = 21


def _planted(N, pairs, q=Q, seed=0):
    """asymmetric estimates whose combined gauged block for pair (i, j) is
    u v^T (both sites carry it, site j's transposed); other blocks zero"""
    rng = np.random.default_rng(seed)
    J = np.zeros((N, q, N, q))
    uv = {}
    for (i, j) in pairs:
        u = rng.normal(0, 1, q)
        v = rng.normal(0, 1, q)
        u -= u.mean()
        v -= v.mean()
        J[i, :, j, :] = np.outer(u, v)
        J[j, :, i, :] = np.outer(u, v).T
        uv[(i, j)] = (u, v)
    return J, uv


@pytest.mark.parametrize("p", [1.0, 2.0, 3.0, 0.5])
def test_lp_norm_of_a_rank_one_gauged_block(p):
    J, uv = _planted(5, [(0, 2), (1, 4)])
    sc = oracle.score_matrix(J, "lp", p)
    for (i, j), (u, v) in uv.items():
        lp = lambda a: (np.abs(a) ** p).sum() ** (1 / p)  # noqa: E731
        assert sc[i, j] == pytest.approx(lp(u) * lp(v), rel=1e-12)
        assert sc[j, i] == sc[i, j]
    assert sc[0, 1] == 0.0 and sc[2, 3] == 0.0


def test_gap_excluded_norm_of_a_rank_one_gauged_block():
    J, uv = _planted(4, [(0, 3)], seed=1)
    (u, v), = uv.values()
    assert oracle.score_matrix(J, "fro", exclude_gap=True)[0, 3] == pytest.approx(
        np.linalg.norm(u[1:]) * np.linalg.norm(v[1:]), rel=1e-12)
    assert oracle.score_matrix(J, "lp", 1.0, exclude_gap=True)[0, 3] == pytest.approx(
        np.abs(u[1:]).sum() * np.abs(v[1:]).sum(), rel=1e-12)
    # the full norm keeps the gap row and column
    assert oracle.score_matrix(J, "fro")[0, 3] == pytest.approx(
        np.linalg.norm(u) * np.linalg.norm(v), rel=1e-12)


def test_norms_are_gauge_invariant():
    # adding a(k) + b(l) + c to an estimate changes no norm (gauge first)
    rng = np.random.default_rng(3)
    N = 4
    J = rng.normal(0, 0.3, (N, Q, N, Q))
    for r in range(N):
        J[r, :, r, :] = 0
    J2 = J.copy()
    J2[1, :, 3, :] += rng.normal(0, 1, Q)[:, None] + rng.normal(0, 1, Q)[None, :] + 0.7
    for kind, p in (("fro", 2), ("lp", 1.5)):
        assert np.allclose(oracle.score_matrix(J, kind, p), oracle.score_matrix(J2, kind, p),
                           rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("a_num", [3, 10000])
def test_burkoff_two_states_symbolic(a_num):
    # q = 2: D_ij evaluated symbolically (sympy) from Eqs. burkoffscore1-2 with
    # the block in the Ising gauge, v = a [[1, -1], [-1, 1]]; a = 1000 puts
    # e^v far beyond the double range, where only a shifted exponent is finite
    sp = pytest.importorskip("sympy")
    a, x, y = sp.Rational(a_num, 10), sp.Rational(1, 5), sp.Rational(7, 10)
    V = sp.Matrix([[a, -a], [-a, a]])
    fi = [x, 1 - x]
    fj = [y, 1 - y]
    w = [[fi[k] * fj[l] * sp.exp(V[k, l]) for l in range(2)] for k in range(2)]
    Z = sum(sum(r) for r in w)
    D = sum(w[k][l] / Z * sp.log(w[k][l] / Z / (fi[k] * fj[l])) for k in range(2) for l in range(2))
    N, q = 2, 2
    J = np.zeros((N, q, N, q))
    J[0, :, 1, :] = np.array(V.tolist(), dtype=float)
    J[1, :, 0, :] = J[0, :, 1, :].T
    freq = np.array([[float(x), float(1 - x)], [float(y), float(1 - y)]])
    got = oracle.score_matrix(J, "burkoff", freq=freq)[0, 1]
    assert got == pytest.approx(float(sp.N(D, 30)), rel=1e-13)


def test_burkoff_information_inequalities():
    # D_ij is the Kullback-Leibler divergence of P^D from f_i f_j: >= 0, and
    # 0 exactly when the coupling block is zero; unseen states contribute 0
    rng = np.random.default_rng(4)
    N = 5
    J = rng.normal(0, 0.4, (N, Q, N, Q))
    for r in range(N):
        J[r, :, r, :] = 0
    f = rng.dirichlet(np.ones(Q), N)
    f[2, 5] = 0.0
    f[2] /= f[2].sum()
    D = oracle.score_matrix(J, "burkoff", freq=f)
    assert np.all(D[np.triu_indices(N, 1)] > 0)
    assert np.all(np.isfinite(D))
    assert np.all(np.abs(oracle.score_matrix(np.zeros_like(J), "burkoff", freq=f)) <= 1e-14)


def test_average_sum_correction_exact_rationals():
    fn = [[0, 3, 1, 4], [3, 0, 5, 9], [1, 5, 0, 2], [4, 9, 2, 0]]
    N = 4
    F = [[Fraction(v) for v in r] for r in fn]
    row = [sum(F[i][j] for j in range(N) if j != i) / (N - 1) for i in range(N)]
    col = [sum(F[i][j] for i in range(N) if i != j) / (N - 1) for j in range(N)]
    tot = sum(F[i][j] for i in range(N) for j in range(N) if i != j) / (N * (N - 1))
    got = oracle.asc(np.array(fn, float))
    for i in range(N):
        for j in range(N):
            exp = 0 if i == j else F[i][j] - col[j] - row[i] + tot
            assert got[i, j] == pytest.approx(float(exp), abs=1e-14)


def test_site_frequencies_brute_force():
    S = synth.add_clusters(synth.small_random(7, 60, 5, gap_p=0.2), 0.4, 5, max_redraw=0.1)
    m, w, _, beff = oracle.reweight(S, 0.8)
    f = oracle.site_freqs(S, w, beff)
    for i in range(S.shape[1]):
        for k in range(Q):
            assert f[i, k] == pytest.approx(sum(w[b] for b in range(S.shape[0]) if S[b, i] == k) / beff,
                                            abs=1e-15)
    assert np.allclose(f.sum(1), 1.0, rtol=1e-13)
