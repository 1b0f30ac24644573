"""Pins of the oracle's symmetric plmDCA (Sec. 3, Eq. npll_1 with the l2
penalty of Eq. l2reg): one minimisation of l_pseudo + R_l2 over fields and
one coupling block per pair, shared by both sites.

None of these re-runs the oracle's formula: a closed form at the origin,
brute-force enumeration of the joint Potts model (Eq. potts_model), central
differences, an independent optimiser (scipy) and the gauge identities the
paper states for the regularised optimum (Eq. symmetricgauge).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

Q = 21


def _pairs(N):
    return [(i, j) for i in range(N) for j in range(i + 1, N)]


def _x(h, blocks, N):
    """pack (h[N,q], {(i,j): J_ij}) the way the problem is parameterised"""
    return np.concatenate([h.ravel()] + [blocks[p].ravel() for p in _pairs(N)])


def _random_x(N, rng, sd=0.3):
    h = rng.normal(0, sd, (N, Q))
    blocks = {p: rng.normal(0, sd, (Q, Q)) for p in _pairs(N)}
    return h, blocks, _x(h, blocks, N)


def test_symmetric_parameter_count():
    # Sec. 6: the symmetric problem has N q (1 + (N - 1) q / 2) parameters
    for N in (3, 10, 120):
        assert oracle.sym_nparams(N) == N * Q * (1 + (N - 1) * Q / 2)


def test_symmetric_objective_and_gradient_at_zero():
    # at theta = 0 every conditional is uniform: l_pseudo = N ln q, and each
    # g_r contributes its closed-form gradient; a shared block collects the
    # gradients of both of its sites, the second transposed:
    #   dl/dh_i(k)    = -(f_i(k) - 1/q)
    #   dl/dJ_ij(k,l) = -(f_ij(k,l) - f_i(k)/q) - (f_ij(k,l) - f_j(l)/q)
    S = synth.add_clusters(synth.small_random(5, 90, 2, gap_p=0.1), 0.4, 2, max_redraw=0.1)
    m, w, _, beff = oracle.reweight(S, 0.8)
    B, N = S.shape
    n = oracle.sym_nparams(N)
    f, g = oracle.sym_objgrad(S, w, beff, np.zeros(n), 0.01, 0.01)
    assert f == pytest.approx(N * math.log(Q), rel=1e-13)
    X = np.zeros((B, N, Q))
    X[np.arange(B)[:, None], np.arange(N)[None, :], S] = 1.0
    fi = np.einsum("b,bik->ik", w, X) / beff
    gh = -(fi - 1.0 / Q)
    assert np.allclose(g[: N * Q].reshape(N, Q), gh, rtol=1e-12, atol=1e-15)
    off = N * Q
    for (i, j) in _pairs(N):
        fij = np.einsum("b,bk,bl->kl", w, X[:, i], X[:, j]) / beff
        exp = -(fij - fi[i][:, None] / Q) - (fij - fi[j][None, :] / Q)
        assert np.allclose(g[off:off + Q * Q].reshape(Q, Q), exp, rtol=1e-12, atol=1e-15)
        off += Q * Q


@pytest.mark.parametrize("N", [3, 4])
def test_symmetric_objective_matches_brute_force_joint(N):
    # one sequence, unit weight: l_pseudo = -sum_r log P(sigma_r | sigma_\\r)
    # with the conditionals read off the enumerated joint Potts model, plus
    # R_l2 = lambda_h sum ||h_i||^2 + lambda_J sum_{i<j} ||J_ij||^2 (each
    # block once, lambda_J not halved)
    rng = np.random.default_rng(10 + N)
    h, blocks, x = _random_x(N, rng, 0.5)
    grids = np.indices((Q,) * N).reshape(N, -1)
    E = np.zeros(grids.shape[1])
    for i in range(N):
        E += h[i, grids[i]]
    for (i, j) in _pairs(N):
        E += blocks[(i, j)][grids[i], grids[j]]
    joint = np.exp(E - E.max()).reshape((Q,) * N)
    lh, lJ = 0.03, 0.07
    pen = lh * (h ** 2).sum() + lJ * sum((b ** 2).sum() for b in blocks.values())
    for t in range(5):
        seq = rng.integers(0, Q, N).astype(np.int8)
        lp = 0.0
        for r in range(N):
            idx = list(seq)
            idx[r] = slice(None)
            cond = joint[tuple(idx)]
            lp -= math.log(cond[seq[r]] / cond.sum())
        f = oracle.sym_objgrad(seq[None, :], np.ones(1), 1.0, x, lh, lJ, grad=False)
        assert f == pytest.approx(lp + pen, rel=1e-12)


def test_symmetric_gradient_central_differences():
    rng = np.random.default_rng(5)
    S = synth.small_random(6, 70, 4, gap_p=0.1)
    m, w, _, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    _, _, x = _random_x(N, rng, 0.2)
    f, g = oracle.sym_objgrad(S, w, beff, x, 0.02, 0.05)
    eps = 1e-5
    for c in rng.choice(x.size, 48, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[c] += eps
        xm[c] -= eps
        fd = (oracle.sym_objgrad(S, w, beff, xp, 0.02, 0.05, grad=False) -
              oracle.sym_objgrad(S, w, beff, xm, 0.02, 0.05, grad=False)) / (2 * eps)
        assert fd == pytest.approx(g[c], rel=1e-6, abs=1e-9)


def test_symmetric_expansion_is_the_transposed_mirror():
    rng = np.random.default_rng(7)
    N = 4
    h, blocks, x = _random_x(N, rng)
    hh, J = oracle.sym_expand(x, N)
    assert np.array_equal(hh, h)
    for (i, j), b in blocks.items():
        assert np.array_equal(J[i, :, j, :], b)
        assert np.array_equal(J[j, :, i, :], b.T)
    for i in range(N):
        assert not J[i, :, i, :].any()


def test_symmetric_minimiser_matches_scipy_within_strong_convexity_bound():
    # l_pseudo is convex and R_l2 adds 2 min(lambda_h, lambda_J) to the
    # Hessian, so ||x - x*|| <= ||grad(x)|| / mu for any x
    scipy_opt = pytest.importorskip("scipy.optimize")
    S = synth.add_clusters(synth.small_random(4, 60, 21, gap_p=0.1), 0.4, 21, max_redraw=0.1)
    m, w, _, beff = oracle.reweight(S, 0.8)
    lh, lJ = 0.01, 0.01
    mu = 2 * min(lh, lJ)
    h, J, info = oracle.solve_symmetric(S, w, beff, lh, lJ, gtol=1e-8)
    assert info["status"] == 0 and info["gnorm"] <= 1e-8

    def fg(x):
        return oracle.sym_objgrad(S, w, beff, x, lh, lJ)

    res = scipy_opt.minimize(fg, np.zeros(info["x"].size), jac=True, method="L-BFGS-B",
                             options=dict(maxiter=50000, gtol=1e-12, ftol=1e-16, maxcor=20))
    bound = (np.linalg.norm(fg(res.x)[1]) + np.linalg.norm(fg(info["x"])[1])) / mu
    assert np.linalg.norm(res.x - info["x"]) <= bound + 1e-12
    assert bound < 1e-4


def test_symmetric_gauge_identities_at_the_minimiser():
    # Eq. symmetricgauge: at the regularised optimum
    #   lambda_J sum_s J_ij(k,s) = lambda_h h_i(k),
    #   lambda_J sum_s J_ij(s,l) = lambda_h h_j(l),   sum_s h_i(s) = 0,
    # each exact up to the residual gradient along the gauge direction that
    # produces it: |violation| <= sqrt(q + 1) ||grad|| / 2 (|sum h| with
    # sqrt(q) ||grad|| / (2 lambda_h))
    S = synth.add_clusters(synth.small_random(5, 90, 22, gap_p=0.1), 0.4, 22, max_redraw=0.1)
    m, w, _, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    lh, lJ = 0.01, 0.03
    h, J, info = oracle.solve_symmetric(S, w, beff, lh, lJ, gtol=1e-9)
    gn = info["gnorm"]
    tol = math.sqrt(Q + 1) * gn / 2 + 1e-14
    for i in range(N):
        assert abs(h[i].sum()) <= math.sqrt(Q) * gn / (2 * lh) + 1e-12
    for (i, j) in _pairs(N):
        assert np.all(np.abs(lJ * J[i, :, j, :].sum(1) - lh * h[i]) <= tol)
        assert np.all(np.abs(lJ * J[i, :, j, :].sum(0) - lh * h[j]) <= tol)
