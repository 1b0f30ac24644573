"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them re-runs the oracle's
own formula: they use closed forms, brute-force enumeration of the joint
Potts model, finite differences, an independent optimiser (scipy), a
least-squares projection, exact rational arithmetic and invariances, chosen
so that a dropped term, a wrong sign or index, or a transposed block fails
at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

Q = 21
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _onehot(S, q=Q):
    B, N = S.shape
    X = np.zeros((B, N, q))
    X[np.arange(B)[:, None], np.arange(N)[None, :], S] = 1.0
    return X


def _clustered(N, B, seed):
    S = synth.small_random(N, B, seed, gap_p=0.1)
    return synth.add_clusters(S, 0.4, seed, max_redraw=0.1)


# ---------------------------------------------------------------------------
# Reweighting (Eq. inverse_weights2)
# ---------------------------------------------------------------------------
def _load_reweight_golden():
    seqs, cases = [], []
    with open(os.path.join(GOLDEN, "reweight_hand.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "seq":
                seqs.append([int(t) for t in tok[2:]])
            elif tok[0] == "case":
                x = float(tok[1])
                bi = tok.index("beff")
                m = [int(t) for t in tok[3:bi]]
                cases.append((x, m, Fraction(tok[bi + 1])))
    return np.array(seqs, np.int8), cases


def test_reweight_hand_worked_golden():
    S, cases = _load_reweight_golden()
    for x, m_exp, beff_exp in cases:
        m, w, w32, beff = oracle.reweight(S, x)
        assert m.tolist() == m_exp
        assert np.array_equal(w, 1.0 / np.array(m_exp, np.float64))
        assert beff == pytest.approx(float(beff_exp), rel=1e-15)


def test_reweight_threshold_is_ceil_xN():
    # Eq. inverse_weights: similarity >= x; the smallest integer count
    for N in [1, 5, 7, 10, 20, 120, 333, 500]:
        for x in [0.0, 0.1, 0.5, 0.7, 0.8, 0.9, 1.0]:
            T = oracle.identity_threshold(x, N)
            exact = Fraction(x).limit_denominator(1000) * N
            assert T == math.ceil(exact), (N, x, T)


def test_reweight_brute_force_small():
    # plain definition on tiny random MSAs, counted by broadcasting
    for seed, (B, N) in enumerate([(1, 3), (7, 5), (40, 12), (64, 33)]):
        S = _clustered(N, B, seed)
        for x in [0.0, 0.5, 0.8, 1.0]:
            T = math.ceil(Fraction(x) * N)
            matches = (S[:, None, :] == S[None, :, :]).sum(-1)
            m_exp = (matches >= T).sum(0)
            m, w, w32, beff = oracle.reweight(S, x)
            assert np.array_equal(m, m_exp)
            assert np.array_equal(w32, (np.float32(1) / m_exp.astype(np.float32)))
            assert beff == pytest.approx(sum(Fraction(1, int(k)) for k in m_exp), rel=1e-15)


def test_reweight_special_cases():
    N = 10
    # all pairwise far apart -> every weight is 1, B_eff = B
    S = np.array([[k] * N for k in range(8)], np.int8)
    m, w, _, beff = oracle.reweight(S, 0.8)
    assert np.all(m == 1) and beff == 8.0
    # k exact copies -> each weight 1/k
    S = np.repeat(np.arange(5, dtype=np.int8)[:, None], N, 1)
    S = np.repeat(S, [1, 2, 3, 4, 5], axis=0)
    m, w, _, beff = oracle.reweight(S, 0.8)
    assert m.tolist() == sum([[k] * k for k in [1, 2, 3, 4, 5]], [])
    assert beff == pytest.approx(5.0, rel=1e-15)
    # x = 0 -> everything is similar to everything
    S = synth.small_random(N, 17, 3)
    m, _, _, beff = oracle.reweight(S, 0.0)
    assert np.all(m == 17) and beff == pytest.approx(1.0, rel=1e-15)
    # x = 1 -> only identical sequences
    m, _, _, _ = oracle.reweight(S, 1.0)
    ident = (S[:, None, :] == S[None, :, :]).all(-1).sum(0)
    assert np.array_equal(m, ident)


def test_reweight_permutation_equivariant():
    S = _clustered(15, 50, 5)
    perm = np.random.default_rng(0).permutation(50)
    m, _, _, beff = oracle.reweight(S, 0.8)
    mp, _, _, beffp = oracle.reweight(S[perm], 0.8)
    assert np.array_equal(mp, m[perm])
    assert beffp == beff  # histogram order makes B_eff order-independent, bit for bit


# ---------------------------------------------------------------------------
# Objective (Eq. g_regdef2)
# ---------------------------------------------------------------------------
def test_objective_at_zero_is_log_q():
    # theta = 0 -> every conditional is 1/q (Eq. condpfinal), penalty 0, so
    # g_r = ln q and sum_b w_b log P = -B_eff ln q
    S = _clustered(9, 70, 1)
    m, w, _, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    f = oracle.objgrad(S, w, beff, np.zeros((N, Q)), np.zeros((N, Q, N, Q)), grad=False)
    assert np.allclose(f, math.log(Q), rtol=1e-14, atol=0)
    assert np.allclose(-f * beff, -beff * math.log(Q), rtol=1e-14)


def _brute_force_conditionals(h, Jsym, q=Q):
    """Joint Potts distribution (Eq. potts_model) by enumeration of all q^N
    states; returns the joint table with shape (q,)*N."""
    N = h.shape[0]
    grids = np.indices((q,) * N).reshape(N, -1)  # [N, q^N]
    E = np.zeros(grids.shape[1])
    for i in range(N):
        E += h[i, grids[i]]
    for i in range(N):
        for j in range(i + 1, N):
            E += Jsym[i, grids[i], j, grids[j]]
    p = np.exp(E - E.max())
    p /= p.sum()
    return p.reshape((q,) * N)


@pytest.mark.parametrize("N", [3, 4])
def test_conditional_matches_brute_force_joint(N):
    rng = np.random.default_rng(N)
    h = rng.normal(0, 1, (N, Q))
    Jsym = np.zeros((N, Q, N, Q))
    for i in range(N):
        for j in range(i + 1, N):
            blk = rng.normal(0, 0.5, (Q, Q))
            Jsym[i, :, j, :] = blk
            Jsym[j, :, i, :] = blk.T
    joint = _brute_force_conditionals(h, Jsym)
    for t in range(6):
        seq = rng.integers(0, Q, N).astype(np.int8)
        S = seq[None, :]
        f, gh, gJ = oracle.objgrad(S, np.ones(1), 1.0, h, Jsym, 0.0, 0.0)
        for r in range(N):
            idx = list(seq)
            idx[r] = slice(None)
            cond = joint[tuple(idx)]
            cond = cond / cond.sum()
            # objective of one sequence with unit weight is -log P(sigma_r | rest)
            assert f[r] == pytest.approx(-math.log(cond[seq[r]]), rel=1e-12, abs=1e-12)
            # dg/dh_r(s) = P(s | rest) - I[sigma_r = s] (Eq. g_gradh2 with B = 1)
            P = gh[r] + (np.arange(Q) == seq[r])
            assert np.allclose(P, cond, rtol=1e-11, atol=1e-14)


# ---------------------------------------------------------------------------
# Gradient (Eqs. g_gradh2, g_gradJ2)
# ---------------------------------------------------------------------------
def test_gradient_closed_form_at_zero():
    # at theta = 0 every P = 1/q, so from the frequency form (Sec. 3.1)
    #   dg/dh_r(s)    = -(f_r(s) - 1/q)
    #   dg/dJ_ri(s,k) = -(f_ri(s,k) - f_i(k)/q),  i != r
    S = _clustered(7, 90, 2)
    m, w, _, beff = oracle.reweight(S, 0.8)
    B, N = S.shape
    X = _onehot(S)
    f1 = np.einsum("b,bis->is", w, X) / beff
    f2 = np.einsum("b,brs,bik->rsik", w, X, X) / beff
    _, gh, gJ = oracle.objgrad(S, w, beff, np.zeros((N, Q)), np.zeros((N, Q, N, Q)))
    assert np.allclose(gh, -(f1 - 1.0 / Q), rtol=0, atol=1e-14)
    exp = -(f2 - f1[None, None, :, :] / Q)
    for r in range(N):
        exp[r, :, r, :] = 0.0
    assert np.allclose(gJ, exp, rtol=0, atol=1e-14)


def test_gradient_central_differences():
    # central differences, step 1e-4, 64 random coordinates at a random theta
    rng = np.random.default_rng(7)
    S = _clustered(8, 60, 3)
    m, w, _, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    lh, lJp = 0.01, 0.005
    for r in [0, 5]:
        h_r = rng.normal(0, 0.1, Q)
        J_r = rng.normal(0, 0.1, (Q, N, Q))
        J_r[:, r, :] = 0.0
        f0, gh, gJ = oracle.site_objgrad(S, w, beff, r, h_r, J_r, lh, lJp)
        theta = np.concatenate([h_r, J_r.ravel()])
        grad = np.concatenate([gh, gJ.ravel()])
        cand = [c for c in range(theta.size) if not (c >= Q and ((c - Q) // Q) % N == r)]
        coords = rng.choice(cand, 64, replace=False)
        eps = 1e-4
        for c in coords:
            tp, tm = theta.copy(), theta.copy()
            tp[c] += eps
            tm[c] -= eps
            fp = oracle.site_objgrad(S, w, beff, r, tp[:Q], tp[Q:].reshape(Q, N, Q), lh, lJp, grad=False)
            fm = oracle.site_objgrad(S, w, beff, r, tm[:Q], tm[Q:].reshape(Q, N, Q), lh, lJp, grad=False)
            fd = (fp - fm) / (2 * eps)
            assert abs(fd - grad[c]) <= 1e-6 * max(1e-3, abs(grad[c])) + 1e-10, (r, c, fd, grad[c])


def test_gradient_rows_sum_to_penalty():
    # rows of (Y - P) sum to zero over s at every theta, so the data part of
    # both gradients sums to zero over the state of r (Sec. 3.2, the remark
    # before Eq. asymmetricgauge)
    rng = np.random.default_rng(11)
    S = _clustered(6, 50, 4)
    m, w, _, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    h = rng.normal(0, 0.3, (N, Q))
    J = rng.normal(0, 0.3, (N, Q, N, Q))
    for r in range(N):
        J[r, :, r, :] = 0
    lh, lJ = 0.02, 0.03
    _, gh, gJ = oracle.objgrad(S, w, beff, h, J, lh, lJ)
    assert np.allclose((gh - 2 * lh * h).sum(1), 0, atol=1e-14)
    assert np.allclose((gJ - 2 * (0.5 * lJ) * J).sum(1), 0, atol=1e-14)
    for r in range(N):
        assert np.all(gJ[r, :, r, :] == 0)  # the diagonal block is not a parameter


def test_penalty_terms_and_halving():
    # g^(reg) - g at fixed theta is lambda_h ||h_r||^2 + 0.5 lambda_J sum ||J_ri||^2
    rng = np.random.default_rng(5)
    S = _clustered(5, 40, 6)
    m, w, _, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    h = rng.normal(0, 0.5, (N, Q))
    J = rng.normal(0, 0.5, (N, Q, N, Q))
    for r in range(N):
        J[r, :, r, :] = 0
    f0 = oracle.objgrad(S, w, beff, h, J, 0.0, 0.0, grad=False)
    f1 = oracle.objgrad(S, w, beff, h, J, 0.3, 0.7, grad=False)
    pen = 0.3 * (h ** 2).sum(1) + 0.35 * (J ** 2).sum((1, 2, 3))
    assert np.allclose(f1 - f0, pen, rtol=1e-13)


# ---------------------------------------------------------------------------
# Gauge (Sec. 3.2): invariance, the Ising-gauge map, its minimal norm
# ---------------------------------------------------------------------------
def _random_asym(N, rng, sd=0.3):
    h = rng.normal(0, sd, (N, Q))
    J = rng.normal(0, sd, (N, Q, N, Q))
    for r in range(N):
        J[r, :, r, :] = 0
    return h, J


def test_gauge_invariance_of_conditionals():
    # adding u(k) to J_ij(k, .) and subtracting it from h_i(k), or adding a
    # constant to h_i, leaves every conditional unchanged (Sec. 3.2)
    rng = np.random.default_rng(3)
    S = _clustered(6, 40, 8)
    m, w, _, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    Jsym = np.zeros((N, Q, N, Q))
    for i in range(N):
        for j in range(i + 1, N):
            blk = rng.normal(0, 0.4, (Q, Q))
            Jsym[i, :, j, :] = blk
            Jsym[j, :, i, :] = blk.T
    h = rng.normal(0, 1, (N, Q))
    f0 = oracle.objgrad(S, w, beff, h, Jsym, 0.0, 0.0, grad=False)
    i, j = 1, 4
    u = rng.normal(0, 1, Q)
    J2, h2 = Jsym.copy(), h.copy()
    J2[i, :, j, :] += u[:, None]      # site i's copy, state of i first
    J2[j, :, i, :] += u[None, :]      # site j's copy of the same block
    h2[i] -= u
    h2[2] += 3.7                      # a constant added to one field
    f1 = oracle.objgrad(S, w, beff, h2, J2, 0.0, 0.0, grad=False)
    assert np.allclose(f0, f1, rtol=1e-12, atol=1e-13)


def test_ising_gauge_is_the_least_squares_projection():
    # Eq. gauge_change2 removes the part of J of the form a(k) + b(l); the
    # result is the minimal-norm member of the gauge class (Sec. 3.3).  The
    # projection is recomputed here by a least-squares solve.
    rng = np.random.default_rng(0)
    for t in range(5):
        Jb = rng.normal(0, 1, (Q, Q))
        G = oracle.ising_gauge_block(Jb)
        A = np.zeros((Q * Q, 2 * Q))
        for k in range(Q):
            for l in range(Q):
                A[k * Q + l, k] = 1
                A[k * Q + l, Q + l] = 1
        coef, *_ = np.linalg.lstsq(A, Jb.ravel(), rcond=None)
        resid = Jb.ravel() - A @ coef
        assert np.allclose(G.ravel(), resid, atol=1e-12)
        assert np.allclose(G.sum(0), 0, atol=1e-12)   # Eq. isinggauge
        assert np.allclose(G.sum(1), 0, atol=1e-12)
        assert np.allclose(oracle.ising_gauge_block(G), G, atol=1e-13)  # idempotent
        a, b = rng.normal(0, 1, Q), rng.normal(0, 1, Q)
        G2 = oracle.ising_gauge_block(Jb + a[:, None] + b[None, :] + 0.7)
        assert np.allclose(G2, G, atol=1e-12)
        assert np.linalg.norm(Jb + a[:, None] + b[None, :]) >= np.linalg.norm(G) - 1e-12


def test_fn_uses_the_transposed_mirror_block():
    # Build site estimates whose Ising-gauge part is a known G_ij, seen from
    # site i as G(k,l) and from site j as G^T (first index at j), each with
    # different gauge junk; then FN_ij must equal ||G_ij||_F exactly (Eqs.
    # gauge_change2, average2, frob_normtrans2).
    rng = np.random.default_rng(1)
    N = 6
    J = np.zeros((N, Q, N, Q))
    G = {}
    for i in range(N):
        for j in range(i + 1, N):
            g = oracle.ising_gauge_block(rng.normal(0, 1, (Q, Q)))
            G[i, j] = g
            a, b = rng.normal(0, 2, Q), rng.normal(0, 2, Q)
            J[i, :, j, :] = g + a[:, None] + b[None, :]
            a, b = rng.normal(0, 2, Q), rng.normal(0, 2, Q)
            J[j, :, i, :] = g.T + a[:, None] + b[None, :]
    fn, cfn = oracle.scores(J)
    for (i, j), g in G.items():
        assert fn[i, j] == pytest.approx(np.linalg.norm(g), rel=1e-12)
        assert fn[j, i] == fn[i, j]
    assert np.all(np.diag(fn) == 0)
    # min / max combiners (Sec. 6) on identical estimates give the same FN
    fmin, _ = oracle.scores(J, "min")
    fmax, _ = oracle.scores(J, "max")
    assert np.allclose(fmin, fn, rtol=1e-12) and np.allclose(fmax, fn, rtol=1e-12)


def _gauge_by_lstsq(M):
    # Ising-gauge part of a q x q block computed as the residual of a
    # least-squares fit of a(k) + b(l) (independent of the oracle's gauge map)
    A = np.zeros((Q * Q, 2 * Q))
    for k in range(Q):
        for l in range(Q):
            A[k * Q + l, k] = 1
            A[k * Q + l, Q + l] = 1
    coef, *_ = np.linalg.lstsq(A, M.ravel(), rcond=None)
    return (M.ravel() - A @ coef).reshape(Q, Q)


def test_min_max_combiners_on_distinct_estimates():
    # Sec. 6 names the elementwise minimum and maximum of the two gauged
    # estimates as alternatives to the average (Eq. average2).  Site i
    # carries G1 (first index at i) and site j carries G2 transposed, each
    # with its own gauge junk; the combined block is then min(G1, G2),
    # max(G1, G2) or (G1 + G2)/2 elementwise and every score follows.
    rng = np.random.default_rng(11)
    N = 5
    J = np.zeros((N, Q, N, Q))
    G1, G2 = {}, {}
    for i in range(N):
        for j in range(i + 1, N):
            g1 = _gauge_by_lstsq(rng.normal(0, 1, (Q, Q)))
            g2 = _gauge_by_lstsq(rng.normal(0, 1, (Q, Q)))
            G1[i, j], G2[i, j] = g1, g2
            a, b = rng.normal(0, 2, Q), rng.normal(0, 2, Q)
            J[i, :, j, :] = g1 + a[:, None] + b[None, :]
            a, b = rng.normal(0, 2, Q), rng.normal(0, 2, Q)
            J[j, :, i, :] = g2.T + a[:, None] + b[None, :]
    expect = {"min": np.minimum, "max": np.maximum, "mean": lambda x, y: 0.5 * (x + y)}
    for comb, op in expect.items():
        fn, _ = oracle.scores(J, comb)
        l1 = oracle.score_matrix(J, kind="lp", p=1.0, combine=comb)
        fro = oracle.score_matrix(J, kind="fro", combine=comb)
        for (i, j) in G1:
            v = op(G1[i, j], G2[i, j])
            assert fn[i, j] == pytest.approx(np.linalg.norm(v), rel=1e-12), comb
            assert fn[j, i] == fn[i, j]
            assert fro[i, j] == pytest.approx(np.linalg.norm(v), rel=1e-12), comb
            assert l1[i, j] == pytest.approx(np.abs(v).sum(), rel=1e-12), comb
    # the three combiners really differ here
    fmin, _ = oracle.scores(J, "min")
    fmax, _ = oracle.scores(J, "max")
    fmean, _ = oracle.scores(J, "mean")
    assert not np.allclose(fmin, fmax) and not np.allclose(fmin, fmean)


def test_gauge_and_average_commute():
    # both maps are linear, so the order does not matter (Sec. 3.2)
    rng = np.random.default_rng(2)
    A, B_ = rng.normal(0, 1, (Q, Q)), rng.normal(0, 1, (Q, Q))
    lhs = 0.5 * (oracle.ising_gauge_block(A) + oracle.ising_gauge_block(B_))
    rhs = oracle.ising_gauge_block(0.5 * (A + B_))
    assert np.allclose(lhs, rhs, atol=1e-13)


def test_scores_invariant_under_gauge_of_estimates():
    rng = np.random.default_rng(4)
    N = 7
    _, J = _random_asym(N, rng)
    fn, cfn = oracle.scores(J)
    J2 = J.copy()
    for r in range(N):
        for i in range(N):
            if i != r:
                a, b = rng.normal(0, 1, Q), rng.normal(0, 1, Q)
                J2[r, :, i, :] += a[:, None] + b[None, :] + rng.normal()
    fn2, cfn2 = oracle.scores(J2)
    assert np.allclose(fn, fn2, atol=1e-12) and np.allclose(cfn, cfn2, atol=1e-12)


# ---------------------------------------------------------------------------
# APC (Eq. corr_norm2) and the contact list
# ---------------------------------------------------------------------------
def test_apc_exact_rational_hand_case():
    N = 5
    rng = np.random.default_rng(9)
    F = [[Fraction(0)] * N for _ in range(N)]
    for i in range(N):
        for j in range(i + 1, N):
            v = Fraction(int(rng.integers(1, 50)), int(rng.integers(1, 9)))
            F[i][j] = F[j][i] = v
    row = [sum(F[i][j] for j in range(N) if j != i) / (N - 1) for i in range(N)]
    tot = sum(F[i][j] for i in range(N) for j in range(N) if i != j) / (N * (N - 1))
    fn = np.array([[float(v) for v in r] for r in F])
    cfn = oracle.apc(fn)
    for i in range(N):
        for j in range(N):
            exp = Fraction(0) if i == j else F[i][j] - row[j] * row[i] / tot
            assert cfn[i, j] == pytest.approx(float(exp), rel=1e-14, abs=1e-14)


def test_topL_order_ties_and_separation():
    N = 12
    s = np.zeros((N, N))
    s[0, 5] = s[5, 0] = 3.0
    s[1, 7] = s[7, 1] = 2.0
    s[2, 9] = s[9, 2] = 2.0      # tie with (1,7): (1,7) first
    s[3, 4] = s[4, 3] = 9.0      # too close in sequence (|i-j| <= 4)
    s[0, 11] = s[11, 0] = -1.0
    top = oracle.topL(s, 4, 5)
    assert top.tolist() == [[0, 5], [1, 7], [2, 9], [0, 6]]
    all_pairs = oracle.topL(s, 1000, 5)
    assert len(all_pairs) == sum(1 for i in range(N) for j in range(i + 5, N))


# ---------------------------------------------------------------------------
# Minimiser (Sec. 5: L-BFGS; Sec. 3.2 stationarity gauge)
# ---------------------------------------------------------------------------
def test_minimiser_matches_scipy_lbfgsb_within_strong_convexity_bound():
    # g^(reg) is strongly convex with mu = 2 min(lambda_h, lambda'_J), so
    # ||theta - theta*|| <= ||grad g(theta)|| / mu for any theta.  scipy's
    # L-BFGS-B is an independent minimiser of the same function.
    scipy_opt = pytest.importorskip("scipy.optimize")
    S = _clustered(5, 150, 12)
    m, w, _, beff = oracle.reweight(S, 0.8)
    B, N = S.shape
    lh, lJ = 0.01, 0.01
    mu = 2 * min(lh, 0.5 * lJ)
    h, J, info = oracle.solve(S, w, beff, lh, lJ, gtol=1e-7)
    assert np.all(info["gnorm"] <= 1e-7)
    for r in range(N):
        def fg(th):
            f, gh, gJ = oracle.site_objgrad(S, w, beff, r, th[:Q], th[Q:].reshape(Q, N, Q), lh, 0.5 * lJ)
            return f, np.concatenate([gh, gJ.ravel()])
        n = Q + Q * N * Q
        res = scipy_opt.minimize(fg, np.zeros(n), jac=True, method="L-BFGS-B",
                                 options=dict(maxiter=20000, gtol=1e-12, ftol=1e-16, maxcor=20))
        g_sp = np.linalg.norm(fg(res.x)[1])
        th_or = np.concatenate([h[r], J[r].ravel()])
        g_or = np.linalg.norm(fg(th_or)[1])
        bound = (g_sp + g_or) / mu
        assert np.linalg.norm(res.x - th_or) <= bound + 1e-12, (r, np.linalg.norm(res.x - th_or), bound)
        assert bound < 1e-3


def test_stationarity_gauge_at_the_minimiser():
    # Eq. asymmetricgauge: sum_s h_r(s) = 0, sum_s J_ri(s,l) = 0,
    # lambda'_J sum_k J_ri(s,k) = lambda_h h_r(s), each up to the residual
    # gradient: |violation| <= sqrt(q) ||grad|| / (2 lambda)
    S = _clustered(6, 120, 13)
    m, w, _, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    lh, lJ = 0.01, 0.01
    lJp = 0.5 * lJ
    h, J, info = oracle.solve(S, w, beff, lh, lJ, gtol=1e-7)
    for r in range(N):
        gmax = info["gnorm"][r]
        tol_h = math.sqrt(Q) * gmax / (2 * lh)
        tol_J = math.sqrt(Q) * gmax / (2 * lJp)
        assert abs(h[r].sum()) <= tol_h + 1e-12
        for i in range(N):
            if i == r:
                continue
            assert np.all(np.abs(J[r, :, i, :].sum(0)) <= tol_J + 1e-12)
            viol = lJp * J[r, :, i, :].sum(1) - lh * h[r]
            assert np.all(np.abs(viol) <= 2 * lJp * tol_J + 2 * lh * tol_h + 1e-12)


def test_solver_reports_and_start_point():
    S = _clustered(4, 30, 14)
    m, w, _, beff = oracle.reweight(S, 0.8)
    h, J, info = oracle.solve(S, w, beff, gtol=1e-6, sites=[2])
    assert info["status"][0] == 0 and info["gnorm"][0] <= 1e-6
    assert np.all(h[[0, 1, 3]] == 0) and np.all(J[[0, 1, 3]] == 0)
    assert np.all(J[2, :, 2, :] == 0)
    # max_iter = 0 returns the origin, whose objective is ln q
    h0, J0, info0 = oracle.solve(S, w, beff, gtol=1e-6, max_iter=0, sites=[1])
    assert np.all(h0 == 0) and info0["f"][0] == pytest.approx(math.log(Q), rel=1e-14)


def test_planted_couplings_recovered_tiny():
    # sanity of the whole rundown on a tiny planted model: the strongest
    # 30 CFN pairs (no separation filter: planted pairs are random) must
    # contain most of the 30 planted pairs.  Threshold set once from the
    # oracle and frozen.
    fam = synth.tiny()
    res = oracle.plmdca(fam.msa, gtol=1e-6)
    N = fam.N
    iu = np.triu_indices(N, 1)
    order = np.argsort(-res["cfn"][iu], kind="stable")[:30]
    got = {(int(iu[0][o]), int(iu[1][o])) for o in order}
    planted = set(map(tuple, fam.model.pairs.tolist()))
    assert len(got & planted) >= 20


def test_apc_all_zero_fn_is_zero():
    # FN_:: = 0 makes the correction 0/0; the reading taken is 0
    cfn = oracle.apc(np.zeros((6, 6)))
    assert np.all(cfn == 0)
