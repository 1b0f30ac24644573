"""GPU score alternatives (Sec. 6) and site frequencies against the oracle.

The GPU computes the scores in FP64 from the same float32 couplings the
oracle reads (cast to double), so they agree to rounding (rtol 1e-9); the
top-L lists must be identical.
"""
import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = 21


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_4832_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def _J(N, seed):
    rng = np.random.default_rng(seed)
    J = rng.normal(0, 0.2, (N, Q, N, Q)).astype(np.float32)
    for r in range(N):
        J[r, :, r, :] = 0
    return J


def test_site_frequencies_match_oracle(ctx):
    from paper_1401_4832_gb300 import api
    S = synth.add_clusters(synth.small_random(37, 1003, 6, gap_p=0.2), 0.3, 6, max_redraw=0.1)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    f = api.msa_frequencies(ctx, torch.from_numpy(S).cuda(), torch.from_numpy(w32).cuda(), beff)
    fo = oracle.site_freqs(S, w32.astype(np.float64), beff)
    assert np.allclose(f.cpu().numpy(), fo, rtol=1e-12, atol=1e-15)


VARIANTS = [
    dict(norm="lp", p=1.0), dict(norm="lp", p=3.0), dict(norm="lp", p=0.5),
    dict(norm="fro", exclude_gap=True), dict(norm="lp", p=1.0, exclude_gap=True),
    dict(norm="fro", correction="asc"), dict(norm="fro", correction="none"),
    dict(norm="lp", p=1.5, combine="min"), dict(norm="fro", combine="max", correction="asc"),
    dict(norm="burkoff"), dict(norm="burkoff", correction="asc"),
]


@pytest.mark.parametrize("v", VARIANTS, ids=lambda v: "-".join(f"{k}={x}" for k, x in v.items()))
def test_score_variant_matches_oracle(ctx, v):
    from paper_1401_4832_gb300 import api
    N = 29
    J = _J(N, 3)
    S = synth.small_random(N, 400, 8, gap_p=0.15)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    freq = oracle.site_freqs(S, w, beff)
    kw = dict(v)
    kind = {"fro": "fro", "lp": "lp", "burkoff": "burkoff"}[kw.get("norm", "fro")]
    sc_o = oracle.score_matrix(J.astype(np.float64), kind, kw.get("p", 2.0),
                               kw.get("exclude_gap", False),
                               freq if kind == "burkoff" else None, kw.get("combine", "mean"))
    corr = kw.get("correction", "apc")
    co_o = oracle.apc(sc_o) if corr == "apc" else oracle.asc(sc_o) if corr == "asc" else sc_o
    if corr == "none":
        np.fill_diagonal(co_o, 0.0)
    sc, co, top = api.plm_scores(ctx, torch.from_numpy(J).cuda(),
                                 freq=torch.from_numpy(freq).cuda() if kind == "burkoff" else None,
                                 **kw)
    assert np.allclose(sc.cpu().numpy(), sc_o, rtol=1e-9, atol=1e-13)
    assert np.allclose(co.cpu().numpy(), co_o, rtol=1e-9, atol=1e-12)
    assert np.array_equal(top.cpu().numpy(), oracle.topL(co_o, N))


def test_score_variant_errors(ctx):
    from paper_1401_4832_gb300 import api, _native
    J = torch.from_numpy(_J(6, 1)).cuda()
    with pytest.raises(_native.PlmError):
        api.plm_scores(ctx, J, norm="burkoff")  # no frequencies
    with pytest.raises(_native.PlmError):
        api.plm_scores(ctx, J, norm="lp", p=0.0)
    f = torch.full((6, Q), 1.0 / Q, dtype=torch.float64, device="cuda")
    with pytest.raises(_native.PlmError):
        api.plm_scores(ctx, J, norm="burkoff", freq=f, exclude_gap=True)


@pytest.mark.parametrize("L", [8, 20, 35, 60])
def test_topL_selection_with_ties_at_the_boundary(ctx, L):
    # one non-zero entry per chosen block: the block's FN is proportional to
    # |v|, so equal v give bitwise equal scores.  Ten distinct scores lie
    # above forty equal ones (the L-th place falls among the equal ones for
    # L = 20, 35 and above them for L = 8); L = 60 takes all fifty.  With no
    # correction the list ranks the FN themselves; it must be the oracle's
    # selection on the same matrix (descending, ties by (i, j)).
    from paper_1401_4832_gb300 import api
    N = 30
    J = np.zeros((N, Q, N, Q), np.float32)
    rng = np.random.default_rng(11)
    pairs = [(i, j) for i in range(N) for j in range(i + 5, N)]
    pick = rng.choice(len(pairs), 50, replace=False)
    for t, p in enumerate(pick):
        i, j = pairs[p]
        J[i, 3, j, 7] = 100.0 + t if t < 10 else 50.0
    sc, co, top = api.plm_scores(ctx, torch.from_numpy(J).cuda(), correction="none", L=L)
    co = co.cpu().numpy()
    top_o = oracle.topL(co, L)
    got = top.cpu().numpy()
    assert np.array_equal(got[:len(top_o)], top_o)
    assert np.all(got[len(top_o):] == -1)


def test_lp2_is_frobenius(ctx):
    # the l_p score with p = 2 is the Frobenius norm (same arithmetic)
    from paper_1401_4832_gb300 import api
    J = torch.from_numpy(_J(17, 5)).cuda()
    a = api.plm_scores(ctx, J, norm="lp", p=2.0)
    b = api.plm_scores(ctx, J, norm="fro")
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_burkoff_large_couplings_match_oracle(ctx):
    # couplings far beyond exp's range (gauged entries of several hundred):
    # both sides take the block maximum off the exponent, so D_ij stays
    # finite and equal to the oracle's
    from paper_1401_4832_gb300 import api
    N = 13
    J = _J(N, 7) * 4000.0
    S = synth.small_random(N, 300, 9, gap_p=0.15)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    freq = oracle.site_freqs(S, w, beff)
    sc_o = oracle.score_matrix(J.astype(np.float64), "burkoff", freq=freq)
    assert np.all(np.isfinite(sc_o))
    sc, co, top = api.plm_scores(ctx, torch.from_numpy(J).cuda(), norm="burkoff",
                                 freq=torch.from_numpy(freq).cuda())
    assert np.allclose(sc.cpu().numpy(), sc_o, rtol=1e-9, atol=1e-12)
    assert np.array_equal(top.cpu().numpy(), oracle.topL(oracle.apc(sc_o), N))
