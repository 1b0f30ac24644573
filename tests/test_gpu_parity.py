"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Bars (written in each test): identity counts and weights bit-exact, B_eff
bit-exact; the exact-FP32 path within relative 1e-6 on the objective and
1e-5 (normwise, infinity norm) on the gradient; solved couplings within the
strong-convexity bound of the oracle's minimiser; identical top-L lists.
"""
import math

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


def _api():
    from paper_1401_4832_gb300 import api
    return api


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(t):
    return t.cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)


def _msas():
    out = {
        "hand": synth.small_random(5, 7, 0),
        "one_seq": synth.small_random(9, 1, 1),
        "one_col": synth.small_random(1, 40, 2),
        "ragged": synth.add_clusters(synth.small_random(37, 203, 3), 0.4, 3, max_redraw=0.1),
        "wide": synth.add_clusters(synth.small_random(70, 130, 4), 0.3, 4, max_redraw=0.15),
        "tiny": synth.tiny().msa,
    }
    return out


# ---------------------------------------------------------------------------
# reweighting: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["hand", "one_seq", "one_col", "ragged", "wide", "tiny"])
@pytest.mark.parametrize("x", [0.0, 0.5, 0.8, 1.0])
def test_reweight_bit_exact(ctx, name, x):
    S = _msas()[name]
    m_o, w_o, w32_o, beff_o = oracle.reweight(S, x)
    m, w, beff = _api().msa_reweight(ctx, _dev(S), x)
    assert np.array_equal(_np(m), m_o)
    assert np.array_equal(_np(w).view(np.uint32), w32_o.view(np.uint32))
    assert beff == beff_o  # same FP64 operations in the same order


def test_reweight_family_size_and_host_buffers(ctx):
    fam = synth.protein_family()
    S = synth.add_clusters(fam.msa, 0.3, 5, max_redraw=0.15)
    m_o, w_o, w32_o, beff_o = oracle.reweight(S, 0.8)
    m, w, beff = _api().msa_reweight(ctx, _dev(S), 0.8)
    assert np.array_equal(_np(m), m_o) and beff == beff_o
    assert np.array_equal(_np(w), w32_o)
    # the same call with host arrays (staged by the library)
    mh, wh, beffh = _api().msa_reweight(ctx, S, 0.8)
    assert isinstance(mh, np.ndarray) and np.array_equal(mh, m_o) and beffh == beff_o


def test_reweight_rejects_bad_states(ctx):
    from paper_1401_4832_gb300 import _native
    S = synth.small_random(10, 20, 6)
    S[3, 4] = 21
    with pytest.raises(_native.PlmError) as e:
        _api().msa_reweight(ctx, _dev(S), 0.8)
    assert e.value.status == _native.PLM_EINVAL


# ---------------------------------------------------------------------------
# objective and gradient: FP32 exact path
# ---------------------------------------------------------------------------
def _random_theta(N, seed, sd=0.2):
    rng = np.random.default_rng(seed)
    h = rng.normal(0, sd, (N, Q))
    J = rng.normal(0, sd, (N, Q, N, Q))
    for r in range(N):
        J[r, :, r, :] = 0
    return h.astype(np.float32).astype(np.float64), J.astype(np.float32).astype(np.float64)


def _check_objgrad(ctx, S, h, J, lh=0.01, lJ=0.01, prec="fp32", rtol_f=1e-6, rtol_g=1e-5):
    m, w, w32, beff = oracle.reweight(S, 0.8)
    f_o, gh_o, gJ_o = oracle.objgrad(S, w, beff, h, J, lh, lJ)
    f, gh, gJ = _api().plm_site_objective_grad(ctx, _dev(S), _dev(w32), beff,
                                               _dev(h.astype(np.float32)),
                                               _dev(J.astype(np.float32)), lh, lJ, prec)
    f, gh, gJ = _np(f), _np(gh), _np(gJ)
    assert np.max(np.abs(f - f_o) / np.abs(f_o)) <= rtol_f
    g_o = np.concatenate([gh_o.ravel(), gJ_o.ravel()])
    g = np.concatenate([gh.ravel(), gJ.ravel()]).astype(np.float64)
    err = np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))
    assert err <= rtol_g, err
    N = S.shape[1]
    for r in range(N):
        assert np.all(gJ[r, :, r, :] == 0)
    return f, gh, gJ


def test_objective_at_zero_is_log_q(ctx):
    S = _msas()["ragged"]
    N = S.shape[1]
    m, w, w32, beff = oracle.reweight(S, 0.8)
    f, gh, gJ = _api().plm_site_objective_grad(ctx, _dev(S), _dev(w32), beff,
                                               _dev(np.zeros((N, Q), np.float32)),
                                               _dev(np.zeros((N, Q, N, Q), np.float32)))
    assert np.allclose(_np(f), math.log(Q), rtol=1e-7, atol=0)


@pytest.mark.parametrize("name", ["one_seq", "ragged", "wide", "tiny"])
def test_objgrad_fp32_matches_oracle(ctx, name):
    S = _msas()[name]
    h, J = _random_theta(S.shape[1], 1)
    _check_objgrad(ctx, S, h, J)


def test_objgrad_fp32_family_size(ctx):
    S = synth.protein_family().msa
    h, J = _random_theta(S.shape[1], 2, sd=0.05)
    _check_objgrad(ctx, S, h, J)


def test_objgrad_lambda_halving_and_host_buffers(ctx):
    S = _msas()["wide"]
    N = S.shape[1]
    h, J = _random_theta(N, 3)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    f_o = oracle.objgrad(S, w, beff, h, J, 0.3, 0.7, grad=False)
    f, gh, gJ = _api().plm_site_objective_grad(ctx, S, w32, beff, h.astype(np.float32),
                                               J.astype(np.float32), 0.3, 0.7)
    assert isinstance(f, np.ndarray)
    assert np.max(np.abs(f - f_o) / np.abs(f_o)) <= 1e-6


# ---------------------------------------------------------------------------
# solve: minimiser within the strong-convexity bound, identical contacts
# ---------------------------------------------------------------------------
def _solve_and_compare(ctx, S, prec, gtol_gpu, sites_checked=None):
    lh, lJ = 0.01, 0.01
    mu = 2 * min(lh, 0.5 * lJ)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    N = S.shape[1]
    h_g, J_g, rep = _api().plm_solve(ctx, _dev(S), gtol=gtol_gpu, prec=prec, max_iter=2000)
    assert rep["n_failed"] == 0, rep
    h_g, J_g = _np(h_g).astype(np.float64), _np(J_g).astype(np.float64)
    sites = list(range(N)) if sites_checked is None else sites_checked
    h_o, J_o, info = oracle.solve(S, w, beff, lh, lJ, gtol=1e-7, sites=sites)
    for t, r in enumerate(sites):
        th_g = np.concatenate([h_g[r], J_g[r].ravel()])
        th_o = np.concatenate([h_o[r], J_o[r].ravel()])
        # the GPU point's true FP64 gradient norm bounds its distance to theta*
        f, gh, gJ = oracle.site_objgrad(S, w, beff, r, h_g[r], J_g[r], lh, 0.5 * lJ)
        gn = math.sqrt((gh ** 2).sum() + (gJ ** 2).sum())
        bound = (gn + info["gnorm"][t]) / mu
        assert np.linalg.norm(th_g - th_o) <= bound * (1 + 1e-6), (r, np.linalg.norm(th_g - th_o), bound)
        assert gn <= max(10 * gtol_gpu, 1e-4), (r, gn)
    return h_g, J_g, h_o, J_o, rep


def test_solve_tiny_fp32_matches_oracle(ctx):
    S = synth.tiny().msa
    h_g, J_g, h_o, J_o, rep = _solve_and_compare(ctx, S, "fp32", 1e-5)
    fn_o, cfn_o = oracle.scores(J_o)
    fn_g, cfn_g, top_g = _api().fn_apc_scores(ctx, _dev(J_g.astype(np.float32)))
    top_o = oracle.topL(cfn_o, S.shape[1], 5)
    assert np.array_equal(_np(top_g)[:len(top_o)], top_o)
    assert np.max(np.abs(_np(cfn_g) - cfn_o)) < 1e-3


# ---------------------------------------------------------------------------
# scores
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 6, 37, 128, 130])  # 128: the most pairs sorted whole; 130: radix select
@pytest.mark.parametrize("combine", ["mean", "min", "max"])
def test_scores_match_oracle(ctx, N, combine):
    rng = np.random.default_rng(N)
    J = rng.normal(0, 0.3, (N, Q, N, Q)).astype(np.float32)
    for r in range(N):
        J[r, :, r, :] = 0
    fn_o, cfn_o = oracle.scores(J.astype(np.float64), combine)
    fn, cfn, top = _api().fn_apc_scores(ctx, _dev(J), combine=combine, L=3 * N, min_sep=1 if N < 6 else 5)
    assert np.allclose(_np(fn), fn_o, rtol=1e-12, atol=1e-12)
    assert np.allclose(_np(cfn), cfn_o, rtol=1e-11, atol=1e-11)
    top_o = oracle.topL(_np(cfn), 3 * N, 1 if N < 6 else 5)
    top = _np(top)
    assert np.array_equal(top[:len(top_o)], top_o)
    assert np.all(top[len(top_o):] == -1)


def test_scores_host_buffers_and_ties(ctx):
    # all couplings zero: every FN and CFN is 0 (the 0/0 correction is taken
    # as 0), so the list is the eligible pairs in (i, j) order
    N = 12
    J = np.zeros((N, Q, N, Q), np.float32)
    fn, cfn, top = _api().fn_apc_scores(ctx, J, L=5)
    assert isinstance(top, np.ndarray)
    assert np.all(np.asarray(fn) == 0) and np.all(np.asarray(cfn) == 0)
    assert top.tolist() == [[0, 5], [0, 6], [0, 7], [0, 8], [0, 9]]
