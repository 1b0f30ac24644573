"""GPU parity of the split-BF16 tensor-core path (tcgen05) against the oracle.

Tolerance, from the arithmetic: Theta = hi + lo with hi = RN_bf16(Theta)
and lo = RN_bf16(Theta - hi) represents Theta to a relative 2^-16 (bf16 has
an 8-bit significand, unit roundoff 2^-8, applied twice); the one-hot
operand is exact; products accumulate in FP32.  A logit is off by at most
2^-16 * sum_i |Theta_ri(s, S_bi)| plus FP32 rounding of the sum, so with
|Theta| <= 0.2-ish and N <= 120 the logits and the objective move by
<= ~1e-4 relative; the residual D is split the same way (2^-16 relative),
so the gradient moves by <= ~1e-3 of its largest entry.  The tests use
1e-4 (objective) and 2e-3 (gradient, infinity norm relative to max |g|).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = 21
RTOL_F = 1e-4
RTOL_G = 2e-3


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


def _theta(N, seed, sd):
    rng = np.random.default_rng(seed)
    h = rng.normal(0, sd, (N, Q)).astype(np.float32)
    J = rng.normal(0, sd, (N, Q, N, Q)).astype(np.float32)
    for r in range(N):
        J[r, :, r, :] = 0
    return h, J


def _compare(ctx, S, h, J, lh=0.01, lJ=0.01):
    m, w, w32, beff = oracle.reweight(S, 0.8)
    f_o, gh_o, gJ_o = oracle.objgrad(S, w, beff, h.astype(np.float64), J.astype(np.float64), lh, lJ)
    f, gh, gJ = _api().plm_site_objective_grad(ctx, _dev(S), _dev(w32), beff, _dev(h), _dev(J),
                                               lh, lJ, "split_bf16")
    f, gh, gJ = f.cpu().numpy(), gh.cpu().numpy(), gJ.cpu().numpy()
    ef = np.max(np.abs(f - f_o) / np.abs(f_o))
    g = np.concatenate([gh.ravel(), gJ.ravel()]).astype(np.float64)
    g_o = np.concatenate([gh_o.ravel(), gJ_o.ravel()])
    eg = np.max(np.abs(g - g_o)) / np.max(np.abs(g_o))
    assert ef <= RTOL_F, ef
    assert eg <= RTOL_G, eg
    N = S.shape[1]
    for r in range(N):
        assert np.all(gJ[r, :, r, :] == 0)
    return ef, eg


def test_tc_objective_at_zero(ctx):
    # theta = 0: every logit is exactly 0 in any precision, so g_r = ln q
    S = synth.small_random(12, 150, 7)
    N = S.shape[1]
    m, w, w32, beff = oracle.reweight(S, 0.8)
    f, gh, gJ = _api().plm_site_objective_grad(ctx, _dev(S), _dev(w32), beff,
                                               _dev(np.zeros((N, Q), np.float32)),
                                               _dev(np.zeros((N, Q, N, Q), np.float32)),
                                               prec="split_bf16")
    assert np.allclose(f.cpu().numpy(), math.log(Q), rtol=1e-6, atol=0)
    _, gh_o, gJ_o = oracle.objgrad(S, w, beff, np.zeros((N, Q)), np.zeros((N, Q, N, Q)))
    assert np.max(np.abs(gJ.cpu().numpy() - gJ_o)) <= 1e-5 * np.max(np.abs(gJ_o))


@pytest.mark.parametrize("N,B,seed", [(3, 40, 1), (9, 129, 2), (20, 300, 3), (37, 203, 4),
                                      (70, 260, 5)])
def test_tc_objgrad_matches_oracle(ctx, N, B, seed):
    # several tiles in both GEMM dimensions, ragged tails (B % 128, N % 8, K % 256)
    S = synth.add_clusters(synth.small_random(N, B, seed), 0.3, seed, max_redraw=0.1)
    h, J = _theta(N, seed, 0.2)
    _compare(ctx, S, h, J)


def test_tc_objgrad_family_size(ctx):
    S = synth.protein_family().msa
    h, J = _theta(S.shape[1], 9, 0.05)
    _compare(ctx, S, h, J)


def test_tc_matches_fp32_path(ctx):
    S = synth.tiny().msa
    N = S.shape[1]
    h, J = _theta(N, 11, 0.3)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    out = {}
    for prec in ("fp32", "split_bf16"):
        f, gh, gJ = _api().plm_site_objective_grad(ctx, _dev(S), _dev(w32), beff, _dev(h), _dev(J),
                                                   0.01, 0.01, prec)
        out[prec] = (f.cpu().numpy(), gJ.cpu().numpy())
    assert np.max(np.abs(out["fp32"][0] - out["split_bf16"][0]) / out["fp32"][0]) <= RTOL_F
    assert np.max(np.abs(out["fp32"][1] - out["split_bf16"][1])) <= RTOL_G * np.max(np.abs(out["fp32"][1]))


def test_tc_solve_tiny_identical_contacts(ctx):
    # the reduced-precision solve must give the oracle's top-L list; the FN
    # error is bounded by (||g_i|| + ||g_j||) / (2 mu) with the GPU point's
    # true gradient norms (strong convexity, mu = 2 min(lambda_h, lambda'_J))
    fam = synth.tiny()
    S = fam.msa
    N = S.shape[1]
    lh, lJ = 0.01, 0.01
    mu = 2 * min(lh, 0.5 * lJ)
    h_g, J_g, rep = _api().plm_solve(ctx, _dev(S), gtol=1e-4, prec="split_bf16")
    assert rep["n_failed"] == 0, rep
    h_g, J_g = h_g.cpu().numpy().astype(np.float64), J_g.cpu().numpy().astype(np.float64)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    gn = np.zeros(N)
    for r in range(N):
        _, gh, gJ = oracle.site_objgrad(S, w, beff, r, h_g[r], J_g[r], lh, 0.5 * lJ)
        gn[r] = math.sqrt((gh ** 2).sum() + (gJ ** 2).sum())
    ro = oracle.plmdca(S, gtol=1e-7)
    fn_g, cfn_g, top_g = _api().fn_apc_scores(ctx, _dev(J_g.astype(np.float32)))
    fn_g = fn_g.cpu().numpy()
    bound = (gn[:, None] + gn[None, :] + 2e-7) / (2 * mu)
    np.fill_diagonal(bound, 0)
    assert np.all(np.abs(fn_g - ro["fn"]) <= bound + 1e-6)
    top_o = ro["top"]
    assert np.array_equal(top_g.cpu().numpy()[:len(top_o)], top_o)


TILE_SHAPES = ([(s, 256, 128, 0, 0) for s in (2, 4, 6, 10)]
               + [(8, c, 128, 0, 0) for c in (32, 128, 144, 160, 176, 192, 224)]
               + [(8, c, 256, 0, 0) for c in (32, 48, 128, 176, 208, 224, 256)]
               + [(s, 256, 128, 1, 0) for s in (4, 8, 10, 12)]
               + [(12, c, 256, 1, 1) for c in (128, 160, 192, 224, 256)])


@pytest.mark.parametrize("sites,cols,rows,pair,gpair", TILE_SHAPES)
def test_tc_every_tile_shape(sites, cols, rows, pair, gpair, monkeypatch):
    # every shape the autotuner may pick gives the same numbers (ragged in
    # both GEMM dimensions: N=37 -> 37 % sites != 0, K = 800 -> K % cols != 0;
    # one CTA packs 6 sites per 128 gradient rows, so the last 256-row tile
    # holds one site and its second half lies wholly beyond N; on CTA pairs
    # R = 37 * 24 = 888 padded rows -> the last 256-row tile holds 120 real
    # rows); widths that are odd multiples of 16 split the epilogue's column
    # groups unevenly; pair = 1: the logits on 2-CTA clusters, gpair = 1:
    # the gradient on 2-CTA clusters
    from paper_1401_4832_gb300 import api
    monkeypatch.setenv("PLMDCA_TC_TILES", f"{sites},{cols},{rows},{pair},{gpair}")
    S = synth.add_clusters(synth.small_random(37, 203, 4), 0.3, 4, max_redraw=0.1)
    h, J = _theta(37, 4, 0.2)
    with api.Context(0) as c:
        _compare(c, S, h, J)


@pytest.mark.parametrize("sites,gpair", [(4, 0), (8, 0), (10, 0), (12, 0), (12, 1)])
@pytest.mark.parametrize("N,B", [(50, 300), (23, 129), (120, 5000)])
def test_tc_pair_logits_ragged(sites, gpair, N, B, monkeypatch):
    # 2-CTA logits tiles: an odd number of 128-sequence tiles (the last pair
    # has one real tile: B = 300 -> 3 tiles, B = 129 -> 2 tiles of which the
    # second holds one sequence), site groups ragged in N, and the family
    # size; the same bars as every other tile shape
    from paper_1401_4832_gb300 import api
    monkeypatch.setenv("PLMDCA_TC_TILES", f"{sites},224,256,1,{gpair}")
    if N == 120:
        S = synth.protein_family().msa
    else:
        S = synth.add_clusters(synth.small_random(N, B, 6), 0.3, 6, max_redraw=0.1)
    h, J = _theta(N, 7, 0.05 if N == 120 else 0.2)
    with api.Context(0) as c:
        _compare(c, S, h, J)


def test_tc_pair_equals_single_cta_logits(monkeypatch):
    # the pair tile and the single-CTA tile accumulate the same products in
    # the same K order: the objective and the residual-driven gradient agree
    # to FP32 rounding of the accumulation (the tensor core's order inside
    # one instruction is its own), checked at 1e-6 relative
    from paper_1401_4832_gb300 import api
    S = synth.add_clusters(synth.small_random(61, 700, 8), 0.3, 8, max_redraw=0.1)
    h, J = _theta(61, 8, 0.1)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    out = {}
    for pair in (0, 1):
        monkeypatch.setenv("PLMDCA_TC_TILES", f"8,224,256,{pair}")
        with api.Context(0) as c:
            f, gh, gJ = api.plm_site_objective_grad(c, _dev(S), _dev(w32), beff, _dev(h), _dev(J),
                                                    0.01, 0.01, "split_bf16")
            out[pair] = (f.cpu().numpy(), gJ.cpu().numpy())
    assert np.allclose(out[0][0], out[1][0], rtol=1e-6, atol=0)
    g0, g1 = out[0][1], out[1][1]
    assert np.max(np.abs(g0 - g1)) <= 1e-5 * np.max(np.abs(g0))


def test_tc_autotuner_tries_every_shape_in_one_process():
    # the tuner launches every candidate (single-CTA and pair logits, every
    # gradient shape and width) in one process: each kernel's shared-memory
    # limit must cover the largest of its shapes, whatever order they come in
    from paper_1401_4832_gb300 import api
    S = synth.add_clusters(synth.small_random(45, 900, 13), 0.3, 13, max_redraw=0.1)
    h, J = _theta(45, 13, 0.1)
    with api.Context(0) as c:
        ef, eg = _compare(c, S, h, J)


@pytest.mark.parametrize("N,B", [(2, 1), (5, 127), (13, 129), (7, 257)])
@pytest.mark.parametrize("tiles", ["12,224,256,1,0", "4,128,256,1,1", "12,256,256,2,1",
                                   "10,176,128,1,0"])
def test_tc_pair_shapes_at_the_edges(N, B, tiles, monkeypatch):
    # smallest problems on the 2-CTA kernels: fewer sites than half a tile
    # (the peer CTA's Theta box lies wholly beyond N and reads zeros), one
    # sequence, a single 128-sequence tile (the pair's second CTA computes
    # nothing), 257 sequences (three tiles, the last with one sequence)
    from paper_1401_4832_gb300 import api
    monkeypatch.setenv("PLMDCA_TC_TILES", tiles)
    S = synth.small_random(N, B, 30 + N)
    h, J = _theta(N, 30 + N, 0.2)
    with api.Context(0) as c:
        _compare(c, S, h, J)
