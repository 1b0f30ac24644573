"""Batched families: many independent families of uneven N and B solved by
one batched L-BFGS, each evaluation covering every family in one launch per
kernel.  Every site's computation depends only on its own family, so the
batched solve must equal separate solves bit for bit; one family is also
checked against the oracle (minimiser bound, identical contacts).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth
from parity_bounds import cfn_bound, compare_top, fn_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1401_4832_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_stream():
    # on a non-default stream the split-BF16 solves run as bench.py times
    # them: CUDA graphs with device-side round loops, two lanes (the batch
    # split at a family boundary, a single family at a tile boundary)
    from paper_1401_4832_gb300 import api
    stream = torch.cuda.Stream()
    c = api.Context(0, stream)
    yield c
    c.close()


def _families():
    # uneven sizes: several tile counts, ragged tails, one very small family
    shapes = [(23, 310, 0), (8, 40, 1), (61, 777, 2), (37, 129, 3), (120, 1000, 4)]
    fams = []
    for N, B, seed in shapes:
        f = synth.family(N, B, int(math.ceil(1.5 * N)), "chain", 0.15, 200, seed + 100,
                         cache=True)
        fams.append(f.msa)
    return fams


@pytest.mark.parametrize("prec,where", [("split_bf16", "default"), ("fp32", "default"),
                                        ("split_bf16", "stream")])
def test_batch_equals_separate_solves(ctx, ctx_stream, prec, where):
    from paper_1401_4832_gb300 import api
    c = ctx if where == "default" else ctx_stream
    msas = _families()
    with torch.cuda.stream(c.stream):
        dev = [torch.from_numpy(m).cuda() for m in msas]
        batch = api.plm_solve_batch(c, dev, gtol=1e-4, prec=prec)
        sep = [api.plm_solve(c, m, gtol=1e-4, prec=prec) for m in dev]
        c.stream.synchronize()
    for m, (h_b, J_b, rep_b), (h_s, J_s, rep_s) in zip(dev, batch, sep):
        assert rep_b["n_converged"] == m.shape[1], rep_b
        assert torch.equal(h_b, h_s) and torch.equal(J_b, J_s)
        assert rep_b["iters"] == rep_s["iters"]


def test_batch_family_matches_oracle(ctx):
    from paper_1401_4832_gb300 import api
    msas = _families()
    batch = api.plm_solve_batch(ctx, [torch.from_numpy(m).cuda() for m in msas], gtol=1e-5,
                                prec="split_bf16")
    lh, lJ = 0.01, 0.01
    mu = 2 * min(lh, 0.5 * lJ)
    for k in (0, 2):
        S = msas[k]
        N = S.shape[1]
        h_g, J_g, rep = batch[k]
        h_g = h_g.cpu().numpy().astype(np.float64)
        J_g = J_g.cpu().numpy().astype(np.float64)
        ro = oracle.plmdca(S, gtol=1e-7)
        m, w, w32, beff = oracle.reweight(S, 0.8)
        for r in range(N):
            _, gh, gJ = oracle.site_objgrad(S, w, beff, r, h_g[r], J_g[r], lh, 0.5 * lJ)
            gn = math.sqrt((gh ** 2).sum() + (gJ ** 2).sum())
            d = np.linalg.norm(np.concatenate([h_g[r] - ro["h"][r], (J_g[r] - ro["J"][r]).ravel()]))
            assert d <= (gn + ro["info"]["gnorm"][r]) / mu * (1 + 1e-6)
        fn, cfn, top = api.fn_apc_scores(ctx, torch.from_numpy(J_g.astype(np.float32)).cuda())
        top_o = ro["top"]
        assert np.array_equal(top.cpu().numpy()[:len(top_o)], top_o)


def _config4_families(count=64):
    # the batch workload's shape: family f seeded with f, N ~ U{50..300},
    # ceil(1.5 N) chain pairs, 15 % gaps; B drawn log-uniformly from
    # [50, 2000] (a tenth of the workload's range) and 50 Gibbs sweeps, to
    # keep the test short
    fams = []
    for f in range(count):
        rng = np.random.default_rng([f, 99])
        N = int(rng.integers(50, 301))
        B = int(round(math.exp(rng.uniform(math.log(50), math.log(2000)))))
        fams.append(synth.family(N, B, int(math.ceil(1.5 * N)), "chain", 0.15, 50, f,
                                 cache=True).msa)
    return fams


def test_batch_of_64_families_equals_separate_solves_and_oracle(ctx_stream):
    # 64 families fill one launch's family table (and its 64 x 2 tensor
    # maps per kernel); the batch must equal the separate solves bit for bit
    # and two families must match the FP64 oracle
    from paper_1401_4832_gb300 import api
    c = ctx_stream
    msas = _config4_families()
    with torch.cuda.stream(c.stream):
        dev = [torch.from_numpy(m).cuda() for m in msas]
        batch = api.plm_solve_batch(c, dev, gtol=1e-4, prec="split_bf16")
        sep = [api.plm_solve(c, m, gtol=1e-4, prec="split_bf16") for m in dev]
        c.stream.synchronize()
    for k, (m, (h_b, J_b, rep_b), (h_s, J_s, rep_s)) in enumerate(zip(dev, batch, sep)):
        assert rep_b["n_converged"] == m.shape[1], (k, rep_b)
        assert torch.equal(h_b, h_s) and torch.equal(J_b, J_s), k
        assert rep_b["iters"] == rep_s["iters"], k
    lh, lJ = 0.01, 0.01
    mu = 2 * min(lh, 0.5 * lJ)
    order = np.argsort([m.shape[0] * m.shape[1] ** 2 for m in msas])
    for k in order[:2]:
        S = msas[k]
        N = S.shape[1]
        h_g, J_g, _ = batch[k]
        h_g = h_g.cpu().numpy().astype(np.float64)
        J_g = J_g.cpu().numpy().astype(np.float64)
        ro = oracle.plmdca(S, gtol=1e-7)
        m, w, w32, beff = oracle.reweight(S, 0.8)
        _, gh, gJ = oracle.objgrad(S, w, beff, h_g, J_g, lh, lJ)
        gn = np.sqrt((gh ** 2).sum(1) + (gJ ** 2).reshape(N, -1).sum(1))
        assert gn.max() <= 2e-4
        for r in range(N):
            d = np.linalg.norm(np.concatenate([h_g[r] - ro["h"][r], (J_g[r] - ro["J"][r]).ravel()]))
            assert d <= (gn[r] + ro["info"]["gnorm"][r]) / mu * (1 + 1e-6), (k, r)
        with torch.cuda.stream(c.stream):
            fn, cfn, top = api.fn_apc_scores(c, batch[k][1])
            c.stream.synchronize()
        bound = fn_bound(gn, ro["info"]["gnorm"], mu)
        assert np.all(np.abs(fn.cpu().numpy() - ro["fn"]) <= bound + 1e-9)
        e = cfn_bound(ro["fn"], bound)
        identical, ok, detail = compare_top(top.cpu().numpy()[:len(ro["top"])], ro["top"],
                                            ro["cfn"], e)
        print(f"batch family {k} (B={S.shape[0]}, N={N}): top-L vs oracle: {detail}")
        assert ok, detail


def test_batch_beyond_one_launch_table(ctx):
    # 67 tiny families: the evaluation kernels run in two launches (64 + 3
    # families); still equal to the separate solves bit for bit
    from paper_1401_4832_gb300 import api
    msas = [synth.small_random(int(6 + f % 11), int(30 + 7 * f), 500 + f) for f in range(67)]
    dev = [torch.from_numpy(m).cuda() for m in msas]
    batch = api.plm_solve_batch(ctx, dev, gtol=1e-4, prec="split_bf16")
    sep = [api.plm_solve(ctx, m, gtol=1e-4, prec="split_bf16") for m in dev]
    for k, ((h_b, J_b, rep_b), (h_s, J_s, rep_s)) in enumerate(zip(batch, sep)):
        assert torch.equal(h_b, h_s) and torch.equal(J_b, J_s), k
        assert rep_b["n_converged"] == msas[k].shape[1], (k, rep_b)
