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
