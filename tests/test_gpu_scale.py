"""The scale workload: N=500 positions (Nq = 10500), B=50000 sequences, 750
planted chain contacts, 20 % gaps.

* Full size, one evaluation at a random point, both precisions: the oracle
  computes the objective and the gradient of three sampled sites one by one
  (its full evaluation would take minutes); bars as in the other parity
  tests (FP32: 1e-6 / 1e-5; split-BF16: 1e-4 / 2e-3).
* A 2000-sequence subsample (drawn without replacement, seed 1): the GPU
  split-BF16 solve against the oracle's solve of four sampled sites (each
  site problem is independent): distance within the strong-convexity bound,
  and FN of the pairs among those sites within its bound; the split-BF16 and
  FP32 GPU solves give the same top-N list up to ties inside the score error.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = 21
LH, LJ = 0.01, 0.01
MU = 2 * min(LH, 0.5 * LJ)


@pytest.fixture(scope="module")
def scale():
    # 20 sweeps keep the test's generation short; the shape is what matters here
    return synth.scale_family(sweeps=20)


@pytest.fixture(scope="module")
def ctx():
    # a non-default stream, as bench.py uses: the split-BF16 solves then run
    # in two lanes with device-side round loops (N = 500: lanes of 256 and
    # 244 sites)
    from paper_1401_4832_gb300 import api
    stream = torch.cuda.Stream()
    c = api.Context(0, stream)
    yield c
    c.close()


@pytest.fixture(autouse=True)
def _on_ctx_stream(ctx):
    with torch.cuda.stream(ctx.stream):
        yield
    ctx.stream.synchronize()


@pytest.mark.parametrize("prec,rf,rg", [("split_bf16", 1e-4, 2e-3), ("fp32", 1e-6, 1e-5)])
def test_scale_objgrad_sampled_sites(ctx, scale, prec, rf, rg):
    from paper_1401_4832_gb300 import api
    S = scale.msa
    B, N = S.shape
    assert (B, N) == (50000, 500)
    # the evaluation takes the weights as an input: unit weights (B_eff = B)
    w32 = np.ones(B, np.float32)
    w64 = np.ones(B)
    beff = float(B)
    rng = np.random.default_rng(5)
    h = rng.normal(0, 0.05, (N, Q)).astype(np.float32)
    J = (rng.normal(0, 0.02, (N, Q, N, Q))).astype(np.float32)
    for r in range(N):
        J[r, :, r, :] = 0
    Sd = torch.from_numpy(S).cuda()
    f, gh, gJ = api.plm_site_objective_grad(ctx, Sd, torch.from_numpy(w32).cuda(), beff,
                                            torch.from_numpy(h).cuda(), torch.from_numpy(J).cuda(),
                                            LH, LJ, prec)
    f, gh, gJ = f.cpu().numpy(), gh.cpu().numpy(), gJ.cpu().numpy()
    for r in (0, 257, 499):
        fo, gho, gJo = oracle.site_objgrad(S, w64, beff, r, h[r].astype(np.float64),
                                           J[r].astype(np.float64), LH, 0.5 * LJ)
        assert abs(f[r] - fo) <= rf * abs(fo), (r, f[r], fo)
        g = np.concatenate([gh[r].ravel(), gJ[r].ravel()]).astype(np.float64)
        go = np.concatenate([gho.ravel(), gJo.ravel()])
        assert np.max(np.abs(g - go)) <= rg * np.max(np.abs(go)), (r, np.max(np.abs(g - go)))


def test_scale_subsample_solve(ctx, scale):
    from paper_1401_4832_gb300 import api
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(scale.B, 2000, replace=False))
    S = np.ascontiguousarray(scale.msa[rows])
    N = S.shape[1]
    Sd = torch.from_numpy(S).cuda()
    h_g, J_g, rep = api.plm_solve(ctx, Sd, gtol=1e-4, prec="split_bf16")
    assert rep["n_converged"] == N, rep
    fn_g, cfn_g, top_g = api.fn_apc_scores(ctx, J_g)
    h_g = h_g.cpu().numpy().astype(np.float64)
    J_g = J_g.cpu().numpy().astype(np.float64)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    sites = [3, 120, 301, 480]
    h_o, J_o, info = oracle.solve(S, w, beff, LH, LJ, gtol=1e-6, sites=sites)
    gn = {}
    for t, r in enumerate(sites):
        _, gh, gJ = oracle.site_objgrad(S, w, beff, r, h_g[r], J_g[r], LH, 0.5 * LJ)
        gn[r] = math.sqrt((gh ** 2).sum() + (gJ ** 2).sum())
        assert gn[r] <= 2e-4
        th_g = np.concatenate([h_g[r], J_g[r].ravel()])
        th_o = np.concatenate([h_o[r], J_o[r].ravel()])
        assert np.linalg.norm(th_g - th_o) <= (gn[r] + info["gnorm"][t]) / MU * (1 + 1e-6)
    # FN of the pairs among the sampled sites (both estimates from solved sites)
    fn_o, _ = oracle.scores(J_o)
    fn_g = fn_g.cpu().numpy()
    go = dict(zip(sites, info["gnorm"]))
    for a in range(len(sites)):
        for b in range(a + 1, len(sites)):
            i, j = sites[a], sites[b]
            bound = (gn[i] + gn[j] + go[i] + go[j]) / (2 * MU)
            assert abs(fn_g[i, j] - fn_o[i, j]) <= bound + 1e-9
    # the plain FP32 path gives the same contacts up to ties in the score error
    h32, J32, rep32 = api.plm_solve(ctx, Sd, gtol=1e-4, prec="fp32")
    fn32, cfn32, top32 = api.fn_apc_scores(ctx, J32)
    cfn32 = cfn32.cpu().numpy()
    tol = 2 * float(np.max(np.abs(cfn_g.cpu().numpy() - cfn32))) + 1e-12
    a = set(map(tuple, top_g.cpu().numpy().tolist()))
    b = set(map(tuple, top32.cpu().numpy().tolist()))
    boundary = cfn32[tuple(top32.cpu().numpy()[-1])]
    for i, j in a ^ b:
        assert abs(cfn32[i, j] - boundary) <= tol
