"""The scale workload: N=500 positions (Nq = 10500), B=50000 sequences, 750
planted chain contacts, 20 % gaps.

* Full size, one evaluation at a random point, both precisions: the oracle
  computes the objective and the gradient of three sampled sites one by one
  (its full evaluation would take minutes); bars as in the other parity
  tests (FP32: 1e-6 / 1e-5; split-BF16: 1e-4 / 2e-3).
* A 2000-sequence subsample (drawn without replacement, seed 1), both
  precisions, against the FP64 oracle's full rundown of all 500 sites
  (to ||grad|| <= 1e-6), stored with the subsample itself in
  tests/golden/scale_subsample_N500_B2000.npz by
  tests/golden/make_scale_golden.py, which calls only the oracle (its solve
  takes about 20 minutes of host time).  Bars: every site reaches gtol;
  four sampled sites, solved again by the oracle here, lie within the
  strong-convexity bound of the GPU point; every pair's FN and CFN within
  the error bound of tests/parity_bounds.py (gradient norms at the GPU point
  computed by the oracle in FP64); the top-N list identical up to ties
  inside that bound, with exact identity printed and recorded.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth
from parity_bounds import cfn_bound, compare_top, fn_bound

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


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "scale_subsample_N500_B2000.npz")


@pytest.fixture(scope="module")
def golden():
    g = np.load(GOLDEN)
    N = g["msa"].shape[1]
    iu = np.triu_indices(N, 1)
    out = dict(msa=g["msa"], gnorm=g["gnorm"], top=g["top"])
    for k in ("fn", "cfn"):
        M = np.zeros((N, N))
        M[iu] = g[k + "_upper"].astype(np.float64)
        out[k] = M + M.T
    return out


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_scale_subsample_solve(ctx, golden, prec, record_property):
    from paper_1401_4832_gb300 import api
    S = golden["msa"]
    assert S.shape == (2000, 500)
    N = S.shape[1]
    Sd = torch.from_numpy(S).cuda()
    h_g, J_g, rep = api.plm_solve(ctx, Sd, gtol=1e-4, prec=prec)
    assert rep["n_converged"] == N, rep
    fn_g, cfn_g, top_g = api.fn_apc_scores(ctx, J_g)
    h_g = h_g.cpu().numpy().astype(np.float64)
    J_g = J_g.cpu().numpy().astype(np.float64)
    m, w, w32, beff = oracle.reweight(S, 0.8)
    # FP64 gradient norms at the GPU point, every site (one oracle evaluation)
    _, gh, gJ = oracle.objgrad(S, w, beff, h_g, J_g, LH, LJ)
    gn = np.sqrt((gh ** 2).sum(1) + (gJ ** 2).reshape(N, -1).sum(1))
    del gJ
    assert gn.max() <= 2e-4, gn.max()
    # four sites solved again by the oracle: distance within the bound
    sites = [3, 120, 301, 480]
    h_o, J_o, info = oracle.solve(S, w, beff, LH, LJ, gtol=1e-6, sites=sites)
    for t, r in enumerate(sites):
        th_g = np.concatenate([h_g[r], J_g[r].ravel()])
        th_o = np.concatenate([h_o[r], J_o[r].ravel()])
        assert np.linalg.norm(th_g - th_o) <= (gn[r] + info["gnorm"][t]) / MU * (1 + 1e-6)
    # every pair against the stored oracle rundown
    bound = fn_bound(gn, golden["gnorm"], MU)
    err = np.abs(fn_g.cpu().numpy() - golden["fn"])
    assert np.all(err <= bound + 1e-6)  # + the float32 rounding of the stored FN
    e = cfn_bound(golden["fn"], bound)
    cerr = np.abs(cfn_g.cpu().numpy() - golden["cfn"])
    assert np.all(cerr <= e + 1e-6)
    top_o = golden["top"]
    identical, ok, detail = compare_top(top_g.cpu().numpy()[:len(top_o)], top_o, golden["cfn"], e)
    print(f"scale subsample {prec}: top-{len(top_o)} vs oracle: {detail}; max |FN err| "
          f"{err.max():.3g} (bound {bound.max():.3g}), max |CFN err| {cerr.max():.3g} "
          f"(bound {e.max():.3g})")
    record_property("top_L_identical", identical)
    record_property("max_cfn_err", float(cerr.max()))
    assert ok, detail
