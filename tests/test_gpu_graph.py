"""The solver's per-iteration launches replayed from CUDA graphs must give
exactly the eager result (same kernels, same order, same arguments)."""
import pytest

from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_graph_replay_equals_eager(prec):
    from paper_1401_4832_gb300 import api
    stream = torch.cuda.Stream()  # graphs need a capturable (non-legacy) stream
    S = torch.from_numpy(synth.tiny().msa).cuda()
    with torch.cuda.stream(stream), api.Context(0, stream) as ctx:
        h1, J1, r1 = api.plm_solve(ctx, S, gtol=1e-5, prec=prec, use_graph=1)
        h0, J0, r0 = api.plm_solve(ctx, S, gtol=1e-5, prec=prec, use_graph=0)
        stream.synchronize()
    assert torch.equal(h0, h1) and torch.equal(J0, J1)
    assert r0["iters"] == r1["iters"] and r0["evals"] == r1["evals"]
    assert r1["n_converged"] == S.shape[1]


@pytest.mark.parametrize("tiles", ["8,224", "8,224,256", "12,224,128,1", "12,176,256,1",
                                   "10,224,128,1", "12,224,256,1,1"])
@pytest.mark.parametrize("which", ["family", "ragged"])
def test_two_lane_pipeline_equals_one_lane(which, tiles, monkeypatch):
    # With graphs on, a one-family tensor-core solve runs in two lanes (two
    # streams, device-side loops, one lane rotated by half a round) when the
    # sites split at a boundary shared by the site groups and the gradient
    # row tiles (6 or 12 sites on one CTA, 32 sites on CTA pairs); with
    # 8-site groups that boundary is a multiple of 24 sites (N = 120: 72 +
    # 48; N = 70: 24 + 46), with 12-site groups one of 12 (N = 120: 60 + 60),
    # with 10-site groups and 128-row tiles one of 30 (N = 120: 60 + 60;
    # N = 70: 30 + 40).
    # Each site's iterates depend only on its own row block, so the result
    # must equal the one-lane eager solve bit for bit.
    from paper_1401_4832_gb300 import api
    monkeypatch.setenv("PLMDCA_TC_TILES", tiles)
    if which == "family":
        S = synth.protein_family().msa
    else:  # N = 70: lanes of 32 and 38 sites, ragged tiles in both GEMM dimensions
        S = synth.add_clusters(synth.small_random(70, 700, 12), 0.3, 12, max_redraw=0.1)
    stream = torch.cuda.Stream()
    Sd = torch.from_numpy(S).cuda()
    with torch.cuda.stream(stream), api.Context(0, stream) as ctx:
        h1, J1, r1 = api.plm_solve(ctx, Sd, gtol=1e-4, prec="split_bf16", use_graph=1)
        h0, J0, r0 = api.plm_solve(ctx, Sd, gtol=1e-4, prec="split_bf16", use_graph=0)
        stream.synchronize()
    assert torch.equal(h0, h1) and torch.equal(J0, J1)
    assert r0["iters"] == r1["iters"] and r0["evals"] == r1["evals"]
    assert r1["n_converged"] == S.shape[1], r1
