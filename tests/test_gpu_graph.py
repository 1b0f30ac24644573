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
