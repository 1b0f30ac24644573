"""Invalid arguments at the C ABI: every entry point of the solve path
rejects them with PLM_EINVAL (a message in plm_last_error), launches
nothing that could fault, and leaves the context usable -- a valid solve on
the same context afterwards gives the result a fresh context gives."""
import numpy as np
import pytest

from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _einval(fn):
    from paper_1401_4832_gb300 import _native
    with pytest.raises(_native.PlmError) as e:
        fn()
    assert e.value.status == _native.PLM_EINVAL, e.value
    assert str(e.value).split(":", 1)[1].strip()  # a message


def test_invalid_arguments_leave_the_context_usable():
    from paper_1401_4832_gb300 import api
    S = synth.tiny().msa
    Sd = torch.from_numpy(S).cuda()
    B, N = S.shape
    bad_state = S.copy()
    bad_state[B // 2, N // 2] = 21
    neg_state = S.copy()
    neg_state[1, 1] = -1
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), api.Context(0, stream) as ctx:
        _einval(lambda: api.plm_solve(ctx, torch.from_numpy(bad_state).cuda()))
        _einval(lambda: api.plm_solve(ctx, torch.from_numpy(neg_state).cuda()))
        _einval(lambda: api.plm_solve(ctx, Sd[:0]))                # no sequences
        _einval(lambda: api.plm_solve(ctx, Sd[:, :1].contiguous()))  # one position
        _einval(lambda: api.plm_solve(ctx, Sd, lbfgs_m=0))
        _einval(lambda: api.plm_solve(ctx, Sd, lbfgs_m=9))
        _einval(lambda: api.plm_solve(ctx, Sd, gtol=-1.0))
        _einval(lambda: api.plm_solve(ctx, Sd, lambda_J=0.0))
        _einval(lambda: api.plm_solve(ctx, Sd, x=1.5))
        _einval(lambda: api.plm_solve(ctx, Sd, max_ls=0))
        _einval(lambda: api.plm_solve_symmetric(ctx, torch.from_numpy(bad_state).cuda()))
        _einval(lambda: api.plm_solve_batch(ctx, []))
        _einval(lambda: api.plm_solve_batch(ctx, [Sd, torch.from_numpy(bad_state).cuda()]))
        m, w, beff = api.msa_reweight(ctx, Sd)
        h0 = torch.zeros((N, 21), device="cuda")
        J0 = torch.zeros((N, 21, N, 21), device="cuda")
        _einval(lambda: api.plm_site_objective_grad(ctx, Sd, w, 0.0, h0, J0))
        _einval(lambda: api.plm_site_objective_grad(ctx, Sd, w, beff, h0, J0, -0.1, 0.01))
        _einval(lambda: api.msa_reweight(ctx, torch.from_numpy(bad_state).cuda()))
        h1, J1, r1 = api.plm_solve(ctx, Sd, gtol=1e-5)
        stream.synchronize()
    with torch.cuda.stream(stream), api.Context(0, stream) as fresh:
        h2, J2, r2 = api.plm_solve(fresh, Sd, gtol=1e-5)
        stream.synchronize()
    assert r1["n_converged"] == N
    assert torch.equal(h1, h2) and torch.equal(J1, J2)
