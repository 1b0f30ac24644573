"""Failure detection without a GPU fault: the bounded wait every
tensor-core pipeline stage uses gives up on a barrier that nothing arrives
on, the kernel records a timeout code and returns, the host reports
PLM_ETIMEOUT, and the same context then solves normally."""
import time

import pytest

from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_1401_4832_gb300 import api
    S = torch.from_numpy(synth.tiny().msa).cuda()
    with api.Context(0) as ctx:
        t0 = time.perf_counter()
        status, code = api.selftest_wait(ctx)
        dt = time.perf_counter() - t0
        assert status == "PLM_ETIMEOUT" and code != 0
        assert 0.2 < dt < 30.0  # the budget is ~2 s of SM clock cycles
        h, J, rep = api.plm_solve(ctx, S, gtol=1e-4, prec="split_bf16")
        torch.cuda.synchronize()
        assert rep["n_converged"] == S.shape[1]
        assert torch.isfinite(J).all()
