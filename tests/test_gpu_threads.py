"""Two contexts driven from two host threads at once (each with its own
stream, so each solve runs its lanes and device-side loops) give exactly
the results of the same solves run one after the other: the library keeps
no per-call state outside the context except per-thread launch parameters
and process-wide caches behind locks."""
import threading

import pytest

from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(msa):
    from paper_1401_4832_gb300 import api
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), api.Context(0, stream) as ctx:
        h, J, rep = api.plm_solve(ctx, torch.from_numpy(msa).cuda(), gtol=1e-4,
                                  prec="split_bf16")
        stream.synchronize()
    return h.cpu(), J.cpu(), rep


def test_two_threads_two_contexts():
    msas = [synth.add_clusters(synth.small_random(70, 700, 12), 0.3, 12, max_redraw=0.1),
            synth.add_clusters(synth.small_random(41, 520, 5), 0.3, 5, max_redraw=0.1)]
    ref = [_solve(m) for m in msas]
    out = [None, None]
    errs = []

    def work(k):
        try:
            for _ in range(3):
                out[k] = _solve(msas[k])
                h, J, rep = out[k]
                assert torch.equal(h, ref[k][0]) and torch.equal(J, ref[k][1])
        except Exception as e:  # reported on the main thread
            errs.append(e)

    ts = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not errs, errs
    for k in range(2):
        assert out[k] is not None and out[k][2]["n_converged"] == msas[k].shape[1]
