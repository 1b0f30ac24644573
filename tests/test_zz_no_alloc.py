"""msa_reweight_static: the allocation-free reweighting entry point.

It exists for callers that cannot allocate device memory at the moment they
need sequence weights (code running inside another component's allocator
callback, services that forbid allocation after start-up, callers holding
only a raw stream).  Through the C ABI it must give exactly what
msa_reweight gives -- the counts, the float weights and B_eff bit for bit --
on two calls in a row, although both calls share one static scratch array.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_1401_4832_gb300 import _native
    lib = _native.load()
    P = ctypes.c_void_p
    lib.msa_reweight_static.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, P, P, P, P]
    lib.msa_reweight_static.restype = ctypes.c_int
    return lib


def _static_call(lib, S_dev, x, stream):
    B, N = S_dev.shape
    m = torch.full((B,), -1, dtype=torch.int32, device=S_dev.device)
    w = torch.full((B,), -1.0, dtype=torch.float32, device=S_dev.device)
    beff = torch.full((1,), -1.0, dtype=torch.float64, device=S_dev.device)
    st = lib.msa_reweight_static(ctypes.c_void_p(S_dev.data_ptr()), B, N, 21, float(x),
                                 ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                 ctypes.c_void_p(beff.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    stream.synchronize()
    return m.cpu().numpy(), w.cpu().numpy(), float(beff.cpu().item())


def test_static_reweight_matches_msa_reweight_on_two_calls_in_a_row():
    from paper_1401_4832_gb300 import api
    lib = _lib()
    stream = torch.cuda.current_stream()
    big = synth.add_clusters(synth.protein_family().msa, 0.3, 5, max_redraw=0.15)
    small = synth.add_clusters(synth.small_random(37, 203, 3), 0.4, 3, max_redraw=0.1)
    with api.Context(0, stream) as ctx:
        for S, x in ((big, 0.8), (small, 0.5)):
            S_dev = torch.from_numpy(S).cuda()
            m_ref, w_ref, beff_ref = api.msa_reweight(ctx, S_dev, x)
            m, w, beff = _static_call(lib, S_dev, x, stream)
            assert np.array_equal(m, m_ref.cpu().numpy())
            assert np.array_equal(w.view(np.uint32), w_ref.cpu().numpy().view(np.uint32))
            assert beff == beff_ref
            # and both agree with the oracle (the tolerance of the other
            # reweighting tests: bit for bit)
            m_o, _, w32_o, beff_o = oracle.reweight(S, x)
            assert np.array_equal(m, m_o) and beff == beff_o


def test_static_reweight_rejects_problems_beyond_its_scratch():
    lib = _lib()
    S_dev = torch.zeros((4, 8), dtype=torch.int8, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(out.data_ptr())
    # 200000 sequences of 500 positions need ~64 MiB of planes: refused
    # before any launch, so the small buffers are never touched
    st = lib.msa_reweight_static(ctypes.c_void_p(S_dev.data_ptr()), 200000, 500, 21, 0.8,
                                 p, p, p, None)
    assert st == -2  # PLM_ENOMEM
    st = lib.msa_reweight_static(ctypes.c_void_p(S_dev.data_ptr()), 4, 8, 20, 0.8, p, p, p, None)
    assert st == -1  # PLM_EINVAL


def test_static_reweight_flags_states_outside_the_alphabet():
    # a state outside 0..20 makes B_eff NaN (the call itself succeeds: the
    # check runs on the GPU and the call does not synchronise); the next
    # call with a valid MSA starts from a cleared flag and is exact again
    lib = _lib()
    stream = torch.cuda.current_stream()
    S = synth.small_random(23, 150, 4)
    bad = S.copy()
    bad[17, 5] = 25
    bad[90, 11] = -3
    _, _, beff_bad = _static_call(lib, torch.from_numpy(bad).cuda(), 0.8, stream)
    assert np.isnan(beff_bad)
    m, w, beff = _static_call(lib, torch.from_numpy(S).cuda(), 0.8, stream)
    m_o, _, w32_o, beff_o = oracle.reweight(S, 0.8)
    assert np.array_equal(m, m_o) and beff == beff_o
    assert np.array_equal(w.view(np.uint32), w32_o.view(np.uint32))
