"""Python binding of the plmDCA C ABI (argument marshalling only).

Every function takes a :class:`Context` plus torch tensors (CUDA or CPU) or
numpy arrays, passes their raw pointers to the C library, and returns
outputs allocated next to the inputs: CUDA tensors when the MSA is on the
GPU, host arrays otherwise (the library stages host arrays through device
memory itself).  All arithmetic happens in the library's CUDA kernels.

Names follow the C calls: ``msa_reweight``, ``plm_site_objective_grad``,
``plm_solve``, ``fn_apc_scores``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N_

Q = 21


def _torch():
    import torch
    return torch


class Context:
    """Owns one ``plm_ctx`` (device workspace) bound to a CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        self.lib = N_.load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.device = device
        self.stream = stream
        handle = ctypes.c_void_p()
        st = self.lib.plm_create(ctypes.byref(handle), device,
                                 ctypes.c_void_p(stream.cuda_stream))
        if st != N_.PLM_OK:
            raise N_.PlmError(st, "plm_create failed")
        self.handle = handle

    def check(self, status):
        if status != N_.PLM_OK:
            msg = self.lib.plm_last_error(self.handle)
            raise N_.PlmError(status, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.plm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:
        return False


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr())
    assert x.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(x.ctypes.data)


def _like(ref, shape, dtype_np):
    """Output buffer beside ``ref``: a CUDA tensor if ref is one, else numpy."""
    if _is_torch(ref) and ref.is_cuda:
        torch = _torch()
        tdt = {np.float32: torch.float32, np.float64: torch.float64,
               np.int32: torch.int32}[dtype_np]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype_np)


def _as_input(x, dtype_np):
    if _is_torch(x):
        torch = _torch()
        tdt = {np.int8: torch.int8, np.float32: torch.float32}[dtype_np]
        return x.to(tdt).contiguous()
    return np.ascontiguousarray(x, dtype=dtype_np)


def msa_reweight(ctx: Context, msa, x: float = 0.8):
    """Step 2 of the rundown (Eq. inverse_weights2): returns (m, w, B_eff)."""
    msa = _as_input(msa, np.int8)
    B, N = msa.shape
    m = _like(msa, (B,), np.int32)
    w = _like(msa, (B,), np.float32)
    beff = ctypes.c_double()
    ctx.check(ctx.lib.msa_reweight(ctx.handle, _ptr(msa), B, N, Q, float(x),
                                   _ptr(m), _ptr(w), ctypes.byref(beff)))
    return m, w, beff.value


def plm_site_objective_grad(ctx: Context, msa, w, beff: float, h, J,
                            lambda_h: float = 0.01, lambda_J: float = 0.01,
                            prec: str = "fp32", grad: bool = True):
    """Objective g_r^(reg) (Eq. g_regdef2) of every site and its gradient
    (Eqs. g_gradh2, g_gradJ2) at (h, J); returns (f[N], gh[N,q], gJ[N,q,N,q]),
    or (f, None, None) with grad=False (the gradient contraction skipped)."""
    msa = _as_input(msa, np.int8)
    B, N = msa.shape
    w = _as_input(w, np.float32)
    h = _as_input(h, np.float32)
    J = _as_input(J, np.float32)
    f = _like(msa, (N,), np.float64)
    gh = _like(msa, (N, Q), np.float32) if grad else None
    gJ = _like(msa, (N, Q, N, Q), np.float32) if grad else None
    ctx.check(ctx.lib.plm_site_objective_grad(
        ctx.handle, _ptr(msa), _ptr(w), float(beff), B, N, Q, _ptr(h), _ptr(J),
        float(lambda_h), float(lambda_J), N_.PRECISIONS[prec], _ptr(f),
        _ptr(gh) if grad else None, _ptr(gJ) if grad else None))
    return f, gh, gJ


def default_opts(**kw) -> N_.plm_opts:
    o = N_.plm_opts()
    N_.load().plm_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = N_.PRECISIONS[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def plm_solve(ctx: Context, msa, raise_on_notconv: bool = False, **opts):
    """Steps 1-3 of the rundown: reweighting and the batched per-site L-BFGS.
    Returns (h[N,q], J[N,q,N,q], report dict incl. 'status')."""
    msa = _as_input(msa, np.int8)
    B, N = msa.shape
    o = default_opts(**opts)
    h = _like(msa, (N, Q), np.float32)
    J = _like(msa, (N, Q, N, Q), np.float32)
    rep = N_.plm_report()
    st = ctx.lib.plm_solve(ctx.handle, _ptr(msa), B, N, Q, ctypes.byref(o),
                           _ptr(h), _ptr(J), ctypes.byref(rep))
    if st != N_.PLM_OK and (st != N_.PLM_ENOTCONV or raise_on_notconv):
        ctx.check(st)
    d = rep.as_dict()
    d["status"] = N_.STATUS_NAMES.get(st, st)
    return h, J, d


def plm_solve_symmetric(ctx: Context, msa, raise_on_notconv: bool = False, **opts):
    """Symmetric plmDCA (Eq. npll_1 with the penalty of Eq. l2reg): one
    minimisation with a single coupling block per pair.  Returns (h[N,q],
    J[N,q,N,q] with J[j,:,i,:] = J[i,:,j,:]^T, report dict incl. 'status')."""
    msa = _as_input(msa, np.int8)
    B, N = msa.shape
    o = default_opts(**opts)
    h = _like(msa, (N, Q), np.float32)
    J = _like(msa, (N, Q, N, Q), np.float32)
    rep = N_.plm_report()
    st = ctx.lib.plm_solve_symmetric(ctx.handle, _ptr(msa), B, N, Q, ctypes.byref(o),
                                     _ptr(h), _ptr(J), ctypes.byref(rep))
    if st != N_.PLM_OK and (st != N_.PLM_ENOTCONV or raise_on_notconv):
        ctx.check(st)
    d = rep.as_dict()
    d["status"] = N_.STATUS_NAMES.get(st, st)
    return h, J, d


def plm_solve_batch(ctx: Context, msas, raise_on_notconv: bool = False, **opts):
    """plm_solve for many families at once (one batched L-BFGS, one launch
    per evaluation kernel for all families).  Returns a list of
    (h, J, report) per family."""
    msas = [_as_input(m, np.int8) for m in msas]
    o = default_opts(**opts)
    n = len(msas)
    fams = (N_.plm_family * n)()
    outs = []
    for k, m in enumerate(msas):
        B, N = m.shape
        h = _like(m, (N, Q), np.float32)
        J = _like(m, (N, Q, N, Q), np.float32)
        fams[k].msa = _ptr(m)
        fams[k].B = B
        fams[k].N = N
        fams[k].h_out = _ptr(h)
        fams[k].J_out = _ptr(J)
        outs.append((h, J))
    reps = (N_.plm_report * n)()
    st = ctx.lib.plm_solve_batch(ctx.handle, fams, n, Q, ctypes.byref(o), reps)
    if st != N_.PLM_OK and (st != N_.PLM_ENOTCONV or raise_on_notconv):
        ctx.check(st)
    res = []
    for k in range(n):
        d = reps[k].as_dict()
        d["status"] = N_.STATUS_NAMES.get(st, st)
        res.append((outs[k][0], outs[k][1], d))
    return res


def fn_apc_scores(ctx: Context, J, combine: str = "mean", L: int | None = None,
                  min_sep: int = 5):
    """Steps 4-6 of the rundown: returns (FN[N,N], CFN[N,N], top[L,2])."""
    J = _as_input(J, np.float32)
    N = J.shape[0]
    L = N if L is None else L
    fn = _like(J, (N, N), np.float64)
    cfn = _like(J, (N, N), np.float64)
    top = _like(J, (L, 2), np.int32)
    ctx.check(ctx.lib.fn_apc_scores(ctx.handle, _ptr(J), N, Q,
                                    {"mean": 0, "min": 1, "max": 2}[combine],
                                    _ptr(fn), _ptr(cfn), _ptr(top), L, min_sep))
    return fn, cfn, top


FORMATS = {"auto": 0, "fasta": 1, "a2m": 1, "stockholm": 2}


def msa_parse(text, fmt: str = "auto", ctx: Context | None = None) -> np.ndarray:
    """An aligned family (FASTA/A2M or Stockholm text, str or bytes) as the
    int8 MSA ``[B, N]``: insert states removed, 0 = gap, 1..20 = ACDEFGHIKLMNPQRSTVWY
    (host code; no GPU needed)."""
    lib = N_.load()
    data = text.encode() if isinstance(text, str) else bytes(text)
    B = ctypes.c_int()
    N = ctypes.c_int()
    h = ctx.handle if ctx is not None else None
    st = lib.msa_parse(h, data, len(data), FORMATS[fmt], None, 0, ctypes.byref(B), ctypes.byref(N))
    if st != N_.PLM_OK:
        if ctx is not None:
            ctx.check(st)
        raise N_.PlmError(st, "msa_parse failed")
    out = np.empty((B.value, N.value), np.int8)
    st = lib.msa_parse(h, data, len(data), FORMATS[fmt], out.ctypes.data_as(ctypes.c_void_p),
                       out.size, ctypes.byref(B), ctypes.byref(N))
    if st != N_.PLM_OK:
        raise N_.PlmError(st, "msa_parse failed")
    return out


def read_msa(path: str, fmt: str = "auto") -> np.ndarray:
    """msa_parse of a file."""
    with open(path, "rb") as fh:
        return msa_parse(fh.read(), fmt)


def msa_frequencies(ctx: Context, msa, w, beff: float):
    """Reweighted single-site frequencies f_i(k), ``[N, q]`` float64."""
    msa = _as_input(msa, np.int8)
    B, N = msa.shape
    w = _as_input(w, np.float32)
    f = _like(msa, (N, Q), np.float64)
    ctx.check(ctx.lib.msa_frequencies(ctx.handle, _ptr(msa), _ptr(w), float(beff), B, N, Q,
                                      _ptr(f)))
    return f


def plm_scores(ctx: Context, J, norm: str = "fro", p: float = 2.0, exclude_gap: bool = False,
               correction: str = "apc", combine: str = "mean", freq=None,
               L: int | None = None, min_sep: int = 5):
    """The Sec. 6 score alternatives: returns (score[N,N], corrected[N,N],
    top[L,2]).  ``norm`` in fro / lp / burkoff (needs ``freq`` from
    msa_frequencies), ``correction`` in apc / asc / none."""
    J = _as_input(J, np.float32)
    N = J.shape[0]
    L = N if L is None else L
    so = N_.plm_score_opts()
    ctx.lib.plm_default_score_opts(ctypes.byref(so))
    so.combine = {"mean": 0, "min": 1, "max": 2}[combine]
    so.norm = N_.NORMS[norm]
    so.p = float(p)
    so.exclude_gap = int(bool(exclude_gap))
    so.correction = N_.CORRECTIONS[correction]
    if freq is not None:
        if _is_torch(freq):
            freq = freq.to(_torch().float64).contiguous()
        else:
            freq = np.ascontiguousarray(freq, np.float64)
    sc = _like(J, (N, N), np.float64)
    co = _like(J, (N, N), np.float64)
    top = _like(J, (L, 2), np.int32)
    ctx.check(ctx.lib.plm_scores(ctx.handle, _ptr(J), N, Q, ctypes.byref(so), _ptr(freq),
                                 _ptr(sc), _ptr(co), _ptr(top), L, min_sep))
    return sc, co, top


def plmdca(ctx: Context, msa, L: int | None = None, min_sep: int = 5, out=None,
           raise_on_notconv: bool = False, **opts):
    """The whole rundown (steps 1-6) on the GPU in one library call
    (``plmdca_run``): the estimates stay on the device between the solve and
    the scores.  Outputs are allocated beside ``msa`` (CUDA tensors, or host
    arrays), or written into ``out`` (a dict with h, J, fn, cfn, top, e.g.
    pinned host tensors).  Returns dict(h, J, report, fn, cfn, top)."""
    msa = _as_input(msa, np.int8)
    B, N = msa.shape
    L = N if L is None else L
    o = default_opts(**opts)
    if out is None:
        out = dict(h=_like(msa, (N, Q), np.float32), J=_like(msa, (N, Q, N, Q), np.float32),
                   fn=_like(msa, (N, N), np.float64), cfn=_like(msa, (N, N), np.float64),
                   top=_like(msa, (L, 2), np.int32))
    rep = N_.plm_report()
    st = ctx.lib.plmdca_run(ctx.handle, _ptr(msa), B, N, Q, ctypes.byref(o), L, min_sep,
                            _ptr(out["h"]), _ptr(out["J"]), _ptr(out["fn"]), _ptr(out["cfn"]),
                            _ptr(out["top"]), ctypes.byref(rep))
    if st != N_.PLM_OK and (st != N_.PLM_ENOTCONV or raise_on_notconv):
        ctx.check(st)
    d = rep.as_dict()
    d["status"] = N_.STATUS_NAMES.get(st, st)
    return dict(h=out["h"], J=out["J"], report=d, fn=out["fn"], cfn=out["cfn"], top=out["top"])


def selftest_wait(ctx: Context):
    """Run the tensor-core pipelines' bounded wait on a barrier nothing
    arrives on (``plm_selftest_wait``, a diagnostic).  Returns (status name,
    timeout code); the expected outcome is ("PLM_ETIMEOUT", non-zero code)
    after about two seconds, with the context still usable."""
    code = ctypes.c_int(0)
    st = ctx.lib.plm_selftest_wait(ctx.handle, ctypes.byref(code))
    return N_.STATUS_NAMES.get(st, st), code.value
