"""FP64 CPU oracle for asymmetric plmDCA -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it
and shares no code with it; the C source (``plm_oracle.c``) writes each step
of the paper's rundown (Sec. 3.5, steps 1-6) out plainly in double
precision.  This module compiles that file with gcc and exposes it through
ctypes on numpy arrays.

Layouts (unpadded, q = 21): MSA int8 ``[B, N]``; fields ``h[N, q]``;
couplings ``J[N, q, N, q]`` with ``J[r, s, i, k] = J^r_{ri}(s, k)`` (the
estimate from site r's problem, first state index at r).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 21


def build(force: bool = False) -> str:
    """Compile ``plm_oracle.c`` into ``_build/liboracle.so`` (portable flags:
    the same source builds on x86_64 and aarch64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # ORACLE_LIB lets the mutation test load a deliberately broken copy
        lib = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.orc_num_threads.restype = I
        lib.orc_set_threads.argtypes = [I]
        lib.orc_set_threads.restype = None
        lib.orc_identity_threshold.argtypes = [D, I]
        lib.orc_identity_threshold.restype = I
        lib.orc_reweight.argtypes = [P, I, I, I, P, P, P, P]
        lib.orc_reweight.restype = None
        lib.orc_site_objgrad.argtypes = [P, P, D, I, I, I, I, P, P, D, D, P, P]
        lib.orc_site_objgrad.restype = D
        lib.orc_objgrad_all.argtypes = [P, P, D, I, I, I, P, P, D, D, P, P, P]
        lib.orc_objgrad_all.restype = None
        lib.orc_solve_sites.argtypes = [P, P, D, I, I, I, D, D, D, I, I, P, I,
                                        P, P, P, P, P, P, P]
        lib.orc_solve_sites.restype = None
        lib.orc_ising_gauge_block.argtypes = [P, I, P]
        lib.orc_ising_gauge_block.restype = None
        lib.orc_scores.argtypes = [P, I, I, I, P, P]
        lib.orc_scores.restype = None
        lib.orc_fn.argtypes = [P, I, I, I, P]
        lib.orc_fn.restype = None
        lib.orc_apc.argtypes = [P, I, P]
        lib.orc_apc.restype = None
        lib.orc_topL.argtypes = [P, I, I, I, P]
        lib.orc_topL.restype = I
        lib.orc_site_freqs.argtypes = [P, P, D, I, I, I, P]
        lib.orc_site_freqs.restype = None
        lib.orc_score_matrix.argtypes = [P, I, I, I, I, D, I, P, P]
        lib.orc_score_matrix.restype = None
        lib.orc_asc.argtypes = [P, I, P]
        lib.orc_asc.restype = None
        lib.orc_sym_nparams.argtypes = [I, I]
        lib.orc_sym_nparams.restype = ctypes.c_size_t
        lib.orc_sym_expand.argtypes = [P, I, I, P, P]
        lib.orc_sym_expand.restype = None
        lib.orc_sym_objgrad.argtypes = [P, P, D, I, I, I, P, D, D, P]
        lib.orc_sym_objgrad.restype = D
        lib.orc_solve_symmetric.argtypes = [P, P, D, I, I, I, D, D, D, I, I, P, P, P, P, P]
        lib.orc_solve_symmetric.restype = I
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _msa(S) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.int8)
    assert S.ndim == 2
    return S


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    """Thread count of the oracle's OpenMP loops over sites (timing only)."""
    _load().orc_set_threads(int(n))


def identity_threshold(x: float, N: int) -> int:
    """Smallest integer match count T with T / N >= x (reading of Eq.
    inverse_weights: similar means similarity >= x)."""
    return _load().orc_identity_threshold(float(x), int(N))


def reweight(S, x: float = 0.8):
    """Step 2 of the rundown (Eq. inverse_weights2).

    Returns ``(m int32[B], w float64[B], w32 float32[B], B_eff float)`` with
    ``w = 1/m`` and ``B_eff = sum_b w_b``.
    """
    S = _msa(S)
    B, N = S.shape
    T = identity_threshold(x, N)
    m = np.zeros(B, np.int32)
    w = np.zeros(B, np.float64)
    w32 = np.zeros(B, np.float32)
    beff = ctypes.c_double(0.0)
    _load().orc_reweight(_ptr(S), B, N, T, _ptr(m), _ptr(w), _ptr(w32),
                         ctypes.byref(beff))
    return m, w, w32, beff.value


def site_objgrad(S, w, beff, r, h_r, J_r, lambda_h, lambda_Jp, grad=True):
    """Objective g_r^(reg) (Eq. g_regdef2) and gradient (Eqs. g_gradh2,
    g_gradJ2) of one site.  ``lambda_Jp`` is lambda'_J (already halved).
    ``h_r`` is [q], ``J_r`` is [q, N, q]."""
    S = _msa(S)
    B, N = S.shape
    w = np.ascontiguousarray(w, np.float64)
    h_r = np.ascontiguousarray(h_r, np.float64)
    J_r = np.ascontiguousarray(J_r, np.float64)
    q = h_r.shape[0]
    assert J_r.shape == (q, N, q)
    gh = np.zeros(q) if grad else None
    gJ = np.zeros((q, N, q)) if grad else None
    f = _load().orc_site_objgrad(_ptr(S), _ptr(w), float(beff), B, N, q, int(r),
                                 _ptr(h_r), _ptr(J_r), float(lambda_h),
                                 float(lambda_Jp),
                                 _ptr(gh) if grad else None,
                                 _ptr(gJ) if grad else None)
    return (f, gh, gJ) if grad else f


def objgrad(S, w, beff, h, J, lambda_h=0.01, lambda_J=0.01, grad=True):
    """All sites at one parameter point: ``f[N]``, ``gh[N, q]``,
    ``gJ[N, q, N, q]``.  ``lambda_J`` is the user's strength; it is halved
    inside (step 1 of the rundown)."""
    S = _msa(S)
    B, N = S.shape
    w = np.ascontiguousarray(w, np.float64)
    h = np.ascontiguousarray(h, np.float64)
    J = np.ascontiguousarray(J, np.float64)
    q = h.shape[1]
    assert h.shape == (N, q) and J.shape == (N, q, N, q)
    f = np.zeros(N)
    gh = np.zeros((N, q)) if grad else None
    gJ = np.zeros((N, q, N, q)) if grad else None
    _load().orc_objgrad_all(_ptr(S), _ptr(w), float(beff), B, N, q, _ptr(h),
                            _ptr(J), float(lambda_h), float(lambda_J), _ptr(f),
                            _ptr(gh) if grad else None,
                            _ptr(gJ) if grad else None)
    return (f, gh, gJ) if grad else f


def solve(S, w, beff, lambda_h=0.01, lambda_J=0.01, gtol=1e-9, m=5,
          max_iter=5000, sites=None, q=Q):
    """Step 3 of the rundown: minimise every g_r^(reg) from the origin with
    L-BFGS (memory m, strong-Wolfe line search).  With ``sites`` given, only
    those site problems are solved (their rows of h and J are filled; the
    others stay zero).

    Returns ``(h[N,q], J[N,q,N,q], info)``; ``info`` holds per-site arrays
    ``iters, status, f, gnorm, nevals`` (in the order of ``sites``).
    """
    S = _msa(S)
    B, N = S.shape
    w = np.ascontiguousarray(w, np.float64)
    h = np.zeros((N, q))
    J = np.zeros((N, q, N, q))
    if sites is None:
        site_arr = None
        count = N
    else:
        site_arr = np.ascontiguousarray(sites, np.int32)
        count = site_arr.shape[0]
    iters = np.zeros(count, np.int32)
    status = np.zeros(count, np.int32)
    f = np.zeros(count)
    gnorm = np.zeros(count)
    nevals = np.zeros(count, np.int32)
    _load().orc_solve_sites(_ptr(S), _ptr(w), float(beff), B, N, q,
                            float(lambda_h), float(lambda_J), float(gtol),
                            int(m), int(max_iter),
                            _ptr(site_arr) if site_arr is not None else None,
                            count, _ptr(h), _ptr(J), _ptr(iters), _ptr(status),
                            _ptr(f), _ptr(gnorm), _ptr(nevals))
    info = dict(iters=iters, status=status, f=f, gnorm=gnorm, nevals=nevals)
    return h, J, info


def ising_gauge_block(Jb):
    """Step 4 (Eq. gauge_change2) on one q x q block."""
    Jb = np.ascontiguousarray(Jb, np.float64)
    q = Jb.shape[0]
    out = np.zeros_like(Jb)
    _load().orc_ising_gauge_block(_ptr(Jb), q, _ptr(out))
    return out


COMBINE = {"mean": 0, "min": 1, "max": 2}


def scores(J, combine="mean"):
    """Steps 4-6: Ising gauge, combination of the two estimates (Eq.
    average2; min/max are the Sec. 6 alternatives), Frobenius norm (Eq.
    frob_normtrans2) and APC (Eq. corr_norm2).  Returns ``(FN, CFN)``, both
    ``[N, N]``."""
    J = np.ascontiguousarray(J, np.float64)
    N, q = J.shape[0], J.shape[1]
    fn = np.zeros((N, N))
    cfn = np.zeros((N, N))
    _load().orc_scores(_ptr(J), N, q, COMBINE[combine], _ptr(fn), _ptr(cfn))
    return fn, cfn


def apc(fn):
    """Eq. corr_norm2 on a given FN matrix (off-diagonal position means)."""
    fn = np.ascontiguousarray(fn, np.float64)
    N = fn.shape[0]
    cfn = np.zeros((N, N))
    _load().orc_apc(_ptr(fn), N, _ptr(cfn))
    return cfn


def site_freqs(S, w, beff, q=Q):
    """Reweighted single-site frequencies f_i(k), ``[N, q]``."""
    S = _msa(S)
    B, N = S.shape
    w = np.ascontiguousarray(w, np.float64)
    f = np.zeros((N, q))
    _load().orc_site_freqs(_ptr(S), _ptr(w), float(beff), B, N, q, _ptr(f))
    return f


SCORE_KINDS = {"fro": 0, "lp": 1, "burkoff": 2}


def score_matrix(J, kind="fro", p=2.0, exclude_gap=False, freq=None, combine="mean"):
    """Sec. 6 score alternatives on the combined Ising-gauged blocks:
    Frobenius, general l_p norm, Burkoff's D_ij (needs ``freq`` [N, q]);
    ``exclude_gap`` leaves state 0 out of the norm sums."""
    J = np.ascontiguousarray(J, np.float64)
    N, q = J.shape[0], J.shape[1]
    out = np.zeros((N, N))
    fr = None if freq is None else np.ascontiguousarray(freq, np.float64)
    _load().orc_score_matrix(_ptr(J), N, q, COMBINE[combine], SCORE_KINDS[kind], float(p),
                             int(bool(exclude_gap)), _ptr(fr) if fr is not None else None,
                             _ptr(out))
    return out


def asc(fn):
    """Average sum correction (Eq. corr_normsum)."""
    fn = np.ascontiguousarray(fn, np.float64)
    N = fn.shape[0]
    out = np.zeros((N, N))
    _load().orc_asc(_ptr(fn), N, _ptr(out))
    return out


def topL(score, L, min_sep=5):
    """Pairs i<j with j-i >= min_sep, by score descending, ties (i, j)
    ascending; ``int32[L', 2]`` with L' = min(L, #eligible)."""
    score = np.ascontiguousarray(score, np.float64)
    N = score.shape[0]
    ij = np.zeros((max(L, 0), 2), np.int32)
    n = _load().orc_topL(_ptr(score), N, int(L), int(min_sep), _ptr(ij))
    return ij[:n]


def plmdca(S, x=0.8, lambda_h=0.01, lambda_J=0.01, gtol=1e-9, m=5,
           max_iter=5000, L=None, min_sep=5):
    """The whole rundown (steps 1-6): returns a dict with the weights, the
    asymmetric estimates, FN, CFN and the top-L list (L = N by default)."""
    S = _msa(S)
    B, N = S.shape
    mcount, w, w32, beff = reweight(S, x)
    h, J, info = solve(S, w, beff, lambda_h, lambda_J, gtol, m, max_iter)
    fn, cfn = scores(J)
    top = topL(cfn, N if L is None else L, min_sep)
    return dict(m=mcount, w=w, w32=w32, beff=beff, h=h, J=J, info=info,
                fn=fn, cfn=cfn, top=top)


# ---------------------------------------------------------------- symmetric
def sym_nparams(N, q=Q):
    """Parameters of the symmetric problem: N q fields + one q x q block per
    pair i < j (Sec. 6: N q (1 + (N - 1) q / 2))."""
    return int(_load().orc_sym_nparams(N, q))


def sym_expand(x, N, q=Q):
    """x = [h | J_ij (i < j, pair order (0,1), (0,2), ...)] -> per-site
    layout (h[N,q], J[N,q,N,q]) with J[j,l,i,k] = J[i,k,j,l] (both copies)."""
    x = np.ascontiguousarray(x, np.float64)
    h = np.zeros((N, q))
    J = np.zeros((N, q, N, q))
    _load().orc_sym_expand(_ptr(x), N, q, _ptr(h), _ptr(J))
    return h, J


def sym_objgrad(S, w, beff, x, lambda_h=0.01, lambda_J=0.01, grad=True, q=Q):
    """l_pseudo + R_l2 (Eqs. npll_1, l2reg) at x and its gradient in x."""
    S = _msa(S)
    B, N = S.shape
    w = np.ascontiguousarray(w, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    g = np.zeros_like(x) if grad else None
    f = _load().orc_sym_objgrad(_ptr(S), _ptr(w), float(beff), B, N, q, _ptr(x),
                                float(lambda_h), float(lambda_J),
                                _ptr(g) if grad else None)
    return (f, g) if grad else f


def solve_symmetric(S, w, beff, lambda_h=0.01, lambda_J=0.01, gtol=1e-7, m=5,
                    max_iter=20000, q=Q):
    """Symmetric plmDCA (Eq. npll_1 + Eq. l2reg) from the origin by the same
    L-BFGS as the site problems.  Returns ``(h, J, info)`` with J in the
    per-site layout (both copies of every block) and info = dict(iters,
    status, f, gnorm, nevals)."""
    S = _msa(S)
    B, N = S.shape
    w = np.ascontiguousarray(w, np.float64)
    x = np.zeros(sym_nparams(N, q))
    f = ctypes.c_double()
    gn = ctypes.c_double()
    ne = ctypes.c_int()
    st = ctypes.c_int()
    it = _load().orc_solve_symmetric(_ptr(S), _ptr(w), float(beff), B, N, q,
                                     float(lambda_h), float(lambda_J), float(gtol),
                                     int(m), int(max_iter), _ptr(x), ctypes.byref(f),
                                     ctypes.byref(gn), ctypes.byref(ne), ctypes.byref(st))
    h, J = sym_expand(x, N, q)
    return h, J, dict(iters=it, status=st.value, f=f.value, gnorm=gn.value,
                      nevals=ne.value, x=x)


def plmdca_symmetric(S, x=0.8, lambda_h=0.01, lambda_J=0.01, gtol=1e-7, m=5,
                     max_iter=20000, L=None, min_sep=5):
    """Reweighting, the symmetric minimisation and the same scoring (the
    two estimates of a block coincide, so the average is the block)."""
    S = _msa(S)
    B, N = S.shape
    mcount, w, w32, beff = reweight(S, x)
    h, J, info = solve_symmetric(S, w, beff, lambda_h, lambda_J, gtol, m, max_iter)
    fn, cfn = scores(J)
    top = topL(cfn, N if L is None else L, min_sep)
    return dict(m=mcount, w=w, w32=w32, beff=beff, h=h, J=J, info=info,
                fn=fn, cfn=cfn, top=top)


# ---------------------------------------------------------------- MSA text
ALPHABET = "ACDEFGHIKLMNPQRSTVWY"  # states 1..20; 0 is the gap


def _state(c):
    # Sec. 4: PFAM marks insert states with lower-case letters and '.',
    # removed before DCA; '-' is a deletion (the gap state).  Reading of the
    # appendix table: O, U and the ambiguity codes B, Z, X become the gap.
    if c == "-" or c in "OUBZX":
        return 0
    if c == "." or c.islower():
        return None
    if c in ALPHABET:
        return 1 + ALPHABET.index(c)
    raise ValueError(f"unexpected character {c!r}")


def parse_msa(text, fmt="auto"):
    """Aligned FASTA/A2M or Stockholm text -> int8 MSA [B, N] (plain Python)."""
    lines = text.splitlines()
    if fmt == "auto":
        first = next((ln for ln in lines if ln.strip()), "")
        fmt = "stockholm" if first.startswith("# STOCKHOLM") else "fasta"
    seqs = []
    if fmt == "fasta":
        for ln in lines:
            if ln.startswith(">"):
                seqs.append([])
            elif ln.strip():
                if not seqs:
                    raise ValueError("sequence data before the first header")
                seqs[-1].extend(ch for ch in ln if not ch.isspace())
    else:
        order, rows = [], {}
        for ln in lines:
            t = ln.strip()
            if not t or t.startswith("#"):
                continue
            if t.startswith("//"):
                break
            name, _, rest = t.partition(" ")
            if name not in rows:
                rows[name] = []
                order.append(name)
            rows[name].extend(ch for ch in rest if not ch.isspace())
        seqs = [rows[n] for n in order]
    out = [[st for st in (_state(c) for c in s) if st is not None] for s in seqs]
    if not out or any(len(r) != len(out[0]) for r in out) or not out[0]:
        raise ValueError("sequences differ in match columns, or none")
    return np.array(out, dtype=np.int8)
