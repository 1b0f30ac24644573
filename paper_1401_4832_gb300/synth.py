"""Seeded synthetic Potts-model MSAs shaped like protein families.

Input generator shared by the CUDA library's tests and benchmark and by the
CPU oracle's tests.  It holds none of the inference method's arithmetic: it
builds a planted sparse Potts model, draws sequences from it with a Gibbs
sampler (``synth_gibbs.c``), and adds gaps.  Protein-family alignments
(PFAM) and structures (PDB) are not available, so these stand in for them
with the shapes the paper describes: N of about 50-500 positions, B from
hundreds to tens of thousands of sequences, q = 21 states with state 0 the
gap (Sec. 2 and Sec. 4).

Recipe (all draws seeded; parameters of one call fully determine the MSA):
  * fields h_i(s) ~ N(0, 1);
  * planted pairs get a q x q block J_ij(k, l) ~ N(0, 0.25) (variance 0.25),
    with J_ji = J_ij^T; all other blocks are zero;
  * contact map: ``"random"`` = uniform distinct pairs i<j; ``"chain"`` = a
    3D-like chain: a random walk of 3.8 A steps whose direction turns by a
    bounded random angle, kept inside a sphere of radius 2.2 N^(1/3) 3.8 A by
    rejection; pairs with j - i >= 4 and C-alpha distance < 8.5 A (the
    paper's contact cut-off, Sec. 4) are candidates, and ceil(1.5 N) of them
    are drawn without replacement;
  * Gibbs sampling: B independent chains from uniform random starts,
    ``sweeps`` systematic sweeps each (counter-based Philox random numbers);
  * gaps: each entry is then set to state 0 with probability ``gap_p``;
  * optional "clustered" rows: a fraction of rows replaced by copies of
    random rows with 0-25 % of their positions redrawn uniformly, so that the
    0.8-identity reweighting has non-trivial weights.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

Q = 21
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_gibbs.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_CACHE = os.path.join(os.path.dirname(_HERE), "_cache", "synth")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.synth_gibbs.argtypes = [I, I, I, I, ctypes.c_uint32, P, P, P, P, P]
            lib.synth_gibbs.restype = I
            lib.synth_philox4x32_10.argtypes = [P, P, P]
            lib.synth_philox4x32_10.restype = None
            _lib = lib
    return _lib


def philox4x32_10(ctr, key):
    """Philox-4x32-10 block function (exposed for a known-answer test)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().synth_philox4x32_10(c.ctypes.data_as(ctypes.c_void_p),
                                k.ctypes.data_as(ctypes.c_void_p),
                                out.ctypes.data_as(ctypes.c_void_p))
    return out


@dataclass
class PlantedModel:
    h: np.ndarray                 # [N, q]
    pairs: np.ndarray             # [P, 2] int, i < j
    blocks: np.ndarray            # [P, q, q], J_ij(k, l) with k at i
    N: int = field(init=False)

    def __post_init__(self):
        self.N = self.h.shape[0]

    def dense_J(self) -> np.ndarray:
        """Symmetric dense couplings ``J[i, k, j, l]`` of the planted model."""
        N, q = self.h.shape
        J = np.zeros((N, q, N, q))
        for (i, j), blk in zip(self.pairs, self.blocks):
            J[i, :, j, :] = blk
            J[j, :, i, :] = blk.T
        return J


def _rng(*key) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence(list(key))))


def random_pairs(N: int, npairs: int, rng) -> np.ndarray:
    all_pairs = np.array([(i, j) for i in range(N) for j in range(i + 1, N)], np.int64)
    npairs = min(npairs, len(all_pairs))
    sel = rng.choice(len(all_pairs), size=npairs, replace=False)
    return all_pairs[np.sort(sel)]


def chain_coords(N: int, rng, step=3.8, max_turn_deg=60.0) -> np.ndarray:
    """Random 3D chain with bounded turn angles, confined to a sphere."""
    R = 2.2 * N ** (1.0 / 3.0) * step
    x = np.zeros((N, 3))
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    cos_max = math.cos(math.radians(max_turn_deg))
    for t in range(1, N):
        for _ in range(1000):
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            if v @ d < cos_max:
                continue
            p = x[t - 1] + step * v
            if np.linalg.norm(p) <= R:
                break
        else:  # stuck at the wall: step straight towards the centre
            v = -x[t - 1] / max(np.linalg.norm(x[t - 1]), 1e-12)
            p = x[t - 1] + step * v
        x[t] = p
        d = v
    return x


def chain_pairs(N: int, npairs: int, rng, cutoff=8.5, min_sep=4) -> np.ndarray:
    x = chain_coords(N, rng)
    dist = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=-1)
    cand = np.array([(i, j) for i in range(N) for j in range(i + min_sep, N)
                     if dist[i, j] < cutoff], np.int64).reshape(-1, 2)
    if len(cand) <= npairs:
        return cand
    sel = rng.choice(len(cand), size=npairs, replace=False)
    return cand[np.sort(sel)]


def planted_model(N: int, npairs: int, contacts: str, seed: int, q: int = Q,
                  j_var: float = 0.25) -> PlantedModel:
    rng = _rng(seed, N, 1)
    h = rng.normal(0.0, 1.0, size=(N, q))
    if contacts == "random":
        pairs = random_pairs(N, npairs, rng)
    elif contacts == "chain":
        pairs = chain_pairs(N, npairs, rng)
    else:
        raise ValueError(contacts)
    blocks = rng.normal(0.0, math.sqrt(j_var), size=(len(pairs), q, q))
    return PlantedModel(h=h, pairs=pairs, blocks=blocks)


def gibbs_sample(model: PlantedModel, B: int, sweeps: int, seed: int) -> np.ndarray:
    N, q = model.h.shape
    # CSR neighbour lists, each edge carrying its block oriented [s_i][s_j]
    edges = [[] for _ in range(N)]
    for (i, j), blk in zip(model.pairs, model.blocks):
        edges[i].append((j, blk))
        edges[j].append((i, blk.T))
    ptr = np.zeros(N + 1, np.int32)
    idx, blks = [], []
    for i in range(N):
        ptr[i + 1] = ptr[i] + len(edges[i])
        for j, blk in edges[i]:
            idx.append(j)
            blks.append(blk)
    idx = np.array(idx if idx else [0], np.int32)
    blks = np.ascontiguousarray(np.array(blks) if blks else np.zeros((1, q, q)))
    h = np.ascontiguousarray(model.h, np.float64)
    out = np.zeros((B, N), np.int8)
    vp = ctypes.c_void_p
    rc = _load().synth_gibbs(N, q, B, sweeps, ctypes.c_uint32(seed & 0xFFFFFFFF),
                             h.ctypes.data_as(vp), ptr.ctypes.data_as(vp),
                             idx.ctypes.data_as(vp), blks.ctypes.data_as(vp),
                             out.ctypes.data_as(vp))
    if rc != 0:
        raise RuntimeError("synth_gibbs failed")
    return out


def add_gaps(S: np.ndarray, p: float, seed: int) -> np.ndarray:
    if p <= 0:
        return S
    rng = _rng(seed, 7)
    S = S.copy()
    S[rng.random(S.shape) < p] = 0
    return S


def add_clusters(S: np.ndarray, frac: float, seed: int, q: int = Q,
                 max_redraw: float = 0.25) -> np.ndarray:
    """Replace a fraction of rows by near-copies of random rows."""
    rng = _rng(seed, 11)
    S = S.copy()
    B, N = S.shape
    nrep = int(round(frac * B))
    rows = rng.choice(B, size=nrep, replace=False)
    for r in rows:
        src = rng.integers(0, B)
        row = S[src].copy()
        nre = int(rng.integers(0, int(max_redraw * N) + 1))
        pos = rng.choice(N, size=nre, replace=False)
        row[pos] = rng.integers(0, q, size=nre)
        S[r] = row
    return S


@dataclass
class Family:
    name: str
    msa: np.ndarray               # int8 [B, N]
    model: PlantedModel

    @property
    def B(self):
        return self.msa.shape[0]

    @property
    def N(self):
        return self.msa.shape[1]


def family(N: int, B: int, npairs: int, contacts: str = "chain", gap_p: float = 0.15,
           sweeps: int = 1000, seed: int = 0, clustered: float = 0.0,
           cache: bool = True, name: str | None = None) -> Family:
    """One synthetic family; cached on disk under ``_cache/synth`` keyed by
    every parameter."""
    key = f"N{N}_B{B}_P{npairs}_{contacts}_g{gap_p}_s{sweeps}_seed{seed}_c{clustered}"
    name = name or key
    model = planted_model(N, npairs, contacts, seed)
    path = os.path.join(_CACHE, hashlib.sha1(key.encode()).hexdigest()[:16] + ".npy")
    if cache and os.path.exists(path):
        msa = np.load(path)
        if msa.shape == (B, N) and msa.dtype == np.int8:
            return Family(name, msa, model)
    msa = gibbs_sample(model, B, sweeps, seed=(seed * 7919 + 17) & 0xFFFFFFFF)
    msa = add_gaps(msa, gap_p, seed)
    if clustered > 0:
        msa = add_clusters(msa, clustered, seed)
    msa = np.ascontiguousarray(msa, np.int8)
    if cache:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npy"
        np.save(tmp, msa)
        os.replace(tmp, path)
    return Family(name, msa, model)


# ---------------------------------------------------------------------------
# The named workloads
# ---------------------------------------------------------------------------
def tiny(seed: int = 0, **kw) -> Family:
    """N=20, B=300, 30 random planted pairs, no gaps, 1000 sweeps."""
    return family(20, 300, 30, "random", 0.0, 1000, seed, name="tiny N=20 B=300", **kw)


def protein_family(seed: int = 0, **kw) -> Family:
    """N=120, B=5000, ceil(1.5N)=180 pairs from a 3D-like chain, 15 % gaps,
    1000 sweeps."""
    return family(120, 5000, 180, "chain", 0.15, 1000, seed,
                  name="family N=120 B=5000", **kw)


def scale_family(seed: int = 0, sweeps: int = 100, **kw) -> Family:
    """N=500, B=50000, 750 pairs from a 3D-like chain, 20 % gaps."""
    return family(500, 50000, 750, "chain", 0.20, sweeps, seed,
                  name="scale N=500 B=50000", **kw)


def batch_families(count: int = 64, sweeps: int = 100, **kw) -> list[Family]:
    """``count`` families, family f seeded with f: N ~ U{50..300},
    B = round(exp(U(ln 500, ln 20000))), ceil(1.5 N) chain pairs, 15 % gaps."""
    fams = []
    for f in range(count):
        rng = _rng(f, 99)
        N = int(rng.integers(50, 301))
        B = int(round(math.exp(rng.uniform(math.log(500), math.log(20000)))))
        fams.append(family(N, B, int(math.ceil(1.5 * N)), "chain", 0.15, sweeps, f,
                           name=f"batch{f} N={N} B={B}", **kw))
    return fams


def small_random(N: int, B: int, seed: int, q: int = Q, gap_p: float = 0.1) -> np.ndarray:
    """Uniform random MSA (no model) for edge-case tests."""
    rng = _rng(seed, N, B, 3)
    S = rng.integers(0, q, size=(B, N)).astype(np.int8)
    return add_gaps(S, gap_p, seed)
