"""The MSA front end: aligned FASTA/A2M and Stockholm text to the int8 MSA.

Insert states (lower-case letters, '.') are removed, as the paper does with
PFAM alignments before DCA (Sec. 4); match states map to 0 = gap ('-') and
1..20 = A C D E F G H I K L M N P Q R S T V W Y; O, U (appendix table) and
the ambiguity codes B, Z, X read as the gap.  The library's reader (C++,
through the C ABI; no GPU) must agree bit for bit with the oracle's plain
Python reader and with the hand-worked golden files.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1401_4832_gb300 import api, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
A = {c: 1 + i for i, c in enumerate("ACDEFGHIKLMNPQRSTVWY")}

# tests/golden/msa_small.a2m worked by hand
EXPECTED = np.array([
    [A["A"], A["C"], 0, A["D"], A["E"]],
    [A["W"], 0, A["Y"], A["Y"], A["K"]],
    [0, 0, 0, 0, 0],
    [A["M"], A["N"], A["P"], A["Q"], A["R"]],
], np.int8)


def test_golden_fasta():
    got = api.read_msa(os.path.join(GOLDEN, "msa_small.a2m"))
    assert np.array_equal(got, EXPECTED)
    text = open(os.path.join(GOLDEN, "msa_small.a2m")).read()
    assert np.array_equal(oracle.parse_msa(text), EXPECTED)


def test_golden_stockholm_interleaved_blocks():
    # the same four sequences in two blocks, with annotation lines
    path = os.path.join(GOLDEN, "msa_small.sto")
    assert np.array_equal(api.read_msa(path), EXPECTED)
    assert np.array_equal(oracle.parse_msa(open(path).read()), EXPECTED)


def _to_a2m(S, rng, insert_p=0.1):
    inv = "-" + "ACDEFGHIKLMNPQRSTVWY"
    lines = []
    for b, row in enumerate(S):
        chars = []
        for st in row:
            chars.append(inv[st])
            if rng.random() < insert_p:  # an insert state after this column
                chars.append(rng.choice(list("acdefghiklmnpqrstvwy.")))
        lines.append(f">s{b} random header {rng.integers(1000)}")
        text = "".join(chars)
        lines.extend(text[k:k + 60] for k in range(0, len(text), 60))
    return "\n".join(lines) + "\n"


def test_round_trip_of_a_synthetic_family_with_inserts():
    rng = np.random.default_rng(1)
    S = synth.small_random(57, 300, 3, gap_p=0.2)
    text = _to_a2m(S, rng)
    assert np.array_equal(api.msa_parse(text), S)
    assert np.array_equal(oracle.parse_msa(text), S)
    sto = "# STOCKHOLM 1.0\n" + "\n".join(
        f"s{b} " + "".join("-ACDEFGHIKLMNPQRSTVWY"[x] for x in row) for b, row in enumerate(S)) + "\n//\n"
    assert np.array_equal(api.msa_parse(sto), S)


@pytest.mark.parametrize("text", [
    "",                                   # no sequences
    ">a\nACD\n>b\nAC\n",                  # different numbers of match columns
    ">a\nAC1D\n",                         # not an alignment character
    "ACD\n>a\nACD\n",                     # data before the first header
    ">a\n...\n",                          # no match columns
])
def test_malformed_input_is_rejected(text):
    from paper_1401_4832_gb300 import _native
    with pytest.raises(_native.PlmError):
        api.msa_parse(text)
    with pytest.raises(ValueError):
        oracle.parse_msa(text)
