"""Input generator checks (the generator holds none of the method's arithmetic)."""
import numpy as np

from paper_1401_4832_gb300 import synth


def test_philox_known_answers():
    # known-answer vectors of Philox-4x32-10 (Salmon et al., SC'11, Random123)
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
        ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
        ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
         [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
    ]
    for ctr, key, out in kat:
        assert synth.philox4x32_10(ctr, key).tolist() == out


def test_generator_is_seeded_and_shaped():
    a = synth.family(12, 50, 8, "random", 0.1, 20, seed=3, cache=False)
    b = synth.family(12, 50, 8, "random", 0.1, 20, seed=3, cache=False)
    c = synth.family(12, 50, 8, "random", 0.1, 20, seed=4, cache=False)
    assert a.msa.shape == (50, 12) and a.msa.dtype == np.int8
    assert np.array_equal(a.msa, b.msa) and not np.array_equal(a.msa, c.msa)
    assert a.msa.min() >= 0 and a.msa.max() < 21


def test_chain_contacts_respect_cutoff_and_separation():
    rng = synth._rng(0, 1)
    pairs = synth.chain_pairs(80, 120, rng)
    assert len(pairs) > 40
    assert np.all(pairs[:, 1] - pairs[:, 0] >= 4)
