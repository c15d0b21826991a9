"""The seeded input generators against published known answers.

The pattern generator on the device and ``gbs_inputs.philox4x32_10`` on the host
are checked bit for bit against each other by the GPU tests; a mistake both
share (a round-key constant, a multiplier, the order of the output words) would
pass that check.  The known-answer vectors published with Philox (Salmon,
Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11;
the ``kat_vectors`` file of the Random123 distribution) pin the host generator
itself, and through the bit-exact GPU comparison the device one too.
"""
import numpy as np

import gbs_inputs as g

# (counter words c0..c3, key words k0, k1) -> output words, Philox4x32 with 10 rounds
PHILOX4X32_10_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


def test_philox4x32_10_known_answers():
    for ctr, key, want in PHILOX4X32_10_KAT:
        got = g.philox4x32_10(np.array(ctr, dtype=np.uint64), key)
        assert [int(x) for x in got] == list(want)


def test_philox4x32_10_vectorised_matches_single():
    # a batch of counters gives, row by row, what each counter gives alone
    ctrs = np.array([k for k, _, _ in PHILOX4X32_10_KAT], dtype=np.uint64)
    key = (0x01234567, 0x89abcdef)
    batch = g.philox4x32_10(ctrs, key)
    for i in range(len(ctrs)):
        assert (batch[i] == g.philox4x32_10(ctrs[i], key)).all()


def test_philox_words_layout():
    # item i draws words from counters (i, block, stream, 0), four words per block in order
    seed, stream = 0x1122334455667788, 5
    w = g.philox_words(seed, stream, np.array([7]), 6)[0]
    key = (seed & 0xFFFFFFFF, seed >> 32)
    b0 = g.philox4x32_10(np.array([7, 0, stream, 0], dtype=np.uint64), key)
    b1 = g.philox4x32_10(np.array([7, 1, stream, 0], dtype=np.uint64), key)
    assert list(w) == list(b0) + list(b1[:2])
