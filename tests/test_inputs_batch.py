"""Seeded batch of independent shells (host side, no GPU)."""
import collections

from chorus_inputs import BATCH_64, _splitmix64_next, small_batch


def test_splitmix64_reference_output():
    # first output of SplitMix64 started from state 0 (Steele, Lea and Flood 2014 generator)
    assert _splitmix64_next(0)[1] == 0xE220A8397B1DCDAF


def test_batch_draws_are_seeded_and_in_range():
    a, b = BATCH_64.shells(), BATCH_64.shells()
    assert [(s.n, s.n_r, s.p, s.seed) for s in a] == [(s.n, s.n_r, s.p, s.seed) for s in b]
    assert len(a) == 64
    for i, s in enumerate(a):
        assert 8 <= s.n <= 32 and 4 <= s.n_r <= 16 and s.p in (2, 3, 4, 5)
        assert s.seed == 4 * 1000 + i
    counts = collections.Counter(s.p for s in a)
    assert set(counts) == {2, 3, 4, 5}
    assert len({(s.n, s.n_r) for s in a}) > 32  # uneven sizes


def test_small_batch_has_every_order():
    assert {s.p for s in small_batch().shells()} == {2, 3, 4, 5}
