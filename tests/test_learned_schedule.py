"""The wavefront order of the learned proposal's sampler, checked against the
network's own masks (oracle/learned.py): the sampler takes the positions of
a 10 x 10 window in steps s = c + 2r and keeps the layer activations of the
last four steps in rings.  That is exact only if every input of position
(r, c) -- the interior spins its layer-1 features read (mask A), the
activations its mask-B taps read at layers 2-4 -- belongs to an earlier step
(the (0, 0) tap excepted, which is the position itself), and every ring tap
reaches one to three steps back.  Also the step sizes: at most five
positions (the rows of three windows fit one m16 tile), 100 in all."""
from __future__ import annotations

from oracle import learned as ol

S = 10


def _step(r, c):
    return c + 2 * r


def _inside(r, c):
    return 0 <= r < S and 0 <= c < S


def test_interior_spins_read_by_layer_1_come_from_earlier_steps():
    inner = ol.interior_mask(S)
    for r in range(S):
        for c in range(S):
            for dy, dx in ol.MASK_A:
                y, x = r + dy, c + dx
                if _inside(y, x) and inner[y, x]:          # a sampled spin
                    assert _step(y, x) < _step(r, c), ((r, c), (dy, dx))


def test_mask_b_taps_reach_one_to_three_steps_back():
    for r in range(S):
        for c in range(S):
            for dy, dx in ol.MASK_B:
                y, x = r + dy, c + dx
                if not _inside(y, x):
                    continue
                d = _step(r, c) - _step(y, x)
                if (dy, dx) == (0, 0):
                    assert d == 0
                else:
                    assert 1 <= d <= 3, ((r, c), (dy, dx), d)


def test_step_sizes():
    counts = [0] * (3 * S - 2)
    for r in range(S):
        for c in range(S):
            counts[_step(r, c)] += 1
    assert sum(counts) == S * S and max(counts) == 5 and min(counts) == 1
    # the first row of step s and its count, as the sampler's tables compute them
    for s, n in enumerate(counts):
        rmin = (s - 8) // 2 if s >= 9 else 0
        rmax = min(S - 1, s // 2)
        assert rmax - rmin + 1 == n
        for r in range(rmin, rmax + 1):
            assert 0 <= s - 2 * r < S
