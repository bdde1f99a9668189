"""Host model of the single-atomic HQ colour protocol (Sec. 3.5.1, "HQS1R")
as the colour kernel runs it, checked under random interleavings.

The kernel packs r << 50 | g << 36 | b << 22 | count (14, 14, 14, 22 bits)
into one 64-bit word per pixel.  Each adder (one point, or a warp group of up
to 32 same-pixel points) does one atomic add of its packed sums and reads the
word's old value.  Let c be the old count and k the adder's count:

- c + k <= 64: the add stays in the word;
- c <= 64 < c + k: this add crossed the limit. Later, the adder exchanges the
  word for 0 and adds the word's old fields and its own sums to the 32-bit
  fallback sums;
- c > 64: the word is past the limit and its owner will reset it, so the
  adder puts its own sums into the fallback.

The resolve adds the word's fields to the fallback sums.  The atomic is one
step and the follow-up another, and any number of other adders may run
between the two.  Every schedule must give the exact totals.  The model
also shows the check has teeth: a count field too narrow for the adds in
flight, or a dropped reset, gives wrong totals.
"""
import random

import pytest

LAYOUT = dict(shift_r=50, shift_g=36, shift_b=22, channel_bits=14, count_bits=22, limit=64)
M64 = (1 << 64) - 1


def simulate(adds, schedule_seed, burst, layout=LAYOUT, reset=True):
    """Run one schedule.  `adds` is a list of ((r, g, b), k).  At each step
    the scheduler issues the next atomic with probability `burst` (always
    when nothing is pending), else finishes a random pending follow-up.
    Returns (resolved totals, exact totals)."""
    rnd = random.Random(schedule_seed)
    cmask = (1 << layout["channel_bits"]) - 1
    kmask = (1 << layout["count_bits"]) - 1
    shifts = (layout["shift_r"], layout["shift_g"], layout["shift_b"])
    limit = layout["limit"]
    word = 0
    fallback = [0, 0, 0, 0]
    pending = []
    i = 0
    while i < len(adds) or pending:
        if i < len(adds) and (not pending or rnd.random() < burst):
            rgb, k = adds[i]
            i += 1
            packed = (rgb[0] << shifts[0]) | (rgb[1] << shifts[1]) | (rgb[2] << shifts[2]) | k
            old, word = word, (word + packed) & M64
            c = old & kmask
            if c + k > limit:
                pending.append((old, rgb, k, c))
        else:
            old, rgb, k, c = pending.pop(rnd.randrange(len(pending)))
            sums = [rgb[0], rgb[1], rgb[2], k]
            if c <= limit:
                if reset:
                    word = 0
                for j, s in enumerate(shifts):
                    sums[j] += (old >> s) & cmask
                sums[3] += c
            fallback = [a + b for a, b in zip(fallback, sums)]
    resolved = [fallback[j] + ((word >> s) & cmask) for j, s in enumerate(shifts)]
    resolved.append(fallback[3] + (word & kmask))
    exact = [sum(a[0][j] for a in adds) for j in range(3)] + [sum(a[1] for a in adds)]
    return resolved, exact


def random_adds(n, k_max, seed):
    rnd = random.Random(seed)
    out = []
    for _ in range(n):
        k = rnd.randint(1, k_max)
        out.append(((rnd.randint(0, 255 * k), rnd.randint(0, 255 * k), rnd.randint(0, 255 * k)), k))
    return out


@pytest.mark.parametrize("k_max", [1, 32])
@pytest.mark.parametrize("burst", [0.3, 0.6, 0.99])
def test_exact_under_random_schedules(k_max, burst):
    for seed in range(25):
        adds = random_adds(3000, k_max, seed)
        got, exact = simulate(adds, seed + 1000, burst)
        assert got == exact, (seed, got, exact)


def test_exact_with_every_adder_in_flight():
    """All atomics land before any follow-up runs: 100k single points and
    then 100k groups of up to 32 points, more than a 16-bit count holds."""
    for k_max in (1, 32):
        adds = random_adds(100_000, k_max, 7 + k_max)
        got, exact = simulate(adds, 3, burst=1.0)
        assert got == exact


def test_narrow_count_field_fails_with_many_in_flight():
    """A 16-bit count wraps when more than 65535 points land between a
    crossing add and its reset, and the totals come out wrong."""
    narrow = dict(LAYOUT, count_bits=16)
    adds = random_adds(70_000, 1, 11)
    got, exact = simulate(adds, 5, burst=1.0, layout=narrow)
    assert got != exact
    got, exact = simulate(adds, 5, burst=1.0)
    assert got == exact


def test_dropped_reset_fails():
    adds = random_adds(3000, 1, 2)
    got, exact = simulate(adds, 9, burst=0.6, reset=False)
    assert got != exact
