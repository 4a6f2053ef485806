"""Column exchanges of one panel (Sec. 2.4: at pivot t of a panel starting with m0
active columns, column l_t < m0 - t is exchanged with the boundary column
m0 - 1 - t). The batched trailing-row update relies on two facts about the
composed permutation (new[p] = old[src(p)]), checked here by brute force on
random exchange sequences:
  * a trailing position p < m0 - bb that receives another column receives it
    from the pivot block [m0 - bb, m0) (so its value can be read from the block
    before any trailing position is overwritten);
  * the moved positions form a permutation of at most 2 bb positions.
"""
import random

import pytest


def compose(m0, swaps):
    """src[p] for every position p after applying the exchanges in order."""
    cur = list(range(m0))  # cur[p] = original position of the column now at p
    for t, l in enumerate(swaps):
        b = m0 - 1 - t
        cur[l], cur[b] = cur[b], cur[l]
    return cur


@pytest.mark.parametrize("seed", range(40))
def test_trailing_destinations_take_block_columns(seed):
    rng = random.Random(seed)
    m0 = rng.randint(1, 600)
    bb = rng.randint(1, min(16, m0))
    # pivot t chooses any active column (0 .. m0-1-t), the boundary included;
    # bias towards the boundary region and repeats to reach chains of exchanges
    swaps = []
    for t in range(bb):
        hi = m0 - 1 - t
        choice = rng.random()
        if choice < 0.3:
            l = hi
        elif choice < 0.6:
            l = rng.randint(max(0, m0 - bb), hi)
        else:
            l = rng.randint(0, hi)
        swaps.append(l)
    src = compose(m0, swaps)
    pb = m0 - bb
    moved = [p for p in range(m0) if src[p] != p]
    assert sorted(src[p] for p in moved) == sorted(moved)  # a permutation of S
    assert len(moved) <= 2 * bb
    for p in moved:
        if p < pb:
            assert src[p] >= pb, (m0, bb, swaps, p, src[p])


def test_worked_chain():
    # m0 = 6, bb = 3: pivot 0 takes column 4 (the next boundary), pivot 1 takes
    # column 1, pivot 2 takes column 1 again
    src = compose(6, [4, 1, 1])
    # pivot 0: positions 4 and 5 exchange; pivot 1: positions 1 and 4 (old 5 -> 1);
    # pivot 2: positions 1 and 3
    assert src == [0, 3, 2, 5, 1, 4]
    pb = 3
    for p in range(pb):
        if src[p] != p:
            assert src[p] >= pb
