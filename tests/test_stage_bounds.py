"""Bounds of the slice kernel's bulk copies, checked on the host for every
entry layout: each copy starts and ends on 16-byte boundaries, covers the
stage's entries, fits its shared-memory slot (stage bytes + 16) (as do the 16-byte
group loads that read records out of it), and reads at most 16
bytes past the last entry (the padding the build adds after each table's
inline codes).  The arithmetic restates the kernel's stage sizing (3, 4 and
8 KB stages, the three shapes: 8W-byte codes, or 4(2W-1)-byte records
rounded down to whole groups of four).  The slot bound is also a static_assert in the kernel source over the
stage size it is compiled with, so a build with another stage size or
another copy rule that overruns a slot does not compile."""
import numpy as np
import pytest

STAGES = (3072, 4096, 8192)


def stage_entries(W, reduced, STAGE):
    # records: whole groups of four (16 (2W - 1) bytes) in a stage, less the
    # three records a copy may start early
    return 4 * (STAGE // (16 * (2 * W - 1))) - 3 if reduced else STAGE // (8 * W)


def copy_of(W, reduced, pos, cnt):
    """(first byte, bytes, entry offset in the slot) of the copy of entries [pos, pos + cnt)."""
    if reduced:
        rb = 4 * (2 * W - 1)
        lo = pos & ~3
        return lo * rb, ((cnt + pos - lo) * rb + 15) & ~15, pos - lo, rb
    if W == 1:
        lo = pos & ~1
        return lo * 8, ((cnt + pos - lo) * 8 + 15) & ~15, pos - lo, 8
    return pos * 8 * W, cnt * 8 * W, 0, 8 * W


@pytest.mark.parametrize("STAGE", STAGES)
@pytest.mark.parametrize("W,reduced", [(1, False), (2, False), (4, False), (1, True), (2, True), (4, True)])
def test_stage_copies_stay_in_bounds(W, reduced, STAGE):
    SLOT = STAGE + 16
    rng = np.random.default_rng(W * 10 + reduced)
    per = stage_entries(W, reduced, STAGE)
    assert per >= 32 and (reduced or per % 32 == 0)
    for n in (1, 2, 3, 5, 97, 1024, 100_003):
        for _ in range(300):
            pos = int(rng.integers(0, n))
            cnt = int(rng.integers(1, min(per, n - pos) + 1))
            start, nbytes, shift, eb = copy_of(W, reduced, pos, cnt)
            assert start % 16 == 0 and nbytes % 16 == 0 and nbytes > 0
            assert nbytes <= SLOT
            # the stage's entries lie inside the copy
            assert start <= pos * eb and (pos + cnt) * eb <= start + nbytes
            assert shift * eb == pos * eb - start
            if reduced:
                # lanes read whole groups of four records (16-byte loads) that
                # hold a stage record: all inside the slot
                groups = (shift + cnt + 3) // 4
                assert groups * 4 * eb <= SLOT and (4 * eb) % 16 == 0
            # at most 16 bytes past the end of the table's n entries
            assert start + nbytes <= n * eb + 16
