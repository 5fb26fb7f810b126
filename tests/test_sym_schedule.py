"""CPU checks of the pair-symmetric evaluation's ordered accumulation (no GPU).

The shared-step evaluation adds each block's j-side sums into one slot per row
chunk, row after row in a fixed order; a row waits for its turn.  The library's
own plan and turn computation are checked here on the host, for every padded
size from one block up to config-scale discs and several resident-CTA counts
(152 SMs x 2, 3, 4 CTAs, and small counts that force many waves): each slot's
writers hold the turns 0 .. n-1 exactly once, slots without writers are the
ones zeroed, and no turn waits on a writer that could be waiting on it.
"""
import pytest

import paper_2006_02501_gb300 as mh


SMALL = [1, 2, 129, 256, 257, 511, 700, 1024, 1100, 2048, 3000, 4097, 8000, 8192, 16384, 16385]
LARGE = [32768, 65537, 100000, 131072, 262144]
CASES = [(N, s) for N in SMALL for s in (3, 17, 152, 152 * 2, 152 * 3)] + \
        [(N, s) for N in LARGE for s in (152, 152 * 3)]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N,slots", CASES)
def test_ordered_accumulation_schedule(N, slots, precision):
    plan = mh.sym_schedule_check(N, slots, precision)
    nB = (N + 255) // 256 * 2
    assert plan["blocks"] == nB
    items = -(-nB // plan["rows_per_item"]) * plan["chunks"]
    if plan["cyclic"]:
        # one item per CTA only when every item is resident at once
        assert plan["grid"] == items <= slots
    else:
        assert plan["grid"] == slots < items


def test_slot_memory_is_linear():
    """The partial sums take C (1 + G) slots, C row chunks and G chains (one):
    O(N C), not O(N^2) (one slot per block distance would be Np/256)."""
    for N in (65537, 262144):
        for slots, precision in ((152 * 3, 0), (152, 1)):
            plan = mh.sym_schedule_check(N, slots, precision)
            assert plan["chains"] == 1
            assert plan["rows_per_item"] == (6 if precision else 3)
            assert 2 * plan["chunks"] <= 40


def test_schedule_check_rejects_bad_arguments():
    with pytest.raises(mh.MHError):
        mh.sym_schedule_check(0, 10)
    with pytest.raises(mh.MHError):
        mh.sym_schedule_check(100, 0)
    with pytest.raises(mh.MHError):
        mh.sym_schedule_check(100, 10, 7)


@pytest.mark.parametrize("N", [1, 2, 127, 128, 129, 255, 256, 257, 300, 383, 384, 385, 1000, 2047, 2048,
                               2100, 2176, 2177, 2500, 4095, 4096, 4097, 9999, 30000])
def test_dd_symmetric_work_map(N):
    """The symmetric double-double kernel (one item per unordered pair of
    64-body blocks, its diagonal block included): every block pair is one
    item, each of the nB partial-sum slots gets every block once, for odd
    and even block counts and a ragged last block, and the kernel's own ring
    schedule takes every body pair inside an item once (the diagonal item's
    unordered pairs once, no self pair)."""
    r = mh.dd_sym_check(N)
    nB = -(-N // 64)
    assert r["blocks"] == nB
    assert r["items"] == nB * (nB + 1) // 2
    assert r["bad_pairs"] == 0 and r["bad_slots"] == 0 and r["bad_body_pairs"] == 0
