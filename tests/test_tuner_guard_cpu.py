"""The learned tuner's guard decision (host logic, no GPU).

The guard compresses a fixed sample of the field with the network's class
and with the default class, and keeps the network's class unless it has
more outliers there, or unless its padding costs more to compute (a global
padding: a field-wide statistic and a pass over the block origins) and the
two estimated sizes tie by the rule the training labels use: within
SIZE_TOL of the smaller one, the cheaper padding wins.
"""
import pytest

from paper_2201_04614_gb300 import tuner as T

# class c: block slot c // 3, padding slot c % 3 (zero, global avg, block avg)
ZERO_B0, GAVG_B0, BAVG_B0 = 0, 1, 2
ZERO_B1, GAVG_B1 = 3, 4


def test_same_class_is_kept():
    assert T.guard_pick(ZERO_B0, ZERO_B0, (5, 1), (10.0, 1.0)) == ZERO_B0


def test_more_outliers_fall_back():
    assert T.guard_pick(ZERO_B1, ZERO_B0, (11, 10), (1.0, 100.0)) == ZERO_B0
    assert T.guard_pick(GAVG_B1, ZERO_B0, (11, 10), (1.0, 100.0)) == ZERO_B0


def test_dearer_padding_on_a_size_tie_falls_back():
    # the global-average class saves outliers but less than SIZE_TOL of size
    lo = 1_000_000.0
    assert T.guard_pick(GAVG_B0, ZERO_B0, (0, 1964), (lo, lo * (1 + 0.5 * T.SIZE_TOL))) == ZERO_B0
    # at the tolerance itself it is still a tie
    assert T.guard_pick(GAVG_B1, ZERO_B0, (0, 10), (lo, lo * (1 + T.SIZE_TOL))) == ZERO_B0
    # per-block padding is dearer than zero padding too
    assert T.guard_pick(BAVG_B0, ZERO_B0, (3, 9), (lo, lo)) == ZERO_B0


def test_dearer_padding_that_pays_is_kept():
    lo = 1_000_000.0
    assert T.guard_pick(GAVG_B0, ZERO_B0, (0, 50_000), (lo, lo * (1 + 2 * T.SIZE_TOL))) == GAVG_B0
    assert T.guard_pick(BAVG_B0, ZERO_B0, (0, 50_000), (lo, lo * 1.1)) == BAVG_B0


def test_dearer_padding_that_is_larger_falls_back():
    assert T.guard_pick(GAVG_B0, ZERO_B0, (0, 0), (2.0e6, 1.0e6)) == ZERO_B0


def test_same_padding_cost_keeps_the_tuned_block_on_a_tie():
    # another block size with the same padding costs nothing more to compute
    assert T.guard_pick(ZERO_B1, ZERO_B0, (0, 0), (1.0e6, 1.0e6)) == ZERO_B1


def test_without_sizes_only_outliers_decide():
    assert T.guard_pick(GAVG_B0, ZERO_B0, (0, 1), None) == GAVG_B0
    assert T.guard_pick(GAVG_B0, ZERO_B0, (2, 1), None) == ZERO_B0


@pytest.mark.parametrize("slot,rank", [(0, 0), (1, 2), (2, 1)])
def test_padding_cost_order_matches_the_labels(slot, rank):
    # zero < per block < global, the order label_of uses to break size ties
    assert T.PAD_RANK[slot] == rank
