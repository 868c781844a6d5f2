"""The ensemble tuner's list-scheduling model (host arithmetic, callable
without a GPU) against schedules worked out by hand."""
import numpy as np
import pytest

from paper_1809_10895_gb300 import rf


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()


def test_equal_instances_fill_whole_waves():
    for n, units in ((8, 4), (9, 4), (3, 5)):
        m = rf.ens_model_makespan(np.full(n, 2.0), np.arange(n), units)
        assert m == 2.0 * -(-n // units)


def test_longest_first_list_schedule():
    # times 3, 3, 2, 2, 2 on two units, heaviest first: {3, 2, 2} and {3, 2}
    # -> 7 (the optimum 6 = {3, 3} / {2, 2, 2} is not a list schedule of this order)
    t = np.array([3.0, 3.0, 2.0, 2.0, 2.0])
    assert rf.ens_model_makespan(t, [0, 1, 2, 3, 4], 2) == 7.0
    # lightest first: {2, 2, 3} and {2, 3} -> 7 as well
    assert rf.ens_model_makespan(t, [2, 3, 4, 0, 1], 2) == 7.0


def test_split_after_the_wide_instances():
    # one unit of 4 CTAs: instance 0 wide (5 s); the next pop (instance 1)
    # splits the unit at t = 5 into 4 single CTAs, which run 1..4 at once
    wide = np.array([5.0, 1.0, 1.0, 1.0, 1.0])
    solo = np.array([20.0, 3.0, 1.5, 4.0, 2.0])
    assert rf.ens_model_makespan(wide, [0, 1, 2, 3, 4], 1, cluster=4, n_wide=1, solo_s=solo) == 9.0
    # nothing wide: the unit splits at once; 4 CTAs run solo times 20, 3, 1.5, 4, then 2 after 1.5
    assert rf.ens_model_makespan(wide, [0, 1, 2, 3, 4], 1, cluster=4, n_wide=0, solo_s=solo) == 20.0


def test_model_argument_errors():
    with pytest.raises(rf.RFError):
        rf.ens_model_makespan([1.0, 2.0], [0, 0], 1)          # not a permutation
    with pytest.raises(rf.RFError):
        rf.ens_model_makespan([1.0, 2.0], [0, 1], 0)          # no unit
    with pytest.raises(rf.RFError):
        rf.ens_model_makespan([1.0, 2.0], [0, 1], 1, cluster=2, n_wide=0)   # split without solo times
