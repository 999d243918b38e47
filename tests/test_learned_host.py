"""Host logic of the learned-preconditioner training (no GPU): the schedule of
combined training pairs."""
import numpy as np
import pytest

from paper_2603_23343_gb300 import learned


def test_combination_schedule_pairs_of_one_problem():
    steps, nprob, per = 5000, 32, 7
    a, b, c = learned.combination_schedule(steps, nprob, per, seed=0)
    assert a.shape == b.shape == (steps,) and c.shape == (steps, 2)
    assert np.all(a != b)
    assert np.all(a // per == b // per)  # the same problem
    assert a.min() >= 0 and max(a.max(), b.max()) < nprob * per
    # every problem and every ordered pair of its snapshots is drawn
    assert len(np.unique(a // per)) == nprob
    assert np.unique(np.stack([a % per, b % per]), axis=1).shape[1] == per * (per - 1)
    # standard-normal coefficients
    assert abs(c.mean()) < 0.05 and abs(c.std() - 1.0) < 0.05
    # seeded: the same schedule again, another one for another seed
    a2, b2, c2 = learned.combination_schedule(steps, nprob, per, seed=0)
    assert np.array_equal(a, a2) and np.array_equal(b, b2) and np.array_equal(c, c2)
    a3, _, _ = learned.combination_schedule(steps, nprob, per, seed=1)
    assert not np.array_equal(a, a3)


def test_combination_schedule_two_pairs():
    a, b, _ = learned.combination_schedule(100, 1, 2, seed=4)
    assert set(zip(a.tolist(), b.tolist())) == {(0, 1), (1, 0)}


def test_combination_schedule_rejects_single_pair():
    with pytest.raises(ValueError):
        learned.combination_schedule(10, 3, 1)
