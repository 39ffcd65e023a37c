"""Partition of independent instances over ranks (host logic of the weak /
instance-sharded multi-GPU mode): contiguous ranges that cover every
instance once, no idle rank while instances remain, and balanced cost."""
import numpy as np
import pytest

from paper_2608_18541_b300.shard import contiguous_shards


def _check(costs, world):
    sh = contiguous_shards(costs, world)
    assert len(sh) == world
    start = 0
    for base, count in sh:
        assert base == start and count >= 0
        start += count
    assert start == len(costs)
    if len(costs) >= world:
        assert all(c >= 1 for _, c in sh)
    return sh


def test_heavy_first_instance_does_not_idle_a_rank():
    assert _check([100, 1, 1], 3) == [(0, 1), (1, 1), (2, 1)]


def test_more_ranks_than_instances():
    sh = _check([5, 7], 4)
    assert sum(c for _, c in sh) == 2 and max(c for _, c in sh) == 1


def test_equal_costs_split_evenly():
    assert _check([1.0] * 12, 4) == [(0, 3), (3, 3), (6, 3), (9, 3)]


@pytest.mark.parametrize("seed", range(20))
def test_random_costs_are_balanced(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 200))
    world = int(rng.integers(1, 9))
    costs = list(rng.integers(1, 14 ** 3, size=n).astype(float))   # atoms of cubes of side <= 14
    sh = _check(costs, world)
    loads = [sum(costs[b:b + c]) for b, c in sh]
    # greedy contiguous split: no rank exceeds the ideal share by more than one instance
    if n >= world:
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9


def test_world_must_be_positive():
    with pytest.raises(ValueError):
        contiguous_shards([1.0], 0)
