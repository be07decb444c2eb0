"""The block partition of an ensemble launch (gea_ensemble_plan), on the
host: members whose weight share is below one block share blocks, up to one
block's worth each, and run in turn; the others own blocks in proportion to
their weights, at least one and at most one per tile; no more blocks than
there are."""
import numpy as np
import pytest

from paper_2303_10499_gb300 import build as B


@pytest.fixture(scope="module")
def gea():
    B.build()
    from paper_2303_10499_gb300 import gea as G
    return G


def check_invariants(plan, w, tiles, blocks):
    nb, grp = plan["blocks"], plan["group"]
    assert plan["used_blocks"] <= blocks
    share = blocks * w / w.sum()
    used = 0
    for g in range(plan["groups"]):
        members = np.flatnonzero(grp == g)
        assert len(members) >= 1
        if len(members) > 1:
            # a shared block: one block's worth of weight at most
            assert (nb[members] == 1).all() and share[members].sum() <= 1.0 + 1e-12
            used += 1
        else:
            used += nb[members[0]]
    assert used == plan["used_blocks"]
    assert (nb >= 1).all() and (nb <= tiles).all()


def test_small_members_share_and_the_large_one_gets_the_rest(gea):
    w = np.r_[np.full(600, 2.0), 650.0]
    tiles = np.r_[np.full(600, 2), 650]
    plan = gea.ensemble_plan(w, tiles, 456)
    check_invariants(plan, w, tiles, 456)
    small_groups = set(plan["group"][:600])
    assert len(small_groups) == 300                       # two members (0.49 blocks each) a block
    assert plan["blocks"][600] == 456 - 300 and plan["used_blocks"] == 456


def test_large_members_in_proportion(gea):
    rng = np.random.default_rng(1)
    w = rng.uniform(1.0, 10.0, 40)
    tiles = np.full(40, 10 ** 6)
    plan = gea.ensemble_plan(w, tiles, 456)
    check_invariants(plan, w, tiles, 456)
    assert plan["groups"] == 40 and plan["used_blocks"] == 456
    share = 456 * w / w.sum()
    # one block at least each, the rest by the largest remainders
    assert (np.abs(plan["blocks"] - share) < 2.0).all()


def test_tiles_cap_the_blocks(gea):
    w = np.array([1.0, 1.0, 100.0])
    tiles = np.array([100, 100, 7])
    plan = gea.ensemble_plan(w, tiles, 456)
    check_invariants(plan, w, tiles, 456)
    assert plan["blocks"][2] == 7


def test_mixed_sizes_of_the_les_ensemble(gea):
    # 85 members each of 100^2, 200^2 and 400^2 cells (16 x 16 tiles), weights
    # tiles x (1 + iterations)^2.5 with their iteration counts
    tiles = np.repeat([49, 169, 625], 85)
    its = np.repeat([43, 55, 77], 85)
    w = tiles * (1.0 + its) ** 2.5
    plan = gea.ensemble_plan(w, tiles, 456)
    check_invariants(plan, w, tiles, 456)
    assert plan["blocks"][-85:].min() >= 3


def test_refuses_what_does_not_fit(gea):
    # shares alternating 0.6 and 0.5 block: packed in member order one to a
    # block, 20 blocks for 20 members, and no block of its own for each on 11
    w = np.tile([6.0, 5.0], 10)
    with pytest.raises(gea.GeaError):
        gea.ensemble_plan(w, np.full(20, 10), 11)
    with pytest.raises(gea.GeaError):
        gea.ensemble_plan(np.array([1.0, 0.0]), np.array([1, 1]), 8)
    with pytest.raises(gea.GeaError):
        gea.ensemble_plan(np.array([1.0, 1.0]), np.array([1, 0]), 8)
