"""The tree property behind the partial projection between the stages of the MR
step: in a graded tree (every block's parent and the parent's 3^d-1 neighbours
exist, Section 2.1), a block of level l with an absent position among its own
3^d-1 neighbours of level l is a leaf.  The GPU step projects, between its
stages, only the parent quadrants of such leaves (and its ghost strips read only
coarse cells over them); this holds only if no such block can be refined.

Checked on the oracle's trees after adaptation by the MR criterion and by the
gradient criterion, in 2D and 3D, with transmissive and periodic boundaries;
and, so that the check can fail, on a hand-built tree that breaks the grading
rule.  No GPU: the trees are the oracle's.
"""
import itertools

import numpy as np
import pytest

import mrfv_inputs as mi
import oracle


def _bc(b, n, periodic):
    if periodic:
        return b % n
    return b if 0 <= b < n else None


def edge_blocks_refined(o, periodic):
    """Blocks (l, index) that have an absent same-level neighbour position and
    are refined, for every level of the oracle's tree."""
    bad = []
    for l in range(1, o.L):  # the finest level has no children
        ex = o.get_exist(l).astype(bool)
        leaf = o.leaf_mask(l)
        shape = ex.shape
        for idx in np.argwhere(ex & ~leaf):
            absent = False
            for off in itertools.product((-1, 0, 1), repeat=o.dim):
                if not any(off):
                    continue
                q = []
                for d in range(o.dim):
                    b = _bc(int(idx[d]) + off[d], shape[d], periodic)
                    if b is None:
                        break
                    q.append(b)
                if len(q) < o.dim:
                    continue  # outside a transmissive domain: not an absent block
                if not ex[tuple(q)]:
                    absent = True
                    break
            if absent:
                bad.append((l, tuple(int(i) for i in idx)))
    return bad


@pytest.mark.parametrize("dim,periodic,criterion", [(2, False, oracle.CRIT_MR), (2, True, oracle.CRIT_MR),
                                                    (2, False, oracle.CRIT_GRAD), (3, False, oracle.CRIT_MR),
                                                    (3, True, oracle.CRIT_GRAD)])
def test_blocks_next_to_an_absent_block_are_leaves(dim, periodic, criterion):
    bc = oracle.BC_PERIODIC if periodic else oracle.BC_TRANSMISSIVE
    if dim == 2:
        o = oracle.Oracle(2, 5, (1, 1, 1), bc=bc)
        o.init(mi.IC_QUADRANTS, mi.quadrant_params(2))
    else:
        o = oracle.Oracle(3, 4, (1, 1, 1), lo=(-1, -1, -1), hi=(1, 1, 1), bc=bc)
        o.init(mi.IC_ELLIPSOID, mi.ellipsoid_params(3))
    refined_somewhere = False
    for _ in range(3):
        o.adapt(criterion, 1e-3, eps_w=0.05)
        assert edge_blocks_refined(o, periodic) == []
        refined_somewhere |= any((o.get_exist(l).astype(bool) & ~o.leaf_mask(l)).any() for l in range(1, o.L))
        o.step(o.dt(0.4))
    assert refined_somewhere  # the trees had refined blocks below level 0 to check


def test_the_check_finds_a_refined_block_next_to_an_absent_one():
    """A tree that breaks the grading rule: level 2 refined in one corner block of
    level 1 whose neighbour position on level 1 is absent."""
    o = oracle.Oracle(2, 4, (1, 1, 1))
    o.init(mi.IC_QUADRANTS, mi.quadrant_params(0))
    ex1 = np.zeros(o.blocks_shape(1), np.uint8)
    ex1[:] = 1
    ex2 = np.zeros(o.blocks_shape(2), np.uint8)
    ex2[0:2, 0:2] = 1  # the children of level-1 block (0, 0)
    ex3 = np.zeros(o.blocks_shape(3), np.uint8)
    ex3[0:2, 0:2] = 1  # the children of level-2 block (0, 0): its neighbour (0, 2) is absent
    for l, ex in ((1, ex1), (2, ex2), (3, ex3)):
        o.set_exist(l, ex)
    assert (2, (0, 0)) not in edge_blocks_refined(o, False)  # (0, 1) and (1, 0), (1, 1) exist
    ex3[:] = 0
    ex3[2:4, 2:4] = 1  # children of level-2 block (1, 1), whose neighbours (2, *) and (*, 2) are absent
    o.set_exist(3, ex3)
    assert (2, (1, 1)) in edge_blocks_refined(o, False)
