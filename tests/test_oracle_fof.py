"""Pins of the oracle's friends-of-friends groups against what the
definition fixes: hand-built chains, gaps and periodic links; the connected
components of scipy's k-d tree pair set (an independent library route);
species selection; and the invariants of a partition into link components."""
import numpy as np
import pytest

import oracle


def test_chain_links_and_gaps():
    b = 0.05
    # a chain at 0.9 b spacing, a gap of 1.1 b, a second chain; y = z = 0.5
    xs = [0.1 + 0.9 * b * k for k in range(5)]
    xs += [xs[-1] + 1.1 * b + 0.9 * b * k for k in range(3)]
    pos = np.array([[x, 0.5, 0.5] for x in xs])
    grp, ng = oracle.fof(pos, np.zeros(len(xs), np.uint8), 1.0, b)
    assert ng == 2
    assert list(grp) == [0] * 5 + [5] * 3


def test_link_across_the_periodic_face():
    b = 0.05
    pos = np.array([[0.01, 0.3, 0.3], [0.99, 0.3, 0.3], [0.5, 0.5, 0.5]])
    grp, ng = oracle.fof(pos, np.zeros(3, np.uint8), 1.0, b)
    assert ng == 2 and list(grp) == [0, 0, 2]


def test_strict_threshold():
    b = 0.25  # exactly representable separations
    pos = np.array([[0.0, 0.0, 0.0], [0.25, 0.0, 0.0], [0.5, 0.0, 0.0], [0.5 + 0.125, 0.0, 0.0]])
    grp, ng = oracle.fof(pos, np.zeros(4, np.uint8), 2.0, b)
    # r == b does not link; 0.125 < b does
    assert list(grp) == [0, 1, 2, 2] and ng == 3


def test_species_mask_ignores_the_other_species():
    b = 0.05
    # two DM particles 1.6 b apart, bridged by a gas particle in the middle
    pos = np.array([[0.4, 0.5, 0.5], [0.4 + 1.6 * b, 0.5, 0.5], [0.4 + 0.8 * b, 0.5, 0.5]])
    sp = np.array([0, 0, 1], np.uint8)
    grp, ng = oracle.fof(pos, sp, 1.0, b, species_mask=1)
    assert list(grp) == [0, 1, -1] and ng == 2
    grp, ng = oracle.fof(pos, sp, 1.0, b, species_mask=3)
    assert list(grp) == [0, 0, 0] and ng == 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_connected_components_of_a_kd_tree(seed):
    spatial = pytest.importorskip("scipy.spatial")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    sparse = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(seed)
    n = 3000
    # clumps plus background so that groups of many sizes appear
    centres = rng.uniform(0, 1, (20, 3))
    pos = np.concatenate([rng.uniform(0, 1, (n // 2, 3)),
                          (centres[rng.integers(0, 20, n - n // 2)] + rng.normal(0, 0.01, (n - n // 2, 3))) % 1.0])
    b = 0.012
    grp, ng = oracle.fof(pos, np.zeros(n, np.uint8), 1.0, b)
    pairs = spatial.cKDTree(pos, boxsize=1.0).query_pairs(b, output_type="ndarray")
    g = sparse.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    ncomp, lab = csgraph.connected_components(g, directed=False)
    assert ng == ncomp
    # canonical label: the smallest index of each component
    smallest = np.full(ncomp, n, np.int64)
    np.minimum.at(smallest, lab, np.arange(n))
    assert np.array_equal(grp, smallest[lab])
    assert ng < n  # some groups really formed


def test_partition_invariants_by_brute_force():
    rng = np.random.default_rng(7)
    n = 400
    pos = rng.uniform(0, 1, (n, 3))
    b = 0.06
    grp, ng = oracle.fof(pos, np.zeros(n, np.uint8), 1.0, b)
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.round(d)
    r2 = (d[..., 0] ** 2 + d[..., 1] ** 2) + d[..., 2] ** 2
    linked = (r2 < b * b) & ~np.eye(n, dtype=bool)
    # linked particles share a group
    i, j = np.nonzero(linked)
    assert np.all(grp[i] == grp[j])
    # every label is the smallest index of its group and the group count matches
    for g in np.unique(grp):
        members = np.flatnonzero(grp == g)
        assert members.min() == g
    assert ng == len(np.unique(grp))
