"""Host planning of grouped submatrices (Section IV-C): periodic k-means on
molecule positions, the union dimensions n_G and Eq. estimatedspeedup,
checked on the CPU against brute force and constructed cases."""
import numpy as np
import pytest

from paper_2004_10811_gb300 import grouping
from synth import random_symmetric_bsr

pytest.importorskip("scipy")


def test_kmeans_keeps_a_cluster_that_straddles_the_boundary():
    """Two tight clusters in a 10 A box, one split by the periodic boundary
    (x near 0 and near 10): minimum-image k-means must keep it whole."""
    rng = np.random.default_rng(1)
    box = np.array([10.0, 10.0, 10.0])
    a = np.array([0.1, 5.0, 5.0]) + rng.normal(0, 0.2, (20, 3))  # straddles x = 0
    b = np.array([5.0, 5.0, 5.0]) + rng.normal(0, 0.2, (20, 3))
    coords = np.mod(np.vstack([a, b]), box)
    assert (coords[:20, 0] > 9).any() and (coords[:20, 0] < 1).any()
    labels = grouping.periodic_kmeans(coords, box, 2, seed=3)
    assert len(np.unique(labels[:20])) == 1 and len(np.unique(labels[20:])) == 1
    assert labels[0] != labels[20]


def circular_means(coords, box, labels):
    ang = 2 * np.pi * coords / box
    k = labels.max() + 1
    c = np.zeros((k, 3))
    for d in range(3):
        cs = np.bincount(labels, weights=np.cos(ang[:, d]), minlength=k)
        sn = np.bincount(labels, weights=np.sin(ang[:, d]), minlength=k)
        c[:, d] = np.mod(np.arctan2(sn, cs) * box[d] / (2 * np.pi), box[d])
    return c


def test_kmeans_labels_are_dense_and_a_fixed_point():
    """Labels 0..k'-1 all used, and at convergence every point is nearest
    (minimum image, brute force) to its own group's circular mean."""
    rng = np.random.default_rng(2)
    box = np.array([20.0, 20.0, 20.0])
    coords = rng.uniform(0, 20, (200, 3))
    labels = grouping.periodic_kmeans(coords, box, 30, seed=0, iters=200)
    assert labels.shape == (200,)
    assert set(np.unique(labels)) == set(range(labels.max() + 1))
    assert labels.max() + 1 <= 30
    centres = circular_means(coords, box, labels)
    diff = coords[:, None, :] - centres[None, :, :]
    diff -= box * np.round(diff / box)  # minimum image
    nearest = np.argmin(np.sum(diff * diff, axis=2), axis=1)
    assert np.array_equal(nearest, labels)


def test_group_dims_is_the_union_of_neighbourhoods():
    sizes = [3, 2, 4, 1, 3, 2, 2, 3]
    m = random_symmetric_bsr(sizes, density=0.35, seed=4, scale=0.5)
    labels = np.array([0, 0, 1, 1, 2, 2, 3, 3])
    dims, groups = grouping.group_dims(m.block_sizes, m.row_ptr, m.col_idx, labels)
    for g, members in enumerate(groups):
        rows = set()
        for j in members:
            rows |= set(m.col_idx[m.row_ptr[j]:m.row_ptr[j + 1]].tolist())
        assert dims[g] == sum(sizes[r] for r in rows)
    # singletons give the single-column dimensions
    single, _ = grouping.group_dims(m.block_sizes, m.row_ptr, m.col_idx, np.arange(len(sizes)))
    for j in range(len(sizes)):
        assert single[j] == sum(sizes[r] for r in m.col_idx[m.row_ptr[j]:m.row_ptr[j + 1]])


def test_estimated_speedup_definition():
    """S = sum_j n_j^3 / sum_G n_G^3 (Eq. estimatedspeedup), or with a cost function."""
    single = np.array([10, 10, 10, 10])
    assert grouping.estimated_speedup(single, single) == 1.0
    # two pairs whose unions are 12 wide: 4000 / (2 * 1728)
    assert abs(grouping.estimated_speedup(single, np.array([12, 12])) - 4000 / 3456) < 1e-15
    # a pair whose union is the sum of both (disjoint neighbourhoods) costs more
    assert grouping.estimated_speedup(single, np.array([20, 20])) < 1.0
    lin = grouping.estimated_speedup(single, np.array([12, 12]), cost=lambda n: np.asarray(n, float))
    assert abs(lin - 40 / 24) < 1e-15


def test_consecutive_groups():
    assert grouping.consecutive_groups(7, 2).tolist() == [0, 0, 1, 1, 2, 2, 3]
    assert grouping.consecutive_groups(4, 1).tolist() == [0, 1, 2, 3]
