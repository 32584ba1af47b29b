"""Pins of the MIS-2 aggregation check used on the GPU's aggregates: it
accepts valid aggregations of small graphs and rejects each planted
mistake (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

from mis2_check import check_mis2_aggregation, sequential_mis2_aggregation


def _grid(nx, ny):
    """5-point grid graph plus one isolated node at the end."""
    idx = np.arange(nx * ny).reshape(nx, ny)
    r, c = [], []
    for a, b in ((idx[:-1, :], idx[1:, :]), (idx[:, :-1], idx[:, 1:])):
        r += a.ravel().tolist() + b.ravel().tolist()
        c += b.ravel().tolist() + a.ravel().tolist()
    n = nx * ny + 1
    return sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))


@pytest.fixture
def valid():
    S = _grid(9, 7)
    agg, roots = sequential_mis2_aggregation(S)
    return S, agg, roots


def test_valid_aggregation_passes(valid):
    S, agg, roots = valid
    check_mis2_aggregation(S, agg, roots)
    assert agg[-1] == -1 and roots.size > 3


def test_path_graph_by_hand():
    """Path 0-1-2-3-4-5-6: roots 0, 3, 6 (distance 3 apart), aggregates
    {0, 1}, {2, 3, 4}, {5, 6}."""
    n = 7
    S = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")
    agg, roots = sequential_mis2_aggregation(S)
    assert roots.tolist() == [0, 3, 6]
    assert agg.tolist() == [0, 0, 1, 1, 1, 2, 2]
    check_mis2_aggregation(S, agg, roots)


def test_roots_within_distance_two_rejected():
    n = 7
    S = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")
    # roots 0 and 2 are two apart
    agg = np.array([0, 0, 1, 1, 1, 2, 2])
    with pytest.raises(AssertionError, match="within distance 2"):
        check_mis2_aggregation(S, agg, np.array([0, 2, 6]))


def test_not_maximal_rejected():
    n = 9
    S = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")
    # roots 0 and 8 only: node 4 is farther than 2 from both
    agg = np.array([0, 0, 0, 0, 0, 1, 1, 1, 1])
    with pytest.raises(AssertionError):
        check_mis2_aggregation(S, agg, np.array([0, 8]))


def test_member_moved_to_a_far_aggregate_rejected(valid):
    S, agg, roots = valid
    bad = agg.copy()
    far = int(np.argmax(np.abs(np.arange(S.shape[0] - 1) - roots[0])))
    assert bad[far] != 0
    bad[far] = 0
    with pytest.raises(AssertionError):
        check_mis2_aggregation(S, bad, roots)


def test_dropped_node_rejected(valid):
    S, agg, roots = valid
    bad = agg.copy()
    bad[np.nonzero((bad >= 0) & ~np.isin(np.arange(bad.size), roots))[0][0]] = -1
    with pytest.raises(AssertionError, match="left out"):
        check_mis2_aggregation(S, bad, roots)


def test_isolated_node_aggregated_rejected(valid):
    S, agg, roots = valid
    bad = agg.copy()
    bad[-1] = 0
    with pytest.raises(AssertionError, match="isolated"):
        check_mis2_aggregation(S, bad, roots)


def test_root_neighbour_in_another_aggregate_rejected():
    n = 7
    S = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")
    # node 4, a neighbour of root 3, placed with root 6
    agg = np.array([0, 0, 1, 1, 2, 2, 2])
    with pytest.raises(AssertionError, match="strong neighbour of a root"):
        check_mis2_aggregation(S, agg, np.array([0, 3, 6]))
