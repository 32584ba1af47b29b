"""Complete validity check of a distance-2 maximal independent set (MIS-2)
aggregation, used on the GPU's aggregates (the aggregation is not unique:
its roots depend on the priorities, so every property that any valid
result has is checked instead, on every node and every aggregate)."""
import numpy as np
import scipy.sparse as sp


def check_mis2_aggregation(S, agg, roots):
    """S: strength graph (n x n, symmetric pattern, no diagonal); agg[i]:
    aggregate of node i (-1: none); roots[a]: the root of aggregate a.
    Asserts:
    - isolated nodes (no strong neighbour) are left out, all others covered;
    - roots[a] lies in aggregate a, roots in increasing node order;
    - the roots are pairwise at graph distance >= 3 (independent at distance 2);
    - every non-isolated node lies within distance 2 of a root (maximal);
    - aggregate a contains every strong neighbour of its root;
    - every member of aggregate a lies within distance 2 of its root;
    - every aggregate is connected in the strength graph (implied by the two
      before it, checked on its own all the same)."""
    n = S.shape[0]
    S = sp.csr_matrix(S, copy=True)
    S.setdiag(0)
    S.eliminate_zeros()
    S.data[:] = 1.0
    deg = np.diff(S.indptr)
    agg = np.asarray(agg)
    roots = np.asarray(roots)
    assert agg.shape == (n,)
    assert np.all(agg[deg == 0] == -1), "an isolated node was aggregated"
    assert np.all(agg[deg > 0] >= 0), "a non-isolated node was left out"
    na = int(agg.max()) + 1
    assert set(np.unique(agg[agg >= 0]).tolist()) == set(range(na))
    assert roots.shape == (na,)
    assert np.all(np.diff(roots) > 0) and roots.min() >= 0 and roots.max() < n
    assert np.array_equal(agg[roots], np.arange(na)), "a root lies outside its aggregate"
    S2 = (S @ S + S + sp.identity(n, format="csr")).tocsr()
    S2.data[:] = 1.0
    RR = S2[roots][:, roots]
    assert RR.nnz == na, "two roots lie within distance 2"
    near = np.asarray(S2[:, roots].sum(axis=1)).ravel()
    assert np.all(near[deg > 0] >= 1), "a node is farther than 2 from every root (not maximal)"
    nb = S[roots]
    rows = np.repeat(np.arange(na), np.diff(nb.indptr))
    assert np.array_equal(agg[nb.indices], rows), "a strong neighbour of a root left its aggregate"
    mem = np.nonzero(agg >= 0)[0]
    sel = sp.csr_matrix((np.ones(mem.size), (mem, roots[agg[mem]])), shape=(n, n))
    assert S2.multiply(sel).nnz == mem.size, "a member lies farther than 2 from its root"
    coo = S.tocoo()
    keep = (agg[coo.row] >= 0) & (agg[coo.row] == agg[coo.col])
    G = sp.csr_matrix((np.ones(int(keep.sum())), (coo.row[keep], coo.col[keep])), shape=(n, n))
    _, lab = sp.csgraph.connected_components(G, directed=False)
    comp_of_agg = np.full(na, -1)
    comp_of_agg[agg[mem]] = lab[mem]
    assert np.array_equal(lab[mem], comp_of_agg[agg[mem]])
    assert np.unique(comp_of_agg).size == na, "an aggregate is not connected"


def sequential_mis2_aggregation(S):
    """A valid MIS-2 aggregation built one node at a time (small graphs
    only): a node becomes a root when no root lies within distance 2, its
    strong neighbours join it, every other node joins the aggregate of an
    aggregated neighbour."""
    S = sp.csr_matrix(S)
    n = S.shape[0]
    ip, ix = S.indptr, S.indices
    nbrs = [set(ix[ip[i]:ip[i + 1]].tolist()) - {i} for i in range(n)]
    is_root = np.zeros(n, bool)
    for i in range(n):
        if not nbrs[i]:
            continue
        d2 = set(nbrs[i])
        for j in nbrs[i]:
            d2 |= nbrs[j]
        if not any(is_root[j] for j in d2 | {i}):
            is_root[i] = True
    roots = np.nonzero(is_root)[0]
    agg = -np.ones(n, np.int64)
    agg[roots] = np.arange(roots.size)
    for a, r in enumerate(roots):
        for j in nbrs[r]:
            agg[j] = a
    first = agg.copy()
    for i in range(n):
        if agg[i] < 0 and nbrs[i]:
            agg[i] = next(first[j] for j in sorted(nbrs[i]) if first[j] >= 0)
    return agg, roots
