"""Seeded synthetic graph generators.

This module is the only code shared by the FP64 oracle and the CUDA path. It
builds undirected, unweighted graphs and returns them as symmetric CSR arrays
(int32 row pointers, int32 column indices, each row sorted ascending, no
self-loops, no duplicate entries). It holds none of the spanning-centrality
arithmetic: no transition probabilities, no series, no solves.

Every generator takes an explicit integer seed and uses numpy's PCG64
``Generator``, so a given (generator, size, seed) triple yields the same graph
on every machine.

Workload families (sizes are the defaults used by the tests and the bench):

* ``tree_plus_gnp``  -- uniform random labelled tree (random Pruefer sequence)
  united with G(n, p) at a target average degree; n = 2,000, avg degree 10.
* ``barabasi_albert`` -- preferential attachment, star seed graph on m0+1
  nodes, each new node attaches to m0 distinct existing nodes drawn from the
  repeated-endpoint list; n = 200,000, m0 = 10 gives m = 1,999,900.
* ``perturbed_grid`` -- rows x cols lattice, a random-weight minimum spanning
  tree is protected, and a fraction of the remaining lattice edges is deleted.
* ``gnp_lcc`` -- G(n, c/(n-1)) restricted to its largest component.
* ``rmat`` -- recursive-matrix (R-MAT) edges, symmetrised, deduplicated,
  largest component, random relabelling.
* ``batch_graphs`` -- the mixed family of many small graphs of uneven size.

Named fixtures (``complete``, ``cycle``, ``path``, ``star``,
``complete_bipartite``, ``petersen``, ``hypercube``, ``barbell``,
``lollipop``, ``grid``) are small graphs whose effective resistances have
closed forms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSRGraph", "from_edges", "largest_component",
    "complete", "cycle", "path", "star", "complete_bipartite", "petersen",
    "hypercube", "barbell", "lollipop", "grid",
    "random_tree", "tree_plus_gnp", "barabasi_albert", "perturbed_grid",
    "gnp_lcc", "rmat", "batch_graphs", "workload",
]


@dataclass
class CSRGraph:
    """Symmetric CSR adjacency of an undirected simple graph."""

    n: int
    row_ptr: np.ndarray  # int32[n + 1]
    col_idx: np.ndarray  # int32[nnz], nnz = 2 m
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def m(self) -> int:
        return self.nnz // 2

    @property
    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edges(self) -> np.ndarray:
        """Undirected edge list (u < v), one row per edge, in CSR order of u."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), self.degree)
        cols = self.col_idx.astype(np.int64)
        keep = rows < cols
        return np.stack([rows[keep], cols[keep]], axis=1)

    def entry_rows(self) -> np.ndarray:
        """Row index of every CSR entry (int64[nnz])."""
        return np.repeat(np.arange(self.n, dtype=np.int64), self.degree)


def from_edges(n: int, u, v, name: str = "", meta: dict | None = None) -> CSRGraph:
    """Build a symmetric, sorted, deduplicated CSR from an undirected edge list.

    Self-loops are dropped and repeated edges are merged.
    """
    u = np.asarray(u, dtype=np.int64).ravel()
    v = np.asarray(v, dtype=np.int64).ravel()
    keep = u != v
    u, v = u[keep], v[keep]
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    # sorted distinct keys (sort + adjacent comparison: the result np.unique
    # gives, without its hash-based path, which is slow on large inputs)
    key = np.sort(rows * np.int64(n) + cols, kind="stable")
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    rows = key // n
    cols = key % n
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("graph too large for int32 CSR")
    return CSRGraph(n=n, row_ptr=row_ptr.astype(np.int32), col_idx=cols.astype(np.int32),
                    name=name, meta=dict(meta or {}))


def largest_component(g: CSRGraph, name: str | None = None) -> CSRGraph:
    """Restrict ``g`` to its largest connected component, relabelled 0..n'-1
    in increasing order of the old labels."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    a = sp.csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    ncomp, lab = connected_components(a, directed=False)
    if ncomp == 1:
        return g
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    newid = np.full(g.n, -1, dtype=np.int64)
    newid[keep] = np.arange(keep.size)
    e = g.edges()
    mask = (newid[e[:, 0]] >= 0) & (newid[e[:, 1]] >= 0)
    e = e[mask]
    return from_edges(keep.size, newid[e[:, 0]], newid[e[:, 1]],
                      name=name if name is not None else g.name, meta=g.meta)


def relabel(g: CSRGraph, perm: np.ndarray) -> CSRGraph:
    """Return the graph with node x renamed perm[x]."""
    e = g.edges()
    return from_edges(g.n, perm[e[:, 0]], perm[e[:, 1]], name=g.name, meta=g.meta)


# ----------------------------------------------------------------------------
# Named fixtures
# ----------------------------------------------------------------------------

def complete(n: int) -> CSRGraph:
    iu, ju = np.triu_indices(n, 1)
    return from_edges(n, iu, ju, name=f"K{n}")


def cycle(n: int) -> CSRGraph:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, name=f"C{n}")


def path(n: int) -> CSRGraph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, name=f"P{n}")


def star(leaves: int) -> CSRGraph:
    return from_edges(leaves + 1, np.zeros(leaves, dtype=np.int64), np.arange(1, leaves + 1),
                      name=f"S{leaves}")


def complete_bipartite(a: int, b: int) -> CSRGraph:
    u, v = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return from_edges(a + b, u.ravel(), v.ravel(), name=f"K{a},{b}")


def petersen() -> CSRGraph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = np.array(outer + spokes + inner)
    return from_edges(10, e[:, 0], e[:, 1], name="petersen")


def hypercube(d: int) -> CSRGraph:
    n = 1 << d
    x = np.arange(n)
    us, vs = [], []
    for b in range(d):
        y = x ^ (1 << b)
        keep = x < y
        us.append(x[keep])
        vs.append(y[keep])
    return from_edges(n, np.concatenate(us), np.concatenate(vs), name=f"Q{d}")


def barbell(k: int, bridge_len: int = 1) -> CSRGraph:
    """Two K_k joined by a path of ``bridge_len`` edges (all path edges are bridges)."""
    us, vs = [], []
    for off in (0, k):
        iu, ju = np.triu_indices(k, 1)
        us.append(iu + off)
        vs.append(ju + off)
    n = 2 * k + (bridge_len - 1)
    chain = [k - 1] + list(range(2 * k, n)) + [k]
    us.append(np.array(chain[:-1]))
    vs.append(np.array(chain[1:]))
    return from_edges(n, np.concatenate(us), np.concatenate(vs), name=f"barbell{k}_{bridge_len}")


def lollipop(k: int, tail: int) -> CSRGraph:
    """K_k with a path of ``tail`` extra nodes hanging off node k-1."""
    iu, ju = np.triu_indices(k, 1)
    chain = np.arange(k - 1, k + tail)
    u = np.concatenate([iu, chain[:-1]])
    v = np.concatenate([ju, chain[1:]])
    return from_edges(k + tail, u, v, name=f"lollipop{k}_{tail}")


def grid(rows: int, cols: int) -> CSRGraph:
    idx = np.arange(rows * cols).reshape(rows, cols)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return from_edges(rows * cols, u, v, name=f"grid{rows}x{cols}")


# ----------------------------------------------------------------------------
# Random families
# ----------------------------------------------------------------------------

def _prufer_tree_edges(n: int, rng: np.random.Generator):
    """Edges of the labelled tree encoded by a uniform random Pruefer sequence.

    The decoding is the textbook linear-time one: repeatedly join the smallest
    current leaf to the next sequence element.
    """
    if n == 1:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    if n == 2:
        return np.array([0]), np.array([1])
    seq = rng.integers(0, n, size=n - 2)
    degree = np.ones(n, dtype=np.int64)
    np.add.at(degree, seq, 1)
    import heapq

    leaves = [i for i in range(n) if degree[i] == 1]
    heapq.heapify(leaves)
    us, vs = [], []
    for x in seq.tolist():
        leaf = heapq.heappop(leaves)
        us.append(leaf)
        vs.append(x)
        degree[x] -= 1
        if degree[x] == 1:
            heapq.heappush(leaves, x)
    a = heapq.heappop(leaves)
    b = heapq.heappop(leaves)
    us.append(a)
    vs.append(b)
    return np.array(us, dtype=np.int64), np.array(vs, dtype=np.int64)


def random_tree(n: int, seed: int) -> CSRGraph:
    rng = np.random.default_rng(seed)
    u, v = _prufer_tree_edges(n, rng)
    return from_edges(n, u, v, name=f"tree{n}_s{seed}")


def _gnp_pairs(n: int, p: float, rng: np.random.Generator):
    """Undirected pairs of G(n, p): the edge count is drawn Binomial(C(n,2), p)
    and that many distinct pairs are then drawn uniformly (which is G(n, p)
    conditioned on its edge count, hence G(n, p))."""
    total = n * (n - 1) // 2
    mcount = int(rng.binomial(total, p))
    chosen = np.zeros(0, dtype=np.int64)
    while chosen.size < mcount:
        need = mcount - chosen.size
        cand = rng.integers(0, total, size=int(need * 1.1) + 16)
        chosen = np.unique(np.concatenate([chosen, cand]))
        if chosen.size > mcount:
            chosen = rng.permutation(chosen)[:mcount]
    # unrank pair index t -> (i, j), i < j, row-major over the upper triangle
    t = chosen.astype(np.float64)
    i = np.floor((2 * n - 1 - np.sqrt((2 * n - 1) ** 2 - 8 * t)) / 2).astype(np.int64)
    start = i * (2 * n - i - 1) // 2
    # guard against floating-point rounding in the square root
    over = start > chosen
    i[over] -= 1
    start = i * (2 * n - i - 1) // 2
    under = chosen - start >= (n - 1 - i)
    i[under] += 1
    start = i * (2 * n - i - 1) // 2
    j = chosen - start + i + 1
    return i, j


def tree_plus_gnp(n: int = 2000, avg_degree: float = 10.0, seed: int = 0) -> CSRGraph:
    """Uniform random spanning tree united with G(n, p), p chosen so that the
    expected edge count is n * avg_degree / 2."""
    rng = np.random.default_rng(seed)
    tu, tv = _prufer_tree_edges(n, rng)
    target = n * avg_degree / 2.0
    p = (target - (n - 1)) / (n * (n - 1) / 2.0)
    gu, gv = _gnp_pairs(n, max(p, 0.0), rng)
    return from_edges(n, np.concatenate([tu, gu]), np.concatenate([tv, gv]),
                      name=f"tree+gnp_n{n}_d{avg_degree:g}_s{seed}",
                      meta={"family": "tree_plus_gnp", "seed": seed})


def barabasi_albert(n: int = 200_000, m0: int = 10, seed: int = 1) -> CSRGraph:
    """Preferential attachment on a star seed graph (nodes 0..m0, centre 0).

    Node v >= m0+1 attaches to m0 distinct earlier nodes, each drawn uniformly
    from the list holding both endpoints of every edge so far (probability
    proportional to degree). m = m0 * (n - m0).
    """
    rng = np.random.default_rng(seed)
    total_edges = m0 + (n - m0 - 1) * m0
    us = np.empty(total_edges, dtype=np.int64)
    vs = np.empty(total_edges, dtype=np.int64)
    ends = np.empty(2 * total_edges, dtype=np.int64)
    us[:m0] = 0
    vs[:m0] = np.arange(1, m0 + 1)
    ends[0:2 * m0:2] = 0
    ends[1:2 * m0:2] = np.arange(1, m0 + 1)
    ne = m0
    nend = 2 * m0
    batch = rng.random(size=(n, 3 * m0))
    for v in range(m0 + 1, n):
        draws = (batch[v] * nend).astype(np.int64)
        picked = []
        seen = set()
        for t in ends[draws].tolist():
            if t not in seen:
                seen.add(t)
                picked.append(t)
                if len(picked) == m0:
                    break
        while len(picked) < m0:  # rare: top up with fresh draws
            t = int(ends[int(rng.random() * nend)])
            if t not in seen:
                seen.add(t)
                picked.append(t)
        us[ne:ne + m0] = v
        vs[ne:ne + m0] = picked
        ends[nend:nend + 2 * m0:2] = v
        ends[nend + 1:nend + 2 * m0:2] = picked
        ne += m0
        nend += 2 * m0
    return from_edges(n, us, vs, name=f"ba_n{n}_m{m0}_s{seed}",
                      meta={"family": "barabasi_albert", "seed": seed})


def perturbed_grid(rows: int = 1000, cols: int = 1000, delete_frac: float = 0.05,
                   seed: int = 2) -> CSRGraph:
    """rows x cols lattice (row-major ids). A minimum spanning tree under i.i.d.
    uniform edge weights is protected; ``delete_frac`` of all lattice edges
    are then deleted uniformly at random among the non-tree edges, so the
    result stays connected (and bipartite)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import minimum_spanning_tree

    rng = np.random.default_rng(seed)
    idx = np.arange(rows * cols).reshape(rows, cols)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    ne = u.size
    w = rng.random(ne) + 1e-9  # strictly positive weights
    n = rows * cols
    mst = minimum_spanning_tree(sp.csr_matrix((w, (u, v)), shape=(n, n))).tocoo()
    tree_key = set()
    tkey = np.minimum(mst.row, mst.col).astype(np.int64) * n + np.maximum(mst.row, mst.col)
    in_tree = np.isin(np.minimum(u, v).astype(np.int64) * n + np.maximum(u, v), tkey)
    del tree_key
    ndel = int(round(delete_frac * ne))
    candidates = np.flatnonzero(~in_tree)
    ndel = min(ndel, candidates.size)
    dele = rng.choice(candidates, size=ndel, replace=False)
    keep = np.ones(ne, dtype=bool)
    keep[dele] = False
    return from_edges(n, u[keep], v[keep], name=f"pgrid_{rows}x{cols}_f{delete_frac:g}_s{seed}",
                      meta={"family": "perturbed_grid", "seed": seed, "bipartite": True})


def gnp_lcc(n: int, avg_degree: float = 8.0, seed: int = 0) -> CSRGraph:
    rng = np.random.default_rng(seed)
    u, v = _gnp_pairs(n, avg_degree / (n - 1), rng)
    g = from_edges(n, u, v)
    return largest_component(g, name=f"gnp_lcc_n{n}_d{avg_degree:g}_s{seed}")


def rmat(scale: int, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 5,
         chunk: int = 1 << 24) -> CSRGraph:
    """R-MAT edges (no per-level noise), random vertex permutation, symmetrised,
    self-loops and duplicates removed, largest component, relabelled."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    nedges = edge_factor * n
    a, b, c, _ = abcd
    us, vs = [], []
    done = 0
    while done < nedges:
        k = min(chunk, nedges - done)
        uu = np.zeros(k, dtype=np.int64)
        vv = np.zeros(k, dtype=np.int64)
        for lvl in range(scale):
            r = rng.random(k, dtype=np.float32)
            bit_u = r >= (a + b)            # quadrants c, d set the row bit
            bit_v = ((r >= a) & (r < a + b)) | (r >= a + b + c)  # quadrants b, d set the column bit
            uu |= bit_u.astype(np.int64) << lvl
            vv |= bit_v.astype(np.int64) << lvl
        us.append(uu)
        vs.append(vv)
        done += k
    perm = rng.permutation(n)
    u = perm[np.concatenate(us)]
    v = perm[np.concatenate(vs)]
    g = from_edges(n, u, v)
    return largest_component(g, name=f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def planted_partition(k: int = 8, size: int = 500, d_in: float = 10.0, d_out: float = 0.5,
                      seed: int = 6) -> CSRGraph:
    """k communities of `size` nodes (community c holds nodes c*size .. (c+1)*size - 1).
    Inside each: a uniform random spanning tree united with G(size, p_in), p_in
    set for an expected internal degree d_in. Between them: a ring of k edges
    (community c to c+1 mod k, random endpoints) keeps the graph connected, and
    G(n, p_out) restricted to pairs in different communities adds an expected
    d_out external neighbours per node. With d_out << d_in the walk leaves a
    community rarely: k - 1 eigenvalues of N lie close to 1 (a bottleneck
    family, where Eq. 6 with lambda_2 alone asks very long lengths)."""
    rng = np.random.default_rng(seed)
    n = k * size
    us, vs = [], []
    for c in range(k):
        tu, tv = _prufer_tree_edges(size, rng)
        p_in = max((size * d_in / 2.0 - (size - 1)) / (size * (size - 1) / 2.0), 0.0)
        gu, gv = _gnp_pairs(size, p_in, rng)
        us += [c * size + tu, c * size + gu]
        vs += [c * size + tv, c * size + gv]
    if k > 1:
        ring = np.arange(k)
        us.append(ring * size + rng.integers(0, size, size=k))
        vs.append(((ring + 1) % k) * size + rng.integers(0, size, size=k))
        p_out = d_out / max(n - size, 1)
        ou, ov = _gnp_pairs(n, p_out, rng)
        cross = ou // size != ov // size
        us.append(ou[cross])
        vs.append(ov[cross])
    return from_edges(n, np.concatenate(us), np.concatenate(vs),
                      name=f"planted_k{k}_s{size}_din{d_in:g}_dout{d_out:g}_s{seed}",
                      meta={"family": "planted_partition", "seed": seed})


def batch_graphs(count: int = 512, nmin: int = 1000, nmax: int = 50000, base_seed: int = 4):
    """Many independent graphs of uneven size. Graph g uses seed base_seed+g,
    n_g = round(exp(U[ln nmin, ln nmax])), and its family cycles with g mod 3:
    G(n, 8/(n-1)) largest component, Barabasi-Albert with 5 edges per node,
    and a perturbed grid on ceil(sqrt n) x ceil(n / ceil(sqrt n)) nodes."""
    out = []
    for gi in range(count):
        seed = base_seed + gi
        rng = np.random.default_rng(seed)
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kind = gi % 3
        if kind == 0:
            g = gnp_lcc(n, 8.0, seed)
        elif kind == 1:
            g = barabasi_albert(n, 5, seed)
        else:
            r = int(math.ceil(math.sqrt(n)))
            c = int(math.ceil(n / r))
            g = perturbed_grid(r, c, 0.05, seed)
        out.append(g)
    return out


def workload(name: str, **kw) -> CSRGraph:
    """The named workloads by what they are (sizes may be overridden)."""
    if name == "tree_gnp_2k":
        return tree_plus_gnp(kw.get("n", 2000), kw.get("avg_degree", 10.0), kw.get("seed", 0))
    if name == "ba_200k":
        return barabasi_albert(kw.get("n", 200_000), kw.get("m0", 10), kw.get("seed", 1))
    if name == "grid_1000":
        return perturbed_grid(kw.get("rows", 1000), kw.get("cols", 1000), 0.05, kw.get("seed", 2))
    if name == "rmat_22":
        return rmat(kw.get("scale", 22), 16, seed=kw.get("seed", 5))
    if name == "planted_200k":
        return planted_partition(kw.get("k", 40), kw.get("size", 5000), kw.get("d_in", 10.0), kw.get("d_out", 0.2),
                                 kw.get("seed", 6))
    raise KeyError(name)
