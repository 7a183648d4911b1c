"""Seeded synthetic inputs: graphs in symmetric CSR form and initial eigenvector blocks.

This module produces input data only. It holds none of the method's arithmetic (no Laplacian,
no polynomial, no solver); both the FP64 oracle and the CUDA path read what it writes.

Graph conventions (shared by every consumer):
  * undirected, no self-loops, no duplicate edges;
  * stored as a symmetric CSR: ``row_ptr`` (n+1, int32), ``col_idx`` (nnz, int32), columns
    sorted ascending inside each row; ``w`` (nnz, float32) or ``None`` for unit weights;
  * a weighted graph carries one weight per undirected edge, written to both directions.

Workload families follow the paper's experiments (all synthetic in the paper too): stochastic
block models and planted clusters (Section 5.4), cliques completed by link prediction
(Appendix A.1), the 3-room grid world
(Section 5.3), and closed-form graphs used to pin the oracle (path, cycle, complete, star,
grid, disjoint cliques; Section 2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSRGraph", "from_edges", "path", "cycle", "complete", "star", "grid", "cliques",
    "sbm", "sbm_regular", "sbm_by_degree", "chung_lu_clusters", "batched_sbm", "concat_graphs",
    "random_graph", "three_room_grid", "gaussian_block", "uniform_edge_weights",
    "common_neighbour_scores", "link_completed_cliques",
    "undirected_edges", "DEFAULT_SEED",
]

DEFAULT_SEED = 20220729


@dataclasses.dataclass
class CSRGraph:
    n: int
    row_ptr: np.ndarray          # int32 [n+1]
    col_idx: np.ndarray          # int32 [nnz]
    w: np.ndarray | None = None  # float32 [nnz] or None (unit weights)
    labels: np.ndarray | None = None  # planted block of each node, if any
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def n_edges(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        """Number of stored neighbours per row (not the weighted degree)."""
        return np.diff(self.row_ptr.astype(np.int64))

    def max_count_degree(self) -> int:
        return int(self.degrees().max()) if self.n else 0


def _stable_argsort(keys, device=None):
    """Indices that sort int64 keys, equal keys in input order (numpy, or torch on `device`:
    the same permutation, for large generators)."""
    if device is None:
        return np.argsort(keys, kind="stable")
    import torch
    t = torch.from_numpy(np.ascontiguousarray(keys)).to(device)
    return torch.sort(t, stable=True).indices.cpu().numpy()


def _first_of_each(keys, device=None):
    """Ascending indices of the first occurrence of every distinct key."""
    order = _stable_argsort(keys, device)
    ks = keys[order]
    head = np.ones(len(ks), dtype=bool)
    head[1:] = ks[1:] != ks[:-1]
    return np.sort(order[head])


def _searchsorted_right(cum, r, device=None):
    if device is None:
        return np.searchsorted(cum, r, side="right")
    import torch
    c = torch.from_numpy(np.ascontiguousarray(cum)).to(device)
    q = torch.from_numpy(np.ascontiguousarray(r)).to(device)
    return torch.searchsorted(c, q, right=True).cpu().numpy()


def from_edges(n: int, a, b, w=None, labels=None, name: str = "", device=None) -> CSRGraph:
    """Build a symmetric CSR from undirected edge endpoint arrays.

    Self-loops are dropped; duplicates of an undirected edge are merged, keeping the first
    weight in input order (the input-hygiene reading for unspecified inputs). `device` (a torch
    device) runs the two sorts there; the result is the same.
    """
    a = np.asarray(a, dtype=np.int64).ravel()
    b = np.asarray(b, dtype=np.int64).ravel()
    keep = a != b
    a, b = a[keep], b[keep]
    if w is not None:
        w = np.asarray(w, dtype=np.float32).ravel()[keep]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = lo * np.int64(n) + hi
    first = _first_of_each(key, device)
    lo, hi = lo[first], hi[first]
    if w is not None:
        w = w[first]
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    order = _stable_argsort(rows * np.int64(n) + cols, device)
    rows, cols = rows[order], cols[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 indexing")
    ww = None
    if w is not None:
        ww = np.concatenate([w, w])[order].astype(np.float32)
    return CSRGraph(n=n, row_ptr=row_ptr.astype(np.int32), col_idx=cols.astype(np.int32),
                    w=ww, labels=None if labels is None else np.asarray(labels, np.int32),
                    name=name)


def undirected_edges(g: CSRGraph):
    """(a, b, w) for every undirected edge with a < b, in CSR order of row a."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    cols = g.col_idx.astype(np.int64)
    up = rows < cols
    w = None if g.w is None else g.w[up]
    return rows[up], cols[up], w


# ----------------------------------------------------------------------------------------
# closed-form graphs (their Laplacian spectra are known; used to pin the oracle)
# ----------------------------------------------------------------------------------------
def path(n: int) -> CSRGraph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, name=f"path{n}")


def cycle(n: int) -> CSRGraph:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, name=f"cycle{n}")


def cycle_csr(n: int) -> CSRGraph:
    """The cycle C_n (n >= 3) built directly in CSR, O(n) memory and time (for sizes where the
    sorting in from_edges would be slow): row r holds r - 1 and r + 1 modulo n, sorted."""
    if n < 3:
        raise ValueError("cycle needs n >= 3")
    r = np.arange(n, dtype=np.int64)
    lo = np.where(r == 0, 1, r - 1)
    hi = np.where(r == 0, n - 1, np.where(r == n - 1, r - 1, r + 1))
    lo[n - 1] = 0
    col = np.empty(2 * n, dtype=np.int32)
    col[0::2] = lo
    col[1::2] = hi
    row_ptr = (2 * np.arange(n + 1, dtype=np.int64)).astype(np.int32)
    return CSRGraph(n=n, row_ptr=row_ptr, col_idx=col, name=f"cycle{n}")


def complete(n: int) -> CSRGraph:
    a, b = np.triu_indices(n, 1)
    return from_edges(n, a, b, name=f"K{n}")


def star(n: int) -> CSRGraph:
    i = np.arange(1, n)
    return from_edges(n, np.zeros(n - 1, np.int64), i, name=f"star{n}")


def grid(rows: int, cols: int) -> CSRGraph:
    idx = np.arange(rows * cols).reshape(rows, cols)
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return from_edges(rows * cols, a, b, name=f"grid{rows}x{cols}")


def cliques(sizes, short_circuit: int = 0, seed: int = DEFAULT_SEED) -> CSRGraph:
    """Disjoint cliques, optionally joined by ``short_circuit`` random inter-clique edges
    (the Section 5.4 generator joins cliques by 0 to 25 such edges)."""
    rng = np.random.default_rng(seed)
    sizes = [int(s) for s in sizes]
    off = np.concatenate([[0], np.cumsum(sizes)])
    a_list, b_list, lab = [], [], []
    for c, s in enumerate(sizes):
        aa, bb = np.triu_indices(s, 1)
        a_list.append(aa + off[c])
        b_list.append(bb + off[c])
        lab.append(np.full(s, c))
    n = int(off[-1])
    labels = np.concatenate(lab)
    if short_circuit and len(sizes) > 1:
        got = 0
        ea, eb = [], []
        while got < short_circuit:
            u = rng.integers(0, n, size=4 * short_circuit)
            v = rng.integers(0, n, size=4 * short_circuit)
            m = labels[u] != labels[v]
            u, v = u[m], v[m]
            take = min(len(u), short_circuit - got)
            ea.append(u[:take])
            eb.append(v[:take])
            got += take
        a_list += ea
        b_list += eb
    return from_edges(n, np.concatenate(a_list), np.concatenate(b_list), labels=labels,
                      name=f"cliques{sizes}")


def common_neighbour_scores(n: int, oa, ob, ra, rb) -> np.ndarray:
    """Common-neighbours link prediction: for each candidate pair (ra[i], rb[i]) the number of
    neighbours its two ends share in the observed graph with undirected edges (oa, ob). Dense
    n x n adjacency: small graphs only."""
    if n > 8192:
        raise ValueError("common_neighbour_scores: n above 8192")
    adj = np.zeros((n, n), dtype=np.float32)
    adj[oa, ob] = 1.0
    adj[ob, oa] = 1.0
    cn = np.zeros(len(ra), dtype=np.float32)
    for s in range(0, len(ra), 4096):
        cn[s:s + 4096] = np.einsum("ij,ij->i", adj[ra[s:s + 4096]], adj[rb[s:s + 4096]])
    return cn


def link_completed_cliques(sizes, short_circuit: int = 25, p_remove: float = 0.2,
                           seed: int = DEFAULT_SEED):
    """App. A.1 workload (clustering probabilistic graphs): a cliques graph of Section 5.4 whose
    edges are each removed with probability ``p_remove``; every removed edge is scored by
    common-neighbours link prediction on the observed graph and put back with its score divided
    by the largest score among the removed edges, so predicted edges carry weights in (0, 1] and
    observed edges weight 1. A removed edge whose ends share no neighbour scores 0 and stays
    out. Returns (graph, removed): removed is the 2 x m array of the removed pairs (i < j)."""
    base = cliques(sizes, short_circuit, seed)
    n = base.n
    rng = np.random.default_rng([seed, 1])
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(base.row_ptr))
    upper = base.col_idx > rows
    a, b = rows[upper], base.col_idx[upper].astype(np.int64)
    drop = rng.random(len(a)) < p_remove
    oa, ob, ra, rb = a[~drop], b[~drop], a[drop], b[drop]
    cn = common_neighbour_scores(n, oa, ob, ra, rb)
    keep = cn > 0
    top = cn.max() if keep.any() else 1.0
    w = np.concatenate([np.ones(len(oa), dtype=np.float32), cn[keep] / top])
    g = from_edges(n, np.concatenate([oa, ra[keep]]), np.concatenate([ob, rb[keep]]), w=w,
                   labels=base.labels, name=f"link_completed_cliques{list(sizes)}")
    return g, np.stack([ra, rb])


# ----------------------------------------------------------------------------------------
# random workloads
# ----------------------------------------------------------------------------------------
def _pairs_within(rng, starts, sizes, m):
    """m uniform ordered pairs (u, v), u != v mostly, inside blocks given per draw."""
    u = starts + (rng.random(m) * sizes).astype(np.int64)
    v = starts + (rng.random(m) * sizes).astype(np.int64)
    return u, v


def sbm(n: int, n_blocks: int, p_in: float, p_out: float, seed: int = DEFAULT_SEED,
        permute: bool = False) -> CSRGraph:
    """Stochastic block model with equal blocks (the last one takes the remainder).

    Edge counts are drawn from the exact binomials of the model; endpoints are drawn
    uniformly inside the pair class and duplicates merged, which for sparse graphs differs
    from the exact model only by the O(m^2/pairs) merged duplicates.
    """
    rng = np.random.default_rng(seed)
    base = n // n_blocks
    sizes = np.full(n_blocks, base, dtype=np.int64)
    sizes[-1] += n - base * n_blocks
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    labels = np.repeat(np.arange(n_blocks), sizes)
    intra_pairs = sizes * (sizes - 1) // 2
    m_in = rng.binomial(intra_pairs, p_in)
    blk = np.repeat(np.arange(n_blocks), m_in)
    u_in, v_in = _pairs_within(rng, starts[blk], sizes[blk], int(m_in.sum()))
    total_pairs = n * (n - 1) // 2
    inter_pairs = total_pairs - int(intra_pairs.sum())
    m_out = int(rng.binomial(inter_pairs, p_out)) if inter_pairs > 0 else 0
    ua, va = [], []
    got = 0
    while got < m_out:
        need = m_out - got
        u = rng.integers(0, n, size=int(need * 1.2) + 16)
        v = rng.integers(0, n, size=int(need * 1.2) + 16)
        keep = labels[u] != labels[v]
        u, v = u[keep][:need], v[keep][:need]
        ua.append(u)
        va.append(v)
        got += len(u)
    a = np.concatenate([u_in] + ua) if ua else u_in
    b = np.concatenate([v_in] + va) if va else v_in
    g = from_edges(n, a, b, labels=labels, name=f"sbm{n}x{n_blocks}")
    if permute:
        g = _permute(g, rng.permutation(n))
    return g


def sbm_regular(n: int, n_blocks: int, d_in: int, d_out: int, seed: int = DEFAULT_SEED) -> CSRGraph:
    """Near-regular stochastic block model by the configuration model: every node gets d_in
    stubs paired uniformly inside its block and d_out stubs paired uniformly across blocks
    (self loops, same-block cross pairs and duplicates dropped). Same block structure and mean
    degree as ``sbm`` with p_in (b-1) = d_in, p_out (n-b) = d_out, without the Poisson
    low-degree tail whose localized eigenvectors crowd the bottom of the spectrum."""
    rng = np.random.default_rng(seed)
    base = n // n_blocks
    sizes = np.full(n_blocks, base, dtype=np.int64)
    sizes[-1] += n - base * n_blocks
    labels = np.repeat(np.arange(n_blocks), sizes)
    stubs = np.repeat(np.arange(n, dtype=np.int64), d_in)
    order = np.lexsort((rng.random(len(stubs)), labels[stubs]))
    s = stubs[order]
    bl = labels[s]
    m = len(s) // 2
    a, b = s[0:2 * m:2], s[1:2 * m:2]
    keep = bl[0:2 * m:2] == bl[1:2 * m:2]
    a, b = a[keep], b[keep]
    out = rng.permutation(np.repeat(np.arange(n, dtype=np.int64), d_out))
    m2 = len(out) // 2
    c, d = out[0:2 * m2:2], out[1:2 * m2:2]
    cross = labels[c] != labels[d]
    return from_edges(n, np.concatenate([a, c[cross]]), np.concatenate([b, d[cross]]),
                      labels=labels, name=f"sbmreg{n}x{n_blocks}")


def sbm_by_degree(n: int, n_blocks: int, mean_degree: float, intra_frac: float,
                  seed: int = DEFAULT_SEED) -> CSRGraph:
    """SBM parameterised by mean degree and the fraction of intra-block edge ends."""
    base = max(n // n_blocks, 2)
    p_in = min(1.0, mean_degree * intra_frac / max(base - 1, 1))
    rest = max(n - base, 1)
    p_out = min(1.0, mean_degree * (1.0 - intra_frac) / rest)
    return sbm(n, n_blocks, p_in, p_out, seed=seed)


def _permute(g: CSRGraph, perm: np.ndarray) -> CSRGraph:
    a, b, w = undirected_edges(g)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    lab = None
    if g.labels is not None:
        lab = np.empty_like(g.labels)
        lab[inv] = g.labels
    return from_edges(g.n, inv[a], inv[b], w=w, labels=lab, name=g.name + "-perm")


def random_graph(n: int, m: int, seed: int = DEFAULT_SEED, hub: int | None = None,
                 hub_degree: int = 0, isolated: int = 0) -> CSRGraph:
    """Uniform random multigraph merged to a simple graph, with optional hub and isolated
    nodes (ragged rows, empty rows and one long row for kernel edge cases)."""
    rng = np.random.default_rng(seed)
    live = n - isolated
    a = rng.integers(0, live, size=m)
    b = rng.integers(0, live, size=m)
    if hub is not None and hub_degree:
        hb = rng.choice(live, size=min(hub_degree, live), replace=False)
        a = np.concatenate([a, np.full(len(hb), hub)])
        b = np.concatenate([b, hb])
    return from_edges(n, a, b, name=f"rand{n}_{m}")


def chung_lu_clusters(n: int, n_clusters: int = 64, gamma: float = 2.5, d_min: float = 4.0,
                      d_max: float = 1e4, sigma: float = 1.0, intra_frac: float = 0.9,
                      target_nnz: float | None = None, weighted: bool = True,
                      seed: int = DEFAULT_SEED, device=None) -> CSRGraph:
    """Planted-cluster Chung-Lu graph: expected degrees from a power law with exponent
    ``gamma`` on [d_min, d_max], clusters of log-normal sizes, a fraction ``intra_frac`` of
    edge ends inside the cluster. Nodes are ordered by cluster. Weights U(0.5, 1.5).
    `device` (a torch device) runs the searches and sorts there; the graph is the same."""
    rng = np.random.default_rng(seed)
    e = 1.0 - gamma
    u = rng.random(n)
    theta = (d_min ** e - u * (d_min ** e - d_max ** e)) ** (1.0 / e)
    if target_nnz is not None:
        theta *= target_nnz / theta.sum()
    sz = rng.lognormal(0.0, sigma, size=n_clusters)
    sz = np.maximum(1, np.floor(sz / sz.sum() * n)).astype(np.int64)
    sz[-1] += n - sz.sum()
    if sz[-1] < 1:
        raise ValueError("cluster sizes do not fit n")
    off = np.concatenate([[0], np.cumsum(sz)])
    labels = np.repeat(np.arange(n_clusters), sz)
    cum = np.cumsum(theta)
    total = cum[-1]
    a_list, b_list = [], []
    # intra-cluster edges: endpoints drawn proportional to theta inside the cluster
    s_c = np.array([cum[off[c + 1] - 1] - (cum[off[c] - 1] if off[c] > 0 else 0.0)
                    for c in range(n_clusters)])
    m_c = rng.poisson(intra_frac * s_c / 2.0)
    for c in range(n_clusters):
        if m_c[c] == 0 or sz[c] < 2:
            continue
        lo = cum[off[c] - 1] if off[c] > 0 else 0.0
        r1 = lo + rng.random(m_c[c]) * s_c[c]
        r2 = lo + rng.random(m_c[c]) * s_c[c]
        a_list.append(np.minimum(_searchsorted_right(cum, r1, device), off[c + 1] - 1))
        b_list.append(np.minimum(_searchsorted_right(cum, r2, device), off[c + 1] - 1))
    m_out = int(rng.poisson((1.0 - intra_frac) * total / 2.0))
    if m_out:
        r1 = rng.random(m_out) * total
        r2 = rng.random(m_out) * total
        ua = np.minimum(_searchsorted_right(cum, r1, device), n - 1)
        va = np.minimum(_searchsorted_right(cum, r2, device), n - 1)
        keep = labels[ua] != labels[va]
        a_list.append(ua[keep])
        b_list.append(va[keep])
    a = np.concatenate(a_list)
    b = np.concatenate(b_list)
    w = rng.uniform(0.5, 1.5, size=len(a)).astype(np.float32) if weighted else None
    return from_edges(n, a, b, w=w, labels=labels, name=f"chunglu{n}", device=device)


def batched_sbm(n_graphs: int, n_min: int = 200, n_max: int = 20000, blocks_min: int = 2,
                blocks_max: int = 8, mean_degree: float = 12.0, intra_frac: float = 0.875,
                seed: int = DEFAULT_SEED):
    """Independent SBMs of log-uniform size and a random number of blocks each."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_graphs)).astype(int)
    nb = rng.integers(blocks_min, blocks_max + 1, size=n_graphs)
    seeds = rng.integers(0, 2**62, size=n_graphs)
    return [sbm_by_degree(int(sizes[i]), int(nb[i]), mean_degree, intra_frac, seed=int(seeds[i]))
            for i in range(n_graphs)]


def concat_graphs(graphs):
    """Block-diagonal union: returns (graph, node_offsets[int64, G+1], nnz_offsets[G+1])."""
    node_off = np.zeros(len(graphs) + 1, dtype=np.int64)
    nnz_off = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        node_off[i + 1] = node_off[i] + g.n
        nnz_off[i + 1] = nnz_off[i] + g.nnz
    rp = np.empty(node_off[-1] + 1, dtype=np.int64)
    rp[0] = 0
    cols = np.empty(nnz_off[-1], dtype=np.int64)
    ws = None if graphs[0].w is None else np.empty(nnz_off[-1], dtype=np.float32)
    for i, g in enumerate(graphs):
        rp[node_off[i] + 1: node_off[i + 1] + 1] = g.row_ptr[1:].astype(np.int64) + nnz_off[i]
        cols[nnz_off[i]: nnz_off[i + 1]] = g.col_idx.astype(np.int64) + node_off[i]
        if ws is not None:
            ws[nnz_off[i]: nnz_off[i + 1]] = g.w
    if rp[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 indexing")
    big = CSRGraph(n=int(node_off[-1]), row_ptr=rp.astype(np.int32),
                   col_idx=cols.astype(np.int32), w=ws, name=f"batch{len(graphs)}")
    return big, node_off, nnz_off


def three_room_grid(s: int = 2, h: int = 10) -> CSRGraph:
    """3-room grid world of Section 5.3: (10s+1) x (30s+1) cells, two inner walls splitting it
    into three rooms, each wall with one door of height about (10s+1)/h cells (centred).
    The wall geometry is not drawn in the text; this reading places full-height walls at
    one and two thirds of the width."""
    H, W = 10 * s + 1, 30 * s + 1
    walls = {W // 3, (2 * W) // 3}
    door = max(1, round(H / h))
    d0 = (H - door) // 2
    free = np.ones((H, W), dtype=bool)
    for c in walls:
        free[:, c] = False
        free[d0:d0 + door, c] = True
    idx = -np.ones((H, W), dtype=np.int64)
    idx[free] = np.arange(free.sum())
    a, b = [], []
    for r in range(H):
        for c in range(W):
            if not free[r, c]:
                continue
            if c + 1 < W and free[r, c + 1]:
                a.append(idx[r, c]); b.append(idx[r, c + 1])
            if r + 1 < H and free[r + 1, c]:
                a.append(idx[r, c]); b.append(idx[r + 1, c])
    return from_edges(int(free.sum()), a, b, name=f"3room_s{s}_h{h}")


# ----------------------------------------------------------------------------------------
# vectors and weights
# ----------------------------------------------------------------------------------------
def gaussian_block(n: int, k: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """V0 with i.i.d. N(0,1) entries (float64, row-major n x k)."""
    return np.random.default_rng(seed).standard_normal((n, k))


def hash_block(rows, k: int, xp=np):
    """Deterministic block for sizes beyond host memory: entry (r, c) = (h & 255) / 256 - 1/2
    with h an integer hash of (r, c), so every value has at most 8 significant bits (exact in
    BF16). `rows` is an integer array (numpy or torch, `xp` its module); the same values come
    out on the host and on a device."""
    r = rows.reshape(-1, 1).to(xp.int64) if xp is not np else np.asarray(rows, np.int64)[:, None]
    c = xp.arange(k, dtype=xp.int64)
    if xp is not np:
        c = c.to(r.device)
    m32 = 0xFFFFFFFF
    h = (r * 0x9E3779B1 + c * 0x85EBCA77) & m32
    h = h ^ (h >> 15)
    h = (h * 0x2C1B3C6D) & m32
    h = h ^ (h >> 12)
    return (h & 255).to(xp.float64) / 256.0 - 0.5 if xp is not np else (h & 255) / 256.0 - 0.5


def uniform_edge_weights(g: CSRGraph, lo: float = 0.5, hi: float = 1.5,
                         seed: int = DEFAULT_SEED) -> CSRGraph:
    """Same graph with one U(lo, hi) float32 weight per undirected edge."""
    a, b, _ = undirected_edges(g)
    w = np.random.default_rng(seed).uniform(lo, hi, size=len(a)).astype(np.float32)
    out = from_edges(g.n, a, b, w=w, labels=g.labels, name=g.name + "-w")
    return out
