"""Seeded synthetic inputs for the dual-variable Gibbs sampler.

This module only *draws inputs*: graphs and log-potential tables shaped
like the paper's workloads (Section 6: Ising grids, random graphs,
fully connected Ising) and the larger families the library is measured on
(3-D Potts grid, dense Potts, a batch of Erdos-Renyi graphs,
Barabasi-Albert Potts).  It holds none of the sampler's arithmetic and is
the only module shared by the CPU oracle and the CUDA path.

A model is the pairwise MRF of Section 4 written in log space:

    log p~(x) = sum_v unary[v, x_v] + sum_e pair[e, x_src[e], x_dst[e]]

with every factor exp(.) strictly positive because every log value is
finite.  Arrays are numpy, float32 for potentials and int32 for indices.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np


@dataclasses.dataclass
class Model:
    n_vars: int
    n_labels: int
    unary: np.ndarray          # float32 [N][L]
    src: np.ndarray            # int32 [E]
    dst: np.ndarray            # int32 [E]
    pair: np.ndarray           # float32 [E][L][L], row = label of src
    grid: Optional[Tuple[int, int, int]] = None   # (nx, ny, nz) for lattice models
    name: str = ""

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])

    def check(self) -> None:
        N, L, E = self.n_vars, self.n_labels, self.n_edges
        assert self.unary.shape == (N, L) and self.unary.dtype == np.float32
        assert self.src.shape == (E,) and self.dst.shape == (E,)
        assert self.pair.shape == (E, L, L) and self.pair.dtype == np.float32
        if E:
            assert self.src.min() >= 0 and self.src.max() < N
            assert self.dst.min() >= 0 and self.dst.max() < N
            assert np.all(self.src != self.dst)


def _f32_uniform(rng, lo, hi, size):
    return (rng.random(size, dtype=np.float32) * np.float32(hi - lo) + np.float32(lo)).astype(np.float32)


def _f32_normal(rng, std, size):
    return (rng.standard_normal(size, dtype=np.float32) * np.float32(std)).astype(np.float32)


# ----------------------------------------------------------------------------- lattices

def grid3d_edges(nx: int, ny: int, nz: int):
    """6-neighbour lattice edges.  Site v = x + nx*(y + ny*z).

    Edge order: all x-edges (x, x+1) in (z, y, x) order, then all y-edges,
    then all z-edges.  Each edge is oriented from the lower to the higher
    coordinate."""
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    parts_s, parts_t = [], []
    if nx > 1:
        parts_s.append(idx[:, :, :-1].ravel()); parts_t.append(idx[:, :, 1:].ravel())
    if ny > 1:
        parts_s.append(idx[:, :-1, :].ravel()); parts_t.append(idx[:, 1:, :].ravel())
    if nz > 1:
        parts_s.append(idx[:-1, :, :].ravel()); parts_t.append(idx[1:, :, :].ravel())
    if not parts_s:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return (np.concatenate(parts_s).astype(np.int32), np.concatenate(parts_t).astype(np.int32))


def ising_grid(rows: int = 32, cols: int = 32, h_std: float = 0.5, j_lo: float = 0.0,
               j_hi: float = 0.3, seed: int = 0) -> Model:
    """2-D 4-neighbour Ising grid, L=2.  Spins sigma = 2x-1; unary h_v*sigma,
    coupling J_e*sigma_s*sigma_t with h ~ N(0, h_std^2), J ~ U[j_lo, j_hi].
    Default: the 32x32 weakly coupled grid (1024 sites, 1984 edges)."""
    rng = np.random.default_rng(seed)
    N = rows * cols
    src, dst = grid3d_edges(cols, rows, 1)
    h = _f32_normal(rng, h_std, N)
    J = _f32_uniform(rng, j_lo, j_hi, src.shape[0])
    unary = np.stack([-h, h], axis=1).astype(np.float32)
    sig = np.array([-1.0, 1.0], np.float32)
    pair = (J[:, None, None] * sig[None, :, None] * sig[None, None, :]).astype(np.float32)
    return Model(N, 2, unary, src, dst, pair, grid=(cols, rows, 1), name=f"ising{rows}x{cols}")


def potts_grid3d(nx: int = 128, ny: Optional[int] = None, nz: Optional[int] = None, L: int = 8,
                 w_half: float = 0.3, u_std: float = 1.0, seed: int = 0) -> Model:
    """3-D 6-neighbour grid with random positive L x L tables exp(U[-w_half, w_half])
    and unaries ~ N(0, u_std^2) per label.  Default: 128^3, L=8."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    src, dst = grid3d_edges(nx, ny, nz)
    unary = _f32_normal(rng, u_std, (N, L))
    pair = _f32_uniform(rng, -w_half, w_half, (src.shape[0], L, L))
    return Model(N, L, unary, src, dst, pair, grid=(nx, ny, nz), name=f"potts3d_{nx}x{ny}x{nz}_L{L}")


# ----------------------------------------------------------------------------- dense

def complete_edges(N: int):
    """All pairs s < t in lexicographic order."""
    s, t = np.triu_indices(N, k=1)
    return s.astype(np.int32), t.astype(np.int32)


def dense_potts(N: int = 4096, L: int = 4, w_std: Optional[float] = None, u_std: float = 1.0,
                seed: int = 0) -> Model:
    """Fully connected model with N(0, w_std^2) log-table entries per label
    pair (default w_std = 0.2/sqrt(N)) and N(0, u_std^2) unaries."""
    if w_std is None:
        w_std = 0.2 / math.sqrt(N)
    rng = np.random.default_rng(seed)
    src, dst = complete_edges(N)
    unary = _f32_normal(rng, u_std, (N, L))
    pair = _f32_normal(rng, w_std, (src.shape[0], L, L))
    return Model(N, L, unary, src, dst, pair, name=f"dense_N{N}_L{L}")


def complete_ising(N: int = 100, beta: float = 0.01, seed: int = 0, unary_std: float = 0.0) -> Model:
    """Fully connected Ising model (Section 6, third model): coupling beta*sigma_s*sigma_t."""
    rng = np.random.default_rng(seed)
    src, dst = complete_edges(N)
    h = _f32_normal(rng, unary_std, N) if unary_std > 0 else np.zeros(N, np.float32)
    unary = np.stack([-h, h], axis=1).astype(np.float32)
    sig = np.array([-1.0, 1.0], np.float32)
    pair = np.broadcast_to(np.float32(beta) * sig[:, None] * sig[None, :], (src.shape[0], 2, 2)).astype(np.float32)
    return Model(N, 2, unary, src, dst, pair.copy(), name=f"complete_ising_N{N}")


# ----------------------------------------------------------------------------- random graphs

def _distinct_pairs(rng, N: int, M: int, forbid_keys: Optional[np.ndarray] = None):
    """M distinct unordered pairs {s,t}, s != t, drawn uniformly and returned
    with s < t, avoiding the keys s*N+t listed in forbid_keys."""
    total = N * (N - 1) // 2
    forb = np.unique(forbid_keys) if forbid_keys is not None else np.zeros(0, np.int64)
    M = int(min(M, total - forb.size))
    keys = np.zeros(0, np.int64)
    while keys.size < M:
        need = M - keys.size
        a = rng.integers(0, N, size=int(need * 1.1) + 8)
        b = rng.integers(0, N, size=a.shape[0])
        keep = a != b
        new = np.minimum(a, b)[keep].astype(np.int64) * N + np.maximum(a, b)[keep]
        if forb.size:
            new = new[~np.isin(new, forb)]
        keys = np.concatenate([keys, new])
        _, first = np.unique(keys, return_index=True)
        keys = keys[np.sort(first)]
    keys = keys[:M]
    return (keys // N).astype(np.int32), (keys % N).astype(np.int32)


def random_graph(N: int = 1000, k: int = 2, L: int = 2, w_std: float = 1.0, u_std: float = 1.0,
                 seed: int = 0) -> Model:
    """Random graph with F = k*N distinct pairwise factors (Section 6, second
    model): unary and pairwise log-potentials ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    src, dst = _distinct_pairs(rng, N, k * N)
    unary = _f32_normal(rng, u_std, (N, L))
    pair = _f32_normal(rng, w_std, (src.shape[0], L, L))
    return Model(N, L, unary, src, dst, pair, name=f"random_N{N}_k{k}")


def tiny_random(N: int, L: int, E: int, w_std: float = 1.0, u_std: float = 1.0, seed: int = 0,
                allow_duplicates: bool = False) -> Model:
    """Small random pairwise model for brute-force checks.  With
    allow_duplicates the same (s, t) pair may carry several factors."""
    rng = np.random.default_rng(seed)
    if allow_duplicates:
        a = rng.integers(0, N, size=E); b = (a + 1 + rng.integers(0, N - 1, size=E)) % N
        src, dst = a.astype(np.int32), b.astype(np.int32)
    else:
        src, dst = _distinct_pairs(rng, N, E)
        flip = rng.random(src.shape[0]) < 0.5          # random orientation
        src, dst = np.where(flip, dst, src).astype(np.int32), np.where(flip, src, dst).astype(np.int32)
    unary = _f32_normal(rng, u_std, (N, L))
    pair = _f32_normal(rng, w_std, (src.shape[0], L, L))
    return Model(N, L, unary, src, dst, pair, name=f"tiny_N{N}_L{L}_E{src.shape[0]}")


def tiny_potts(N: int, L: int, E: int, beta_max: float = 0.8, u_std: float = 1.0, seed: int = 0) -> Model:
    """Small Potts model w_e(a,b) = beta_e [a=b] for brute-force checks."""
    rng = np.random.default_rng(seed)
    src, dst = _distinct_pairs(rng, N, E)
    unary = _f32_normal(rng, u_std, (N, L))
    beta = _f32_uniform(rng, 0.0, beta_max, src.shape[0])
    pair = (beta[:, None, None] * np.eye(L, dtype=np.float32)[None]).astype(np.float32)
    return Model(N, L, unary, src, dst, pair, name=f"tinypotts_N{N}_L{L}")


def ferro_potts_grid3d(nx: int = 128, ny: Optional[int] = None, nz: Optional[int] = None, L: int = 8,
                       beta_lo: float = 0.0, beta_hi: float = 1.0, u_std: float = 0.5, seed: int = 0) -> Model:
    """3-D 6-neighbour grid with ferromagnetic Potts tables w_e(a,b) = beta_e [a=b],
    beta_e ~ U[beta_lo, beta_hi], and unaries ~ N(0, u_std^2) (Swendsen-Wang workloads)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    src, dst = grid3d_edges(nx, ny, nz)
    unary = _f32_normal(rng, u_std, (N, L))
    beta = _f32_uniform(rng, beta_lo, beta_hi, src.shape[0])
    pair = np.zeros((src.shape[0], L, L), np.float32)
    pair[:, np.arange(L), np.arange(L)] = beta[:, None]
    return Model(N, L, unary, src, dst, pair, grid=(nx, ny, nz), name=f"ferro3d_{nx}x{ny}x{nz}_L{L}")


def ferro_potts_graph(N: int, L: int, E: int, beta_lo: float = 0.05, beta_hi: float = 1.5, u_std: float = 1.0,
                      p_zero: float = 0.0, seed: int = 0) -> Model:
    """Random graph with generalised ferromagnetic Potts tables w_e(a,b) = beta_{e,a} [a=b]
    (a coupling per label, ~ U[beta_lo, beta_hi]; each set to 0 with probability p_zero)."""
    rng = np.random.default_rng(seed)
    src, dst = _distinct_pairs(rng, N, E)
    unary = _f32_normal(rng, u_std, (N, L))
    beta = _f32_uniform(rng, beta_lo, beta_hi, (src.shape[0], L))
    if p_zero > 0:
        beta[rng.random(beta.shape) < p_zero] = 0.0
    pair = np.zeros((src.shape[0], L, L), np.float32)
    pair[:, np.arange(L), np.arange(L)] = beta
    return Model(N, L, unary, src, dst, pair, name=f"ferro_graph_N{N}_L{L}")


def ba_potts(N: int = 1_000_000, m: int = 5, L: int = 4, beta_max: float = 0.8, u_std: float = 1.0,
             seed: int = 0) -> Model:
    """Barabasi-Albert preferential-attachment graph (m edges per new node,
    seeded by a star on the first m+1 nodes) with Potts factors
    w_e(a,b) = beta_e [a=b], beta_e ~ U[0, beta_max], unaries ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    m0 = m + 1
    src_l = [np.full(m, 0, np.int64)]
    dst_l = [np.arange(1, m0, dtype=np.int64)]
    # repeated-node list: each endpoint appears once per incident edge
    rep = np.zeros(2 * m * N + 2 * m0, np.int64)
    nrep = 0
    for a, b in zip(src_l[0], dst_l[0]):
        rep[nrep] = a; rep[nrep + 1] = b; nrep += 2
    block = 4096
    new_src = np.empty((N - m0) * m, np.int64)
    new_dst = np.empty((N - m0) * m, np.int64)
    pos = 0
    v = m0
    while v < N:
        hi = min(N, v + block)
        # pre-draw plenty of candidate indices for this block of new nodes
        cand = rng.random((hi - v, 4 * m))
        for r in range(hi - v):
            targets = []
            for q in cand[r]:
                tgt = int(rep[int(q * nrep)])
                if tgt not in targets:
                    targets.append(tgt)
                    if len(targets) == m:
                        break
            while len(targets) < m:                       # rare: too many repeats
                tgt = int(rep[int(rng.random() * nrep)])
                if tgt not in targets:
                    targets.append(tgt)
            node = v + r
            for tgt in targets:
                new_src[pos] = tgt; new_dst[pos] = node; pos += 1
                rep[nrep] = tgt; rep[nrep + 1] = node; nrep += 2
        v = hi
    src = np.concatenate([src_l[0], new_src[:pos]]).astype(np.int32)
    dst = np.concatenate([dst_l[0], new_dst[:pos]]).astype(np.int32)
    unary = _f32_normal(rng, u_std, (N, L))
    beta = _f32_uniform(rng, 0.0, beta_max, src.shape[0])
    pair = (beta[:, None, None] * np.eye(L, dtype=np.float32)[None]).astype(np.float32)
    return Model(N, L, unary, src, dst, pair, name=f"ba_N{N}_m{m}_L{L}")


# ----------------------------------------------------------------------------- ER batch

@dataclasses.dataclass
class ErGraphSpec:
    n_vars: int
    n_labels: int
    mean_degree: float
    seed: int


def er_batch_specs(n_graphs: int = 2000, n_min: int = 100, n_max: int = 50000,
                   deg_lo: float = 3.0, deg_hi: float = 20.0, labels=(2, 4, 8, 16), seed: int = 0):
    """Per-graph sizes of the batched dynamic workload: N_g = floor(exp(U[ln n_min,
    ln n_max])), mean degree d_g ~ U[deg_lo, deg_hi], L_g uniform over `labels`."""
    rng = np.random.default_rng(seed)
    n = np.floor(np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_graphs))).astype(np.int64)
    d = rng.uniform(deg_lo, deg_hi, n_graphs)
    Ls = rng.choice(np.array(labels), n_graphs)
    seeds = rng.integers(0, 2**62, n_graphs)
    return [ErGraphSpec(int(n[g]), int(Ls[g]), float(d[g]), int(seeds[g])) for g in range(n_graphs)]


def er_graph(spec: ErGraphSpec, w_half: float = 0.5, u_std: float = 1.0) -> Model:
    """One Erdos-Renyi graph G(N, p) with p = d/(N-1): the edge count is
    Binomial(N(N-1)/2, p) and the edges are distinct uniform pairs.  Tables
    exp(U[-w_half, w_half]) per entry, unaries ~ N(0, u_std^2)."""
    rng = np.random.default_rng(spec.seed)
    N, L = spec.n_vars, spec.n_labels
    total = N * (N - 1) // 2
    p = min(1.0, spec.mean_degree / max(1, N - 1))
    M = int(rng.binomial(total, p))
    src, dst = _distinct_pairs(rng, N, M)
    unary = _f32_normal(rng, u_std, (N, L))
    pair = _f32_uniform(rng, -w_half, w_half, (src.shape[0], L, L))
    return Model(N, L, unary, src, dst, pair, name=f"er_N{N}_L{L}")


def er_edit(model: Model, frac: float, rng: np.random.Generator, w_half: float = 0.5):
    """One edit of the dynamic workload: remove ceil(frac*E) existing edges
    chosen uniformly and add as many new non-duplicate, non-self-loop edges
    with fresh tables.  Returns (remove_positions, add_src, add_dst, add_pair)
    where remove_positions index the model's current edge list."""
    E = model.n_edges
    k = int(math.ceil(frac * E)) if E else 0
    rem = np.sort(rng.choice(E, size=k, replace=False)) if k else np.zeros(0, np.int64)
    N = model.n_vars
    existing = (np.minimum(model.src, model.dst).astype(np.int64) * N
                + np.maximum(model.src, model.dst))
    s, t = _distinct_pairs(rng, N, k, forbid_keys=existing)
    pair = _f32_uniform(rng, -w_half, w_half, (s.shape[0], model.n_labels, model.n_labels))
    return rem.astype(np.int64), s, t, pair


class ErBatchEdits:
    """Edits of the batched dynamic workload for all graphs at once, with the
    distributions of er_edit: every round removes ceil(frac E_g) edges of every
    graph g chosen uniformly, and adds as many new distinct pairs {s, t},
    s < t, absent from the graph (its edges before the round), with tables
    exp(U[-w_half, w_half]).  Keeps each graph's edge list (graph-local
    endpoints and the batch's class slots) and the sorted keys of all edges,
    key = base_g + s N_g + t, so that a round costs O(edits + sum E_g) numpy
    work and no table is kept on the host."""

    def __init__(self, models, first_slots, seed: int = 1, w_half: float = 0.5):
        self.G = len(models)
        self.n = np.array([m.n_vars for m in models], np.int64)
        self.L = np.array([m.n_labels for m in models], np.int64)
        self.base = np.concatenate([[0], np.cumsum(self.n * self.n)[:-1]]).astype(np.int64)
        self.lo = [np.minimum(m.src, m.dst).astype(np.int32) for m in models]
        self.hi = [np.maximum(m.src, m.dst).astype(np.int32) for m in models]
        self.src = [m.src.astype(np.int32) for m in models]
        self.dst = [m.dst.astype(np.int32) for m in models]
        self.slot = [np.arange(m.n_edges, dtype=np.int64) + int(first_slots[g]) for g, m in enumerate(models)]
        self.keys = np.sort(np.concatenate([self.base[g] + self.lo[g].astype(np.int64) * self.n[g] + self.hi[g]
                                            for g in range(self.G)]))
        self.rng = np.random.default_rng(seed)
        self.w_half = w_half
        self._pending = None

    def n_edges(self):
        return int(sum(len(s) for s in self.src))

    def counts(self, frac: float):
        """Removals (= additions) of every graph in one round."""
        return np.array([int(math.ceil(frac * len(s))) if len(s) else 0 for s in self.src], np.int64)

    def edit(self, frac: float = 0.01):
        """Arrays of one round for the batch's edit calls: (remove_graph,
        remove_slot, add_graph, add_src, add_dst, add_tables_flat)."""
        rng, G = self.rng, self.G
        k = self.counts(frac)
        rem = [np.sort(rng.choice(len(self.src[g]), size=int(k[g]), replace=False)) if k[g] else
               np.zeros(0, np.int64) for g in range(G)]
        # additions: candidate pairs for the missing count of every graph until all are met
        acc_keys = np.zeros(0, np.int64)
        acc_g = np.zeros(0, np.int64)
        missing = k.copy()
        while missing.sum() > 0:
            gid = np.repeat(np.arange(G, dtype=np.int64), missing)
            a = np.floor(rng.random(gid.shape[0]) * self.n[gid]).astype(np.int64)
            b = np.floor(rng.random(gid.shape[0]) * self.n[gid]).astype(np.int64)
            ok = a != b
            gid, a, b = gid[ok], a[ok], b[ok]
            key = self.base[gid] + np.minimum(a, b) * self.n[gid] + np.maximum(a, b)
            pos = np.searchsorted(self.keys, key)
            fresh = (pos >= self.keys.shape[0]) | (self.keys[np.minimum(pos, self.keys.shape[0] - 1)] != key)
            acc_keys = np.concatenate([acc_keys, key[fresh]])
            acc_g = np.concatenate([acc_g, gid[fresh]])
            _, first = np.unique(acc_keys, return_index=True)
            first = np.sort(first)
            acc_keys, acc_g = acc_keys[first], acc_g[first]
            # keep at most k_g per graph (in draw order)
            order = np.argsort(acc_g, kind="stable")
            acc_keys, acc_g = acc_keys[order], acc_g[order]
            starts = np.searchsorted(acc_g, np.arange(G))
            rank = np.arange(acc_g.shape[0]) - starts[acc_g]
            keep = rank < k[acc_g]
            acc_keys, acc_g = acc_keys[keep], acc_g[keep]
            missing = k - np.bincount(acc_g, minlength=G)
        local = acc_keys - self.base[acc_g]
        s_new = (local // self.n[acc_g]).astype(np.int32)
        t_new = (local % self.n[acc_g]).astype(np.int32)
        tables = _f32_uniform(rng, -self.w_half, self.w_half, int((self.L[acc_g] ** 2).sum()))
        rm_g = np.repeat(np.arange(G, dtype=np.int32), k)
        rm_slot = np.concatenate([self.slot[g][rem[g]] for g in range(G)]) if G else np.zeros(0, np.int64)
        self._pending = (k, rem, acc_g, s_new, t_new)
        return (rm_g, rm_slot.astype(np.int64), acc_g.astype(np.int32), s_new, t_new, tables)

    def apply(self, new_slots):
        """Record the round once the batch has applied it (new_slots: the
        class slots of the additions, in the order of edit's arrays)."""
        k, rem, acc_g, s_new, t_new = self._pending
        starts = np.concatenate([[0], np.cumsum(k)])
        rm_keys = []
        for g in range(self.G):
            r = rem[g]
            rm_keys.append(self.base[g] + self.lo[g][r].astype(np.int64) * self.n[g] + self.hi[g][r])
            keep = np.ones(len(self.src[g]), bool)
            keep[r] = False
            a, b = s_new[starts[g]:starts[g + 1]], t_new[starts[g]:starts[g + 1]]
            self.src[g] = np.concatenate([self.src[g][keep], a])
            self.dst[g] = np.concatenate([self.dst[g][keep], b])
            self.lo[g] = np.concatenate([self.lo[g][keep], np.minimum(a, b)])
            self.hi[g] = np.concatenate([self.hi[g][keep], np.maximum(a, b)])
            self.slot[g] = np.concatenate([self.slot[g][keep], np.asarray(new_slots[starts[g]:starts[g + 1]], np.int64)])
        rmk = np.sort(np.concatenate(rm_keys)) if rm_keys else np.zeros(0, np.int64)
        keys = np.delete(self.keys, np.searchsorted(self.keys, rmk))
        add = np.sort(self.base[acc_g] + np.minimum(s_new, t_new).astype(np.int64) * self.n[acc_g]
                      + np.maximum(s_new, t_new))
        self.keys = np.insert(keys, np.searchsorted(keys, add), add)
        self._pending = None


# ----------------------------------------------------------------------------- blocks

def adjacency(n_vars: int, src: np.ndarray, dst: np.ndarray):
    """Undirected neighbour lists as CSR (ptr [N+1], nbr [2E]), neighbours of
    each site in edge order."""
    a = np.concatenate([src, dst]).astype(np.int64)
    b = np.concatenate([dst, src]).astype(np.int64)
    order = np.argsort(a, kind="stable")
    ptr = np.zeros(n_vars + 1, np.int64)
    ptr[1:] = np.cumsum(np.bincount(a, minlength=n_vars))
    return ptr, b[order]


def bfs_blocks(model: Model, block: int = 16, seed: int = 0) -> np.ndarray:
    """Partition the sites into connected blocks of at most `block` sites,
    grown breadth-first from unassigned seeds taken in a seeded random order.
    Returns the block id of every site (int32 [N])."""
    N = model.n_vars
    rng = np.random.default_rng(seed)
    ptr, nbr = adjacency(N, model.src, model.dst)
    ptr = ptr.tolist(); nbr = nbr.tolist()
    bid = [-1] * N
    nb = 0
    for s in rng.permutation(N).tolist():
        if bid[s] >= 0:
            continue
        members = [s]; bid[s] = nb; head = 0
        while head < len(members) and len(members) < block:
            v = members[head]; head += 1
            for w in nbr[ptr[v]:ptr[v + 1]]:
                if bid[w] < 0:
                    bid[w] = nb; members.append(w)
                    if len(members) == block:
                        break
        nb += 1
    return np.asarray(bid, np.int32)
