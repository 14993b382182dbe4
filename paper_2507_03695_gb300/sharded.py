"""Edges sharded over ranks with one Reducer step (Section III, "High-Level
Algorithm"; Algorithm 2).

The edge list is cut into edge-balanced contiguous slices, one per rank
(Algorithm 2 partitions the graph by rank). Each rank runs the whole JT pass
on its slice with a private parent array over all vertices, flattens it
(pointer jumping), and sends its forest -- the pairs (v, parent of v) of its
non-root vertices, at most n per rank -- to the Reducer, which processes the
received pairs like graph edges in one more pass and flattens: its labels are
the labels of the whole graph. The exchange is the paper's single
communication step; its volume is at most min(E, (ranks - 1) * n) pairs
(Section V, analysis). Every computation runs in the library's kernels; this
module only slices, gathers and hands buffers to the C ABI.

The gather uses torch.distributed (NCCL between GPUs). Host-side helpers
(`edge_range`, `gather_to_reducer`) work on any backend and on CPU tensors.
"""
from __future__ import annotations

from . import binding as _b


def edge_range(n_edges: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of rank's edge-balanced contiguous slice: the first
    n_edges % world ranks take one edge more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    q, r = divmod(n_edges, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def shard_forest(n_vertices: int, edges_slice, stream=None, graph=None, **options):
    """The JT pass over one rank's slice on a private parent array, pointer
    jumping, and the forest as an (count, 2) int32 device tensor of
    (v, root of v) pairs. `graph`: a Graph on n_vertices to reuse (else one
    is created with `options` and freed)."""
    if graph is not None:
        graph.run(edges_slice, None, stream)  # ends with pointer jumping: P holds root names
        return graph.forest_pairs(stream)
    with _b.Graph(n_vertices, **options) as g:
        g.run(edges_slice, None, stream)
        return g.forest_pairs(stream).clone()


def gather_to_reducer(pairs_local, dist, reducer: int = 0):
    """Concatenation of every rank's (count, 2) pair tensor, on the reducer
    rank (None elsewhere). Counts are exchanged first; the pair lists are
    padded to the largest count for one all-gather and trimmed afterwards."""
    import torch
    world = dist.get_world_size()
    if world == 1:
        return pairs_local
    dev = pairs_local.device
    count = torch.tensor([pairs_local.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(count) for _ in range(world)]
    dist.all_gather(counts, count)
    counts = [int(c.item()) for c in counts]
    width = max(max(counts), 1)
    padded = torch.zeros((width, 2), dtype=torch.int32, device=dev)
    padded[: pairs_local.shape[0]] = pairs_local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded)
    if dist.get_rank() != reducer:
        return None
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def reduce_forests(n_vertices: int, pairs_all, labels_out=None, stream=None, graph=None, **options):
    """The Reducer: one JT pass over the gathered pairs, then pointer jumping
    into labels_out (uint32[n_vertices] as an int32 device tensor).
    `graph`: a Graph on n_vertices to reuse."""
    if graph is not None:
        graph.run(pairs_all, labels_out, stream)
        graph.sync()
        return labels_out
    with _b.Graph(n_vertices, **options) as g:
        g.run(pairs_all, labels_out, stream)
        g.sync()
    return labels_out


def run_sharded(n_vertices: int, edges_local, dist, labels_out=None, reducer: int = 0, stream=None,
                graph=None, reducer_graph=None, **options):
    """One sharded computation: this rank's slice -> its forest -> the
    Reducer's pass. Returns labels_out on the reducer rank, None elsewhere."""
    pairs = shard_forest(n_vertices, edges_local, stream, graph, **options)
    pairs_all = gather_to_reducer(pairs, dist, reducer)
    if pairs_all is None:
        return None
    return reduce_forests(n_vertices, pairs_all, labels_out, stream, reducer_graph, **options)
