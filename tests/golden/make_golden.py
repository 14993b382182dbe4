"""Writes the stored expected values of the full-size workloads.

Calls only the CPU oracle (oracle/) on inputs from the seeded generators
(graphgen/); nothing here touches the CUDA path. For each workload it stores
the SHA-256 of the generated edge array (to detect generator drift between
machines), the SHA-256 of the oracle's min-id label array, the component
count, the oracle's maximum-degree vertex m, the SHA-256 of the root-value
labels under that m (Eq. 1), and a few sampled labels.

Usage: python tests/golden/make_golden.py rmat24_ef16 grid8192x8192_p0.9 [rmat28_ef16 batch4096 serving_rmat26 ...]
Large R-MAT inputs are generated and fed to the oracle in chunks.
"""
from __future__ import annotations

import hashlib
import json
import os
import re
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

CHUNK = 1 << 26


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8)).hexdigest()


def golden_for(w: graphgen.Workload) -> dict:
    t0 = time.time()
    n = w.n_vertices
    h_edges = hashlib.sha256()
    uf = oracle.StreamingUnionFind(n)
    deg = np.zeros(n, dtype=np.uint64)
    if w.kind == "rmat":
        total = w.n_edges
        for b in range(0, total, CHUNK):
            e = graphgen.rmat(w.scale, total, w.seed, w.scramble, b, min(total, b + CHUNK))
            h_edges.update(e.view(np.uint8))
            uf.add(e)
            oracle.degree_add(n, e, deg)
        chunks_for_rv = lambda: (graphgen.rmat(w.scale, total, w.seed, w.scramble, b, min(total, b + CHUNK))  # noqa: E731
                                 for b in range(0, total, CHUNK))
    else:
        e_all = w.host_edges()
        total = len(e_all)
        h_edges.update(e_all.view(np.uint8))
        uf.add(e_all)
        oracle.degree_add(n, e_all, deg)
        chunks_for_rv = lambda: iter([e_all])  # noqa: E731
    L = uf.min_labels()
    uf.close()
    m = int(np.flatnonzero(deg == deg.max())[0])
    # root-value labels under Eq. 1 with the planted vertex m
    Lr = np.where(L == L[m], 0, L + 1).astype(np.uint32)
    # ... and computed independently by the R-ordered union-find when the input fits
    if total <= (1 << 29):
        e_cat = np.concatenate(list(chunks_for_rv()))
        Lr2 = oracle.root_value_labels(n, e_cat, m)
        assert np.array_equal(Lr, Lr2)
        del e_cat
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(n, size=min(64, n), replace=False))
    return {
        "workload": w.name,
        "n_vertices": n,
        "n_edges": int(total),
        "edges_sha256": h_edges.hexdigest(),
        "labels_min_id_sha256": sha(L),
        "num_components": int(oracle.num_components(L)),
        "max_degree_vertex": m,
        "max_degree": int(deg[m]),
        "labels_root_value_sha256": sha(Lr),
        "giant_component_size": int(np.count_nonzero(L == L[m])),
        "sample_vertices": sample.tolist(),
        "sample_min_id_labels": L[sample].tolist(),
        "oracle_seconds": round(time.time() - t0, 1),
    }


def golden_batch(n_graphs: int, seed: int) -> dict:
    t0 = time.time()
    b = graphgen.batch(n_graphs, seed)
    L = oracle.batch_min_labels(b.edges, b.vtx_off, b.edge_off)
    return {
        "workload": f"batch{n_graphs}", "n_graphs": n_graphs, "seed": seed,
        "n_vertices": int(b.vtx_off[-1]), "n_edges": int(b.edge_off[-1]),
        "edges_sha256": sha(b.edges), "labels_sha256": sha(L),
        "num_components": int(np.count_nonzero(L == (np.arange(len(L), dtype=np.int64)
                                                     - np.repeat(b.vtx_off[:-1].astype(np.int64),
                                                                 np.diff(b.vtx_off.astype(np.int64)))))),
        "oracle_seconds": round(time.time() - t0, 1),
    }


def serving_schedule(n_pool: int) -> list:
    """The inserts of the full-size serving check, as (offset, count) slices of
    one pool of uniform pairs: the bench's executor burst (512 batches of 2^17
    pairs) and four side-path inserts of 2^20 pairs (at least 2^18 pairs each,
    so the server runs them as full edge passes on a side stream)."""
    size, span = 1 << 17, n_pool - (1 << 17)
    sched = [((i * 104729) % span, size) for i in range(512)]
    sched += [(n_pool - (k + 1) * (1 << 20), 1 << 20) for k in range(4)]
    return sched


def golden_serving() -> dict:
    """Resident R-MAT scale 26 (the serving configuration's graph) after the
    inserts of serving_schedule: the labels are those of the union of the
    graph's edges and every inserted pair (inserts commute)."""
    t0 = time.time()
    w = graphgen.RMAT26
    n, total = w.n_vertices, w.n_edges
    pool_n, pool_seed = 1 << 26, 61
    pool = graphgen.pairs(n, pool_n, pool_seed)
    sched = serving_schedule(pool_n)
    uf = oracle.StreamingUnionFind(n)
    h_edges = hashlib.sha256()
    for b in range(0, total, CHUNK):
        e = graphgen.rmat(w.scale, total, w.seed, w.scramble, b, min(total, b + CHUNK))
        h_edges.update(e.view(np.uint8))
        uf.add(e)
    for off, cnt in sched:
        uf.add(pool[off:off + cnt])
    L = uf.min_labels()
    uf.close()
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(n, size=64, replace=False))
    return {
        "workload": "serving_rmat26", "graph": w.name, "n_vertices": n, "n_edges": int(total),
        "edges_sha256": h_edges.hexdigest(),
        "pool_pairs": pool_n, "pool_seed": pool_seed, "pool_sha256": sha(pool),
        "inserts": [[int(o), int(c)] for o, c in sched],
        "labels_min_id_sha256": sha(L), "num_components": int(oracle.num_components(L)),
        "sample_vertices": sample.tolist(), "sample_min_id_labels": L[sample].tolist(),
        "oracle_seconds": round(time.time() - t0, 1),
    }


def main(names):
    for name in names:
        if name == "serving_rmat26":
            g = golden_serving()
            path = os.path.join(HERE, f"{name}.json")
            text = json.dumps(g, indent=1)
            # one line per (offset, count) insert slice
            text = re.sub(r"\[\n\s+(\d+),\n\s+(\d+)\n\s+\]", r"[\1, \2]", text)
            with open(path, "w") as f:
                f.write(text + "\n")
            print(path, g["num_components"], g["oracle_seconds"], "s")
            continue
        if name == "batch4096":
            g = golden_batch(graphgen.BATCH_GRAPHS, graphgen.BATCH_SEED)
            path = os.path.join(HERE, f"{name}.json")
            with open(path, "w") as f:
                json.dump(g, f, indent=1)
                f.write("\n")
            print(path, g["num_components"], g["oracle_seconds"], "s")
            continue
        w = graphgen.WORKLOADS[name]
        g = golden_for(w)
        path = os.path.join(HERE, f"{name}.json")
        with open(path, "w") as f:
            json.dump(g, f, indent=1)
            f.write("\n")
        print(path, g["num_components"], g["oracle_seconds"], "s")


if __name__ == "__main__":
    main(sys.argv[1:] or ["rmat16_ef16", "rmat24_ef16", "grid8192x8192_p0.9"])
