#!/usr/bin/env python
"""Writes the stored K-Best results that the full-batch GPU parity tests compare against.

Every value in the files this script writes comes from the CPU oracle (`oracle/`) run on the
seeded synthetic workloads of `paper_2605_00830_gb300/workloads.py`; nothing here touches the
CUDA path. One file per target, `tests/golden/kbest_<target>.txt`:

    # <description>
    # target <name>; written by: python tests/golden/make_kbest_golden.py <name>
    # columns: pair cost n_evals map_digest
    0 123 456789 0123456789abcdef
    ...

`map_digest` is the 64-bit BLAKE2b digest of the pair's vertex map (g2 image of every g1
vertex, -1 = deleted) as little-endian int32: equal digests mean equal maps, so a test
compares cost, evaluation count and map of every pair without storing the maps themselves.

Usage: python tests/golden/make_kbest_golden.py [target ...] [--threads N]
(no target: every target; the large ones take many minutes of host CPU).
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2605_00830_gb300 import workloads as W  # noqa: E402


def map_digest(mapping) -> str:
    """64-bit BLAKE2b digest of a vertex map as little-endian int32."""
    a = np.ascontiguousarray(np.asarray(mapping, dtype="<i4"))
    return hashlib.blake2b(a.tobytes(), digest_size=8).hexdigest()


def _size_sweep(n, n_pairs):
    return lambda: W.config_size_sweep(n_pairs=n_pairs, n=n)


# name -> (workload constructor, description). Each workload carries its own K (or per-pair
# K) and cost model; every target runs variant A in index order, as the batches do.
TARGETS = {
    "config2": (lambda: W.config2(),
                "config 2: 20,000 molecule-like pairs (10-40 vertices), setting-1 costs, K = 100, seed 2"),
    "config3": (lambda: W.config3(),
                "config 3: 4,096 dense ER pairs (50-200 vertices), unit costs, K = 256, seed 3"),
    "config4": (lambda: W.config4(),
                "config 4: 64 BA pairs (500-1,000 vertices), unit costs, K = 1024, seed 4"),
    "config5_2000": (lambda: W.config5(max_requests=2000),
                     "config 5: the first 2,000 queries of the 5,000 req/s serving stream, "
                     "each at its drawn K in {32, 128, 512}, setting-1 costs, seed 5"),
    "widebeam": (lambda: W.config_wide_beam(),
                 "wide beam: 16 molecule-like pairs (18-22 vertices), setting-1 costs, K = 100,000, seed 6"),
    "sizesweep_200": (_size_sweep(200, 2),
                      "size sweep: 2 pairs of G(200, 0.4) graphs, 4 labels, setting-1 costs, K = 5,000, seed 7"),
    "sizesweep_300": (_size_sweep(300, 2),
                      "size sweep: 2 pairs of G(300, 0.4) graphs, 4 labels, setting-1 costs, K = 5,000, seed 7"),
    "sizesweep_500": (_size_sweep(500, 1),
                      "size sweep: 1 pair of G(500, 0.4) graphs, 4 labels, setting-1 costs, K = 5,000, seed 7"),
    "sizesweep_950": (_size_sweep(950, 1),
                      "size sweep: 1 pair of G(950, 0.4) graphs, 4 labels, setting-1 costs, K = 5,000, seed 7"),
}


def golden_path(name: str) -> str:
    return os.path.join(HERE, f"kbest_{name}.txt")


def load(name: str):
    """(pair index array, cost, n_evals, digests) of a stored target."""
    idx, cost, nev, dig = [], [], [], []
    with open(golden_path(name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, b, c, d = line.split()
            idx.append(int(a))
            cost.append(int(b))
            nev.append(int(c))
            dig.append(d)
    return np.array(idx), np.array(cost, np.int64), np.array(nev, np.int64), dig


def write(name: str, threads: int) -> None:
    from oracle import oracle as O   # the oracle is the only source of the stored values

    make, desc = TARGETS[name]
    w = make()
    # heaviest pairs first so that the pool's last tasks are short
    est = [w.graphs[int(a)].n * w.graphs[int(b)].n ** 2 *
           (int(w.k_per_pair[p]) if w.k_per_pair is not None else w.K)
           for p, (a, b) in enumerate(w.pairs)]
    order = list(np.argsort(est)[::-1])
    t0 = time.time()
    res = O.kbest_workload(w, order, threads=threads)
    by_pair = {int(p): r for p, r in zip(order, res)}
    tmp = golden_path(name) + ".tmp"
    with open(tmp, "w") as f:
        f.write(f"# {desc}\n")
        f.write(f"# target {name}; written by: python tests/golden/make_kbest_golden.py {name}\n")
        f.write("# columns: pair cost n_evals map_digest "
                "(64-bit BLAKE2b of the map as little-endian int32, -1 = deleted)\n")
        for p in range(w.n_pairs):
            c, m, n = by_pair[p]
            f.write(f"{p} {c} {n} {map_digest(m)}\n")
    os.replace(tmp, golden_path(name))
    print(f"{name}: {w.n_pairs} pairs in {time.time() - t0:.1f} s", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("targets", nargs="*")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    for name in a.targets or list(TARGETS):
        write(name, a.threads)


if __name__ == "__main__":
    main()
