"""Accuracy of the K-Best search on the seeded workloads, computed with the oracle alone.

TEST INFRASTRUCTURE: this script calls only the oracle (and the seeded input generators);
the GPU path is bit-identical to the oracle, so every figure here also describes it.

K-Best returns the cost of one complete vertex map, an upper bound on the GED that becomes
exact once K is at least the widest level (Sec. 4.1). Three measurements:

  exact     the 200-pair tiny batch (5-8 vertices, unit costs): how often the result equals
            the exact GED (brute force over every injective partial map, Sec. 2.2) and the
            mean relative excess, for a sweep of K, both branching orders (index order as in
            Algorithm 1, and the descending-degree extension) and both final steps
            (variant A: the best K leaves are completed; variant B: every last-level
            successor is completed)
  identity  how often d(G, G) = 0 at the batch's own K (zero-cost partial maps tie, and a
            beam cut among ties can lose the identity map)
  symmetry  how often d(g1, g2) = d(g2, g1) at the batch's own K (the costs are symmetric:
            deletion and insertion cost the same, so the exact GED is symmetric; the beam
            branches only the source graph, so K-Best need not be)

Run:  python oracle/accuracy_report.py [--pairs-tiny 200] [--pairs-molecule 400] [--threads N]
"""
from __future__ import annotations

import argparse
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from oracle import oracle as O                      # noqa: E402
from paper_2605_00830_gb300 import workloads as W   # noqa: E402


def _pmap(fn, items, threads):
    if threads <= 1:
        return [fn(x) for x in items]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, items))


def exact_sweep(w, ks, threads):
    """Rows (K, order, variant, exact rate, mean relative excess, worst excess)."""
    pairs = [(w.graphs[int(a)], w.graphs[int(b)]) for a, b in w.pairs]
    ged = np.array(_pmap(lambda gb: O.brute_ged(gb[0], gb[1], w.cost)[0], pairs, threads))
    rows = []
    for K in ks:
        for order in (0, 1):
            for variant in ((0, 1) if K == w.K else (0,)):
                got = np.array(_pmap(lambda gb: O.kbest(gb[0], gb[1], w.cost, K, variant,
                                                        order=order)[0], pairs, threads))
                assert (got >= ged).all(), "K-Best went below the exact GED"
                rel = np.where(ged > 0, (got - ged) / np.maximum(ged, 1), 0.0)
                rows.append((K, order, variant, float((got == ged).mean()),
                             float(rel.mean()), int((got - ged).max())))
    return rows, ged


def identity_rate(graphs, cost, K, threads, order=0):
    got = _pmap(lambda g: O.kbest(g, g, cost, K, order=order)[0], graphs, threads)
    return float(np.mean([c == 0 for c in got])), len(got)


def symmetry_rate(w, K, threads, order=0):
    pairs = [(w.graphs[int(a)], w.graphs[int(b)]) for a, b in w.pairs]
    fwd = _pmap(lambda gb: O.kbest(gb[0], gb[1], w.cost, K, order=order)[0], pairs, threads)
    bwd = _pmap(lambda gb: O.kbest(gb[1], gb[0], w.cost, K, order=order)[0], pairs, threads)
    fwd, bwd = np.array(fwd), np.array(bwd)
    return float((fwd == bwd).mean()), float(np.abs(fwd - bwd).mean()), len(pairs)


def k_gain(w, K, K_big, threads):
    """How much a much wider beam changes the result on pairs too large for brute force:
    (share of pairs lowered, mean relative drop, share of pairs raised, #pairs). K-Best is
    not monotone in K, so a wider beam can also end on a worse leaf."""
    pairs = [(w.graphs[int(a)], w.graphs[int(b)]) for a, b in w.pairs]
    a = np.array(_pmap(lambda gb: O.kbest(gb[0], gb[1], w.cost, K)[0], pairs, threads))
    b = np.array(_pmap(lambda gb: O.kbest(gb[0], gb[1], w.cost, K_big)[0], pairs, threads))
    better = b < a
    rel = np.where(a > 0, (a - b) / np.maximum(a, 1), 0.0)
    return float(better.mean()), float(rel.mean()), float((b > a).mean()), len(pairs)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--pairs-tiny", type=int, default=200)
    ap.add_argument("--pairs-molecule", type=int, default=400)
    ap.add_argument("--ks", default="1,4,16,64,256,1024")
    ap.add_argument("--k-big", type=int, default=5000)
    args = ap.parse_args(argv)
    t0 = time.time()

    w1 = W.config1(args.pairs_tiny)
    rows, ged = exact_sweep(w1, [int(k) for k in args.ks.split(",")], args.threads)
    print(f"tiny ER batch: {w1.n_pairs} pairs, 5-8 vertices, unit costs; "
          f"exact GED by brute force (mean {ged.mean():.2f})")
    print("| K | order | final step | exact | mean relative excess | worst excess |")
    print("|---|---|---|---|---|---|")
    for K, order, variant, ex, rel, worst in rows:
        print(f"| {K} | {'degree' if order else 'index'} | {'B' if variant else 'A'} | "
              f"{100 * ex:.1f} % | {100 * rel:.2f} % | {worst} |")

    g1 = [w1.graphs[i] for i in range(len(w1.graphs))]
    idr, n = identity_rate(g1, w1.cost, w1.K, args.threads)
    sr, sd, ns = symmetry_rate(w1, w1.K, args.threads)
    print(f"tiny ER batch, K = {w1.K}: d(G,G) = 0 for {100 * idr:.1f} % of {n} graphs; "
          f"d(g1,g2) = d(g2,g1) for {100 * sr:.1f} % of {ns} pairs (mean |diff| {sd:.3f})")

    w2 = W.config2(args.pairs_molecule)
    g2 = [w2.graphs[i] for i in range(len(w2.graphs))]
    for order in (0, 1):
        idr, n = identity_rate(g2, w2.cost, w2.K, args.threads, order)
        sr, sd, ns = symmetry_rate(w2, w2.K, args.threads, order)
        print(f"molecule-like batch (first {w2.n_pairs} pairs), K = {w2.K}, "
              f"{'degree' if order else 'index'} order: d(G,G) = 0 for {100 * idr:.1f} % "
              f"of {n} graphs; d(g1,g2) = d(g2,g1) for {100 * sr:.1f} % of {ns} pairs "
              f"(mean |diff| {sd:.3f})")
    wk = W.subset(w2, range(min(100, w2.n_pairs)))
    better, rel, worse, nk = k_gain(wk, w2.K, args.k_big, args.threads)
    print(f"molecule-like batch (first {nk} pairs): K = {args.k_big} lowers the K = {w2.K} "
          f"result on {100 * better:.1f} % of pairs (mean relative drop {100 * rel:.2f} %), "
          f"raises it on {100 * worse:.1f} %")
    print(f"({time.time() - t0:.0f} s on {args.threads} threads)")
    return rows


if __name__ == "__main__":
    main()
