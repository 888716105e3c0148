"""Write capped_quality.json: the CPU oracle's whole multilevel runs with a
per-row neighbour cap of the distance matrix (korder_capped; Sec. 3.2.1 with
the cap that keeps large k feasible), one line per seed, with the
neighbourhood preservation and normalised stress (Sec. 4.1) of each layout.

The GPU's capped whole-run test compares its own runs' statistics with
these.  Only graphgen (seeded inputs) and oracle/ run here.

  python tests/golden/make_capped_quality.py [--procs N]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

GRAPH = dict(gen="barabasi_albert", args=[3000, 3, 2])
PARAMS = dict(k=3, M=5, epochs=100, b=1.0, stop_nodes=500, row_cap=30, mode=0)
SEEDS = 96


def one(seed):
    import graphgen as gg
    import oracle as orc
    n, s, d = getattr(gg, GRAPH["gen"])(*GRAPH["args"])
    Y = orc.run(n, s, d, orc.Params(**PARAMS, seed=seed))
    rp, col = orc.canonical_graph(n, s, d)
    return seed, orc.neighbourhood_preservation(rp, col, Y, 2), orc.stress(rp, col, Y)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import oracle as orc
    orc.build()
    t0 = time.time()
    out = {}
    with mp.get_context("spawn").Pool(args.procs) as pool:
        for seed, npv, st in pool.imap_unordered(one, range(SEEDS)):
            out[seed] = [npv, st]
    rec = {"graph": GRAPH, "params": PARAMS, "seeds": SEEDS, "runs": [out[sd] for sd in range(SEEDS)],
           "note": "oracle whole runs with capped rows (NP, stress) per seed, written by make_capped_quality.py"}
    with open(os.path.join(HERE, "capped_quality.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(f"{SEEDS} runs in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
