"""Writes the disorder range of the 1.015e9-site honeycomb workload (22528 x 22528 cells,
W = 1 eV, lattice seed 0x7B1A5) with the oracle's own disorder draw: the smallest and largest
q_i = u_i >> 8 over all 2 x 22528 x 22528 sites, u_i the disorder-stream Philox draw of site i,
so that V_i = W (q_i 2^-24 - 1/2).  The oracle needs the whole lattice's Gershgorin bounds to
rescale H on a window of it; evaluating them takes every site, so they are stored.

Run from the repository root:  python tests/golden/make_disorder_range.py
Calls only oracle/ (the Philox generator of the disorder stream).
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(ROOT, "tests", "golden", "honeycomb22528_W1_disorder_range.json")
LX = LY = 22528
SEED = 0x7B1A5
W = 1.0
CHUNK = 1 << 24


def chunk_range(bounds):
    sys.path.insert(0, ROOT)
    from oracle.philox import draw_u32, STREAM_DISORDER
    lo, hi = bounds
    u = draw_u32(SEED, np.arange(lo, hi, dtype=np.uint64), STREAM_DISORDER)
    q = u >> np.uint32(8)
    return int(q.min()), int(q.max())


def main():
    n = 2 * LX * LY
    parts = [(a, min(n, a + CHUNK)) for a in range(0, n, CHUNK)]
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(chunk_range, parts)
    qmin = min(r[0] for r in res)
    qmax = max(r[1] for r in res)
    rec = {"lattice": {"kind": "honeycomb", "L": [LX, LY], "W": W, "seed": SEED, "sites": n},
           "q_min": qmin, "q_max": qmax,
           "V_min": W * (qmin * 2.0 ** -24 - 0.5), "V_max": W * (qmax * 2.0 ** -24 - 0.5),
           "definition": "q_i = (Philox4x32-10 disorder draw of site i) >> 8, V_i = W (q_i 2^-24 - 1/2)",
           "writer": "tests/golden/make_disorder_range.py (oracle.philox only)"}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
