"""Write tests/golden/sc_exact_small.json.

Exact spanning centrality of a few small hand-written graphs, by Definition 2.1
itself: every (n-1)-edge subset is enumerated and the spanning trees holding
each edge are counted (oracle.exact.kirchhoff_bruteforce). Calls only the
oracle. Re-run with:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
from oracle import exact  # noqa: E402

CASES = {
    # name: (n, undirected edge list)
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4)]),
    "diamond": (4, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)]),
    "wheel5": (6, [(0, 1), (0, 2), (0, 3), (0, 4), (0, 5), (1, 2), (2, 3), (3, 4), (4, 5), (5, 1)]),
    "kite_tail": (6, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3), (3, 4), (4, 5)]),
    "theta": (7, [(0, 1), (1, 2), (2, 6), (0, 3), (3, 6), (0, 4), (4, 5), (5, 6)]),
}


def main():
    out = {"source": "Definition 2.1 by exhaustive spanning-tree enumeration", "cases": []}
    for name, (n, edges) in CASES.items():
        g = gg.from_edges(n, [a for a, _ in edges], [b for _, b in edges])
        sc = exact.kirchhoff_bruteforce(g.n, g.row_ptr, g.col_idx)
        keys = sorted(sc)
        out["cases"].append({"name": name, "n": n, "edges": [list(e) for e in edges],
                             "edges_sorted": [list(k) for k in keys],
                             "sc": [f"{sc[k].numerator}/{sc[k].denominator}" for k in keys]})
    with open(os.path.join(HERE, "sc_exact_small.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
