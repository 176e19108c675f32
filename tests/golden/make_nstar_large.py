"""Writes nstar_large.txt: the oracle's n* for a few samples on lattices too large to rank inside a
test (L = 48: 254.8M sites, L = 64: 1.07G sites).  Calls only the oracle (its Philox order and its
Newman--Ziff sweep); takes about 15 minutes and 20 GB of memory on one core.

    python tests/golden/make_nstar_large.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

CASES = [(48, 1, [1, 7, 127]), (64, 1, [127])]  # (L, seed, masks)


def main():
    lines = ["# n* of the oracle's Newman--Ziff sweep (first n whose new site joins x1 = 0 and x1 = L-1),",
             "# written by make_nstar_large.py from the oracle only.  Columns: L mask seed nstar"]
    for L, seed, masks in CASES:
        t = time.time()
        perm, rk = oracle.rank(L, seed)
        for m in masks:
            lines.append(f"{L} {m} {seed} {oracle.nz(L, m, perm, rk)[0]}")
        del perm, rk
        print(f"L={L} done in {time.time() - t:.0f} s", flush=True)
    with open(os.path.join(HERE, "nstar_large.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
