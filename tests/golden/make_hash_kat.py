"""Writes hash_kat.txt: known answers for the IBLT cell/checksum convention.

Calls only ``oracle`` (and ``ppgen`` for the key values).  The convention is
one the paper leaves open (it asks for r hash functions and a pseudorandom
checkSum, Sec. 6); this file freezes it so that both sides can be held to it.

Run from the repository root:  python tests/golden/make_hash_kat.py
"""
import os
import sys

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

import oracle  # noqa: E402
import ppgen  # noqa: E402

CASES = [(1 << 26, 3, 0x13027014), (4096, 4, 7), (1000, 3, 1), (257, 5, 123456789),
         (3, 3, 0), (16, 2, 99)]


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hash_kat.txt")
    lines = ["# IBLT hash convention, written by make_hash_kat.py from the oracle.",
             "# table n r seed | seeds s_0..s_r | offsets off_0..off_r",
             "# key x | cells c_0..c_{r-1} | checksum"]
    for n, r, seed in CASES:
        seeds = oracle.hash_seeds(seed, r)
        offs = oracle.part_offsets(n, r)
        lines.append(f"table {n} {r} {seed} | " + " ".join(str(int(s)) for s in seeds)
                     + " | " + " ".join(str(int(o)) for o in offs))
        keys = list(ppgen.distinct_keys(6, seed + 1)) + [0, (1 << 64) - 1]
        import numpy as np
        cells = oracle.key_cells(n, r, seed, np.array(keys, dtype=np.uint64))
        for x, cs in zip(keys, cells):
            lines.append(f"key {int(x)} | " + " ".join(str(int(c)) for c in cs)
                         + f" | {oracle.checksum(seed, r, int(x))}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
