"""Write golden_products.txt: small seeded products computed by the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py
Each line: na nb a_hex b_hex c_hex (little-endian words joined, most significant first).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth                      # noqa: E402
from oracle import clmul as O     # noqa: E402

PAIRS = [(1, 1), (2, 2), (7, 5), (63, 64), (64, 64), (65, 63), (100, 200), (128, 1),
         (257, 255), (1000, 24), (1024, 1024), (2047, 2049), (4096, 4096)]


def main():
    lines = ["# Seeded products from the CPU oracle (oracle/clmul.py), written by make_golden.py.",
             "# na nb a b c  (hex of the polynomial as an integer, bit t = coefficient of x^t)"]
    for idx, (na, nb) in enumerate(PAIRS):
        a = synth.mask_tail(synth.operand(synth.config_seed(9, 2 * idx), na), na)
        b = synth.mask_tail(synth.operand(synth.config_seed(9, 2 * idx + 1), nb), nb)
        c = O.mul(a, na, b, nb)
        lines.append(f"{na} {nb} {O.words_to_int(a):x} {O.words_to_int(b):x} {O.words_to_int(c):x}")
    with open(os.path.join(HERE, "golden_products.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
