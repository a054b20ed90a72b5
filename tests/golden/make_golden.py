"""Recompute the closed-form golden values in this folder and check the stored files.

The values come from the closed forms derived in README.md (no oracle or CUDA code is
involved). Run: python tests/golden/make_golden.py
"""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def square_rows():
    rows = []
    for alpha, beta in [(2.0, 4.5), (3.0, 6.0), (2.0, 4.0)]:
        E = 2.0 + 2.0 ** (1.0 - beta / 2.0)
        c = (2.0 + alpha - beta) * E / (4.0 * math.sqrt(2.0) / 2.0)
        rows.append((alpha, beta, E, c))
    return rows


def check():
    stored = []
    with open(os.path.join(HERE, "square_energy.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                stored.append(tuple(float(x) for x in line.split()))
    for a, b in zip(stored, square_rows()):
        for x, y in zip(a, b):
            assert abs(x - y) <= 1e-15 * max(1.0, abs(y)), (a, b)
    return True


if __name__ == "__main__":
    print("square_energy.txt consistent:", check())
