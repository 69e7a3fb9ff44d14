"""Writes the stored expected values under tests/golden/ that are not printed
in the paper.  Uses only numpy (GF(2) matrix powers), never the CUDA path."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def gf2_pow(M, n):
    R = np.eye(M.shape[0], dtype=np.int64)
    B = M.copy()
    while n:
        if n & 1:
            R = (R @ B) % 2
        B = (B @ B) % 2
        n >>= 1
    return R


def lfsr_matrix(taps=0xB400, w=16):
    # column j = image of basis vector e_j under one step
    M = np.zeros((w, w), np.int64)
    for j in range(w):
        img = (taps if j == 0 else 0) ^ ((1 << j) >> 1)
        for i in range(w):
            M[i, j] = (img >> i) & 1
    return M


def vec_to_int(v):
    return int(sum(int(b) << i for i, b in enumerate(v)))


def main():
    M = lfsr_matrix()
    e0 = np.zeros(16, np.int64)
    e0[0] = 1
    lines = open(os.path.join(HERE, "lfsr_b400.txt")).read().splitlines()
    lines = [l for l in lines if l.startswith("#")]
    for n in [1, 2, 3, 16, 100, 1000, 10000, 65534, 65535]:
        lines.append("%d 0x%04x" % (n, vec_to_int(gf2_pow(M, n) @ e0 % 2)))
    open(os.path.join(HERE, "lfsr_b400.txt"), "w").write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
