"""Writes the closed-form fixtures in this folder (stdlib math only; no GPU
code, no oracle arithmetic is needed for a closed form).

    python tests/golden/make_golden.py

toeplitz_sigma_n64.txt
    Singular values of the tridiagonal Toeplitz matrix with diagonal a = 2 and
    off-diagonals c = -1 (also those of R from its QR factorisation):
    sigma_k = |a + 2 c cos(k pi / (n + 1))|, k = 1..n, n = 64 (eigenvalues of a
    symmetric tridiagonal Toeplitz matrix, a textbook closed form).
bidiag_ones_sigma_n10.txt
    Singular values of the n x n upper bidiagonal matrix with every d_i = e_i = 1:
    sigma_k = 2 cos(k pi / (2 n + 1)), k = 1..n, n = 10 (B^T B is tridiagonal
    Toeplitz with a perturbed corner; closed form from its characteristic
    polynomial recursion).
"""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, header, values):
    with open(os.path.join(HERE, name), "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line.strip() + "\n")
        for v in sorted(values, reverse=True):
            f.write(repr(float(v)) + "\n")


def main():
    n = 64
    write("toeplitz_sigma_n64.txt",
          "sigma_k = |2 - 2 cos(k pi / 65)|, k = 1..64: tridiagonal Toeplitz (a=2, c=-1)\n"
          "written by tests/golden/make_golden.py",
          [abs(2.0 - 2.0 * math.cos(k * math.pi / (n + 1))) for k in range(1, n + 1)])
    n = 10
    write("bidiag_ones_sigma_n10.txt",
          "sigma_k = 2 cos(k pi / 21), k = 1..10: upper bidiagonal, all entries 1\n"
          "written by tests/golden/make_golden.py",
          [2.0 * math.cos(k * math.pi / (2 * n + 1)) for k in range(1, n + 1)])


if __name__ == "__main__":
    main()
