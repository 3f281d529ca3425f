"""Coefficients of the start-distortion polynomial used by the mixed-form entropy.

The expansion starts from p(u) = u - u^3/3 + 2u^5/15 instead of tanh(u), so
the chain's argument is 2^n artanh(p(u)) rather than 2^n u.  The entropy term
Tr(Y T) therefore takes 2^n <delta(U), T> with

    delta(u) = artanh(p(u)) - u = u^7 g(u^2),

and g is fitted here on |u| <= 1: least squares for the absolute error of
u^7 g(u^2) at Chebyshev nodes of [0, 1], in 50-digit arithmetic (delta(u)
cancels badly in double precision for small u).  Prints the coefficients
c_0..c_d of g(s) = sum c_j s^j and the maximum absolute error on [0, 1].

    python paper_2303_03529_gb300/csrc/fit_start_distortion.py [degree]
"""
import sys

import mpmath as mp


def delta(u):
    return mp.atanh(u - u ** 3 / 3 + 2 * u ** 5 / 15) - u


def fit(degree: int, nodes: int = 400):
    mp.mp.dps = 50
    us = [mp.cos(mp.pi * (2 * i + 1) / (4 * nodes)) for i in range(nodes)]  # in (0, 1]
    A = mp.matrix(nodes, degree + 1)
    b = mp.matrix(nodes, 1)
    for i, u in enumerate(us):
        for j in range(degree + 1):
            A[i, j] = u ** 7 * u ** (2 * j)
        b[i] = delta(u)
    c = mp.lu_solve(A.T * A, A.T * b)
    err = mp.mpf(0)
    for k in range(1, 4001):
        u = mp.mpf(k) / 4000
        g = sum(c[j] * u ** (2 * j) for j in range(degree + 1))
        err = max(err, abs(u ** 7 * g - delta(u)))
    return [c[j] for j in range(degree + 1)], err


if __name__ == "__main__":
    d = int(sys.argv[1]) if len(sys.argv) > 1 else 6
    c, err = fit(d)
    print("max |error| on [0, 1]:", mp.nstr(err, 3))
    for j, x in enumerate(c):
        print(f"c{j} = {mp.nstr(x, 17)}")
