"""Central second-derivative weights of any even accuracy order, from the
polynomial-interpolation linear system (the paper's stencil generation, Sec.
"Compile-Time Stencil Generation": a polynomial of order q = p + n - 1 for a
derivative of order p = 2 and accuracy n, the unknowns reduced by symmetry).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: exact rational
arithmetic (``fractions.Fraction``), no code shared with the GPU library.

On the points -r..r (r = n/2) the symmetric weights w_0, w_1..w_r (w_-j = w_j)
make the stencil exact on every polynomial of degree <= 2r + 1:
    sum_j w_j j^k = 2 if k == 2 else 0     for k = 0..2r
(odd k vanish by symmetry), i.e.  w_0 + 2 sum_{j>=1} w_j = 0  and
sum_{j>=1} w_j j^(2m) = [m == 1]  for m = 1..r.  The cross Laplacian in d
dimensions applies the same weights along every axis:
    L_h f = (1/h^2) [ d w_0 f_0 + sum_{j=1..r} w_j P_j ],
    P_j = sum over axes of (f(+j e_a) + f(-j e_a)).
"""
from fractions import Fraction


def second_derivative_weights(order: int):
    """Exact (w_0, w_1, ..., w_r) for accuracy ``order`` (even, >= 2)."""
    if order < 2 or order % 2:
        raise ValueError("accuracy order must be even and >= 2")
    r = order // 2
    # rows m = 1..r: sum_j w_j j^(2m) = [m == 1]
    A = [[Fraction(j ** (2 * m)) for j in range(1, r + 1)] + [Fraction(1 if m == 1 else 0)]
         for m in range(1, r + 1)]
    for col in range(r):  # Gauss-Jordan elimination, exact
        piv = next(i for i in range(col, r) if A[i][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for i in range(r):
            if i != col and A[i][col] != 0:
                f = A[i][col]
                A[i] = [a - f * b for a, b in zip(A[i], A[col])]
    w = [A[i][r] for i in range(r)]
    return [-2 * sum(w)] + w


def kernel_weights(order: int, dims: int):
    """The doubles a kernel uses: (d w_0, w_1, ..., w_r), each the exact rational
    rounded once to FP64."""
    w = second_derivative_weights(order)
    return [float(dims * w[0])] + [float(x) for x in w[1:]]


def lambda_max(order: int, dims: int) -> float:
    """Largest eigenvalue of -h^2 L_h (at theta = pi on every axis)."""
    w = second_derivative_weights(order)
    one = -(w[0] + 2 * sum(wj * (-1) ** j for j, wj in enumerate(w[1:], start=1)))
    return float(dims * one)
