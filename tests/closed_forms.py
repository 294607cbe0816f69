"""Closed forms used to pin the oracle and the class table (exact integers).

* Unlabelled digraphs on n vertices (no loops): Burnside's lemma over S_n.  A
  permutation with cycle type lambda acts on the n(n-1) ordered pairs with
  sum_i (l_i - 1) + 2 * sum_{i<j} gcd(l_i, l_j) cycles, so the number of
  classes is sum over lambda of 2^cycles(lambda) / z_lambda.
* Weakly connected ones: inverse Euler transform of that sequence.
* Labelled weakly connected digraphs:
  c(n) = 2^{n(n-1)} - sum_{j=1}^{n-1} C(n-1, j-1) c(j) 2^{(n-j)(n-j-1)}.
"""
from fractions import Fraction
from math import comb, factorial, gcd


def _partitions(n, maxpart=None):
    if maxpart is None:
        maxpart = n
    if n == 0:
        yield []
        return
    for p in range(min(n, maxpart), 0, -1):
        for rest in _partitions(n - p, p):
            yield [p] + rest


def _z(lam):
    out = 1
    for p in set(lam):
        c = lam.count(p)
        out *= p ** c * factorial(c)
    return out


def digraph_classes(n):
    """Number of isomorphism classes of loopless digraphs on n vertices."""
    total = Fraction(0)
    for lam in _partitions(n):
        cyc = sum(l - 1 for l in lam)
        for i in range(len(lam)):
            for j in range(i + 1, len(lam)):
                cyc += 2 * gcd(lam[i], lam[j])
        total += Fraction(2 ** cyc, _z(lam))
    assert total.denominator == 1
    return int(total)


def _mobius(n):
    res, p, m = 1, 2, n
    while p * p <= m:
        if m % p == 0:
            m //= p
            if m % p == 0:
                return 0
            res = -res
        p += 1
    if m > 1:
        res = -res
    return res


def connected_classes(nmax):
    """Inverse Euler transform: weakly connected classes for n = 1..nmax."""
    a = [digraph_classes(n) for n in range(nmax + 1)]  # a[0] = 1
    c = [0] * (nmax + 1)
    for n in range(1, nmax + 1):
        c[n] = n * a[n] - sum(c[k] * a[n - k] for k in range(1, n))
    b = [0] * (nmax + 1)
    for n in range(1, nmax + 1):
        s = sum(_mobius(n // d) * c[d] for d in range(1, n + 1) if n % d == 0)
        assert s % n == 0
        b[n] = s // n
    return b


def labelled_connected(nmax):
    c = [0] * (nmax + 1)
    for n in range(1, nmax + 1):
        c[n] = 2 ** (n * (n - 1)) - sum(
            comb(n - 1, j - 1) * c[j] * 2 ** ((n - j) * (n - j - 1)) for j in range(1, n))
    return c
