"""Exact colour algebra for one quark line plus k gluons -- TEST INFRASTRUCTURE ONLY.

The matrix element is decomposed as M = sum_sigma (T^{a_sigma1} ... T^{a_sigmak})_{i j} A(sigma)
(Mangano-Parke, Phys. Rep. 200 (1991) 301, colour decomposition with one quark line), so

    sum_colours |M|^2 = sum_{sigma,tau} A(sigma) C(sigma,tau) A(tau)^*,
    C(sigma,tau)      = sum_{a, i, j} (T^sigma)_{ij} ((T^tau)_{ij})^*
                      = Tr(T^{sigma1} ... T^{sigmak} T^{tauk} ... T^{tau1}).

This module evaluates those traces exactly with Fractions, by the SU(N) Fierz identity
sum_a (T^a)_{ij} (T^a)_{kl} = 1/2 (delta_il delta_kj - 1/N delta_ij delta_kl), applied one
summed label at a time:

    Tr(A T^a B T^a)   = 1/2 (Tr A Tr B - 1/N Tr(A B))
    Tr(A T^a) Tr(B T^a) = 1/2 (Tr(A B) - 1/N Tr A Tr B)
    Tr(1) = N,  Tr(T^a) = 0.

Only tests/, __graft_entry__.smoke() and bench.py may import this module.  Nothing here is
shared with the CUDA path.  Jamp index convention: the lexicographic rank of sigma among
the permutations of (0..k-1).
"""
from fractions import Fraction
from functools import lru_cache
from itertools import permutations

NC = 3


def _canon(traces):
    """Canonical, hashable form of a product of traces (each a tuple of labels)."""
    out = []
    for t in traces:
        if len(t) == 0:
            out.append(())
            continue
        # rotate to the lexicographically smallest rotation (cyclicity of the trace)
        rots = [t[i:] + t[:i] for i in range(len(t))]
        out.append(min(rots))
    return tuple(sorted(out))


@lru_cache(maxsize=None)
def _eval(traces):
    """Value of prod_t Tr(prod T^{labels of t}), summed over every label (each appears twice)."""
    value = Fraction(1)
    rest = []
    for t in traces:
        if len(t) == 0:
            value *= NC
        elif len(t) == 1:
            return Fraction(0)
        else:
            rest.append(t)
    if not rest:
        return value
    # pick the first label of the first trace and find its partner
    t0 = rest[0]
    a = t0[0]
    # same trace?
    j = None
    for pos in range(1, len(t0)):
        if t0[pos] == a:
            j = pos
            break
    others = rest[1:]
    if j is not None:
        # Tr(T^a B T^a A) with B = t0[1:j], A = t0[j+1:]
        B = t0[1:j]
        A = t0[j + 1:]
        term1 = _eval(_canon(others + [A, B]))
        term2 = _eval(_canon(others + [A + B]))
        return value * Fraction(1, 2) * (term1 - Fraction(1, NC) * term2)
    # partner in another trace
    for ti, t1 in enumerate(others):
        if a in t1:
            pos = t1.index(a)
            # Tr(A T^a) with A = t0[1:] (rotated: Tr(T^a A) = Tr(A T^a))
            A = t0[1:]
            # Tr(B T^a) with B = t1[pos+1:] + t1[:pos]
            B = t1[pos + 1:] + t1[:pos]
            rem = others[:ti] + others[ti + 1:]
            term1 = _eval(_canon(rem + [A + B]))
            term2 = _eval(_canon(rem + [A, B]))
            return value * Fraction(1, 2) * (term1 - Fraction(1, NC) * term2)
    raise ValueError("unpaired colour label")


def orderings(k):
    """All orderings of the k gluon labels, lexicographic (the jamp index convention)."""
    return list(permutations(range(k)))


def colour_entry(sigma, tau):
    """C(sigma,tau) = Tr(T^sigma (T^tau)^dagger), exact."""
    word = tuple(sigma) + tuple(reversed(tau))
    return _eval(_canon([word]))


@lru_cache(maxsize=None)
def colour_matrix_exact(k):
    """Exact ncol x ncol colour matrix (tuple of tuples of Fractions), ncol = k!."""
    perms = orderings(k)
    return tuple(tuple(colour_entry(s, t) for t in perms) for s in perms)


def colour_matrix(k):
    """Colour matrix as a float64 numpy array."""
    import numpy as np
    ex = colour_matrix_exact(k)
    return np.array([[float(x) for x in row] for row in ex], dtype=np.float64)
