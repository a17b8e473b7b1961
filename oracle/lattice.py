"""Velocity sets and isotropy-derived weights (oracle, test infrastructure).

Paper: Sec. II.  The D3Q19 set with c_s^2 = 1/3 carries the populations; the
Shan-Chen force (Eq. (8)) sums over the 18 non-rest vectors with weights
W(1) = 1/6, W(2) = 1/12 "ensuring 4-th order lattice force isotropy".  The
flat runs (Sec. IV) use the 2-D projection W(1) = 1/3, W(2) = 1/12.

Nothing here is typed in from a table: the lattice weights are solved from
the moment conditions of the second-order Maxwellian and the forcing weights
from the isotropy conditions, in exact rational arithmetic.  The paper's
printed E4 and D2Q9 values pin the solver (tests/golden/paper_constants.json).

Population order (an interface convention shared with the C-ABI, each side
writing its own table):

    0: ( 0, 0, 0)
    1: (+1, 0, 0)   2: (-1, 0, 0)   3: ( 0,+1, 0)   4: ( 0,-1, 0)
    5: ( 0, 0,+1)   6: ( 0, 0,-1)
    7: (+1,+1, 0)   8: (-1,-1, 0)   9: (+1,-1, 0)  10: (-1,+1, 0)
   11: (+1, 0,+1)  12: (-1, 0,-1)  13: (+1, 0,-1)  14: (-1, 0,+1)
   15: ( 0,+1,+1)  16: ( 0,-1,-1)  17: ( 0,+1,-1)  18: ( 0,-1,+1)
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from math import prod

import numpy as np

CS2 = Fraction(1, 3)          # c_s^2 = 1/3 (Sec. II)

D3Q19 = np.array([
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
], dtype=np.int64)

D1Q3 = np.array([(0,), (1,), (-1,)], dtype=np.int64)

# forcing stencils: the shells |xi|^2 they use (Sec. II; E6/E8 are the wider
# isotropic stencils the paper cites for the force)
STENCIL_SHELLS = {"E4": (1, 2), "E6": (1, 2, 3, 4), "E8": (1, 2, 3, 4, 5, 6, 8)}
STENCIL_ORDER = {"E4": 4, "E6": 6, "E8": 8}


def integer_shell(dim: int, sq: int) -> list[tuple[int, ...]]:
    """All integer vectors of Z^dim with squared length ``sq``, sorted."""
    r = int(np.floor(np.sqrt(sq)))
    return sorted(v for v in itertools.product(range(-r, r + 1), repeat=dim)
                  if sum(c * c for c in v) == sq)


def _solve_exact(A: list[list[Fraction]], b: list[Fraction]) -> list[Fraction]:
    """Gauss-Jordan elimination over the rationals for a square system."""
    n = len(A)
    M = [list(map(Fraction, row)) + [Fraction(bi)] for row, bi in zip(A, b)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        p = M[col][col]
        M[col] = [v / p for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                fac = M[r][col]
                M[r] = [a - fac * c for a, c in zip(M[r], M[col])]
    return [M[r][n] for r in range(n)]


def _moment(vectors, powers) -> int:
    """sum over vectors of prod_alpha v_alpha^powers_alpha (brute force)."""
    return sum(prod(v[a] ** p for a, p in enumerate(powers)) for v in vectors)


def lattice_weights(vectors: np.ndarray, cs2: Fraction = CS2) -> list[Fraction]:
    """Per-vector weights w_i of a velocity set, one unknown per shell.

    Conditions (the moments that make the equilibrium of Eq. (6) reproduce
    the Maxwellian's): sum w = 1, sum w xi_x^2 = c_s^2 and, where the set has
    a second non-rest shell, sum w xi_x^2 xi_y^2 = c_s^4.
    """
    vecs = [tuple(int(c) for c in v) for v in vectors]
    dim = len(vecs[0])
    shells = sorted({sum(c * c for c in v) for v in vecs})
    members = {s: [v for v in vecs if sum(c * c for c in v) == s] for s in shells}
    rows, rhs = [], []
    rows.append([len(members[s]) for s in shells]); rhs.append(Fraction(1))
    p2 = (2,) + (0,) * (dim - 1)
    rows.append([_moment(members[s], p2) for s in shells]); rhs.append(cs2)
    if len(shells) > 2:
        p22 = (2, 2) + (0,) * (dim - 2)
        rows.append([_moment(members[s], p22) for s in shells]); rhs.append(cs2 * cs2)
    w_shell = _solve_exact(rows, rhs)
    ws = dict(zip(shells, w_shell))
    return [ws[sum(c * c for c in v)] for v in vecs]


def _double_factorial_odd(k: int) -> int:
    """(k-1)!! for even k >= 0 (the count of pairings of k indices)."""
    out = 1
    for j in range(k - 1, 0, -2):
        out *= j
    return out


def _monomial_classes(dim: int, order: int) -> list[tuple[int, ...]]:
    """Exponent tuples a_1 >= a_2 >= ... >= 0, all even, summing to ``order``."""
    out = []
    for t in itertools.product(range(0, order + 1, 2), repeat=dim):
        if sum(t) == order and list(t) == sorted(t, reverse=True):
            out.append(t)
    return out


def forcing_weights(shells, order: int, dim: int = 3) -> list[Fraction]:
    """Shell weights W(|xi|^2) of an isotropic forcing stencil.

    The stencil sum  sum_a W(|xi_a|^2) xi_a^{al_1} ... xi_a^{al_2k}  must be
    e_{2k} times the fully symmetric isotropic tensor for every even rank
    2k <= ``order`` (Sec. II, the isotropy requirement behind Eq. (8)), and
    e_2 = 1 (Sec. II, below Eq. (10)).  For a cubic stencil a component whose
    index multiplicities are (a, b, c, ...) of the isotropic tensor equals
    e_{2k} (a-1)!!(b-1)!!(c-1)!!; equating the ratio across all classes of one
    rank gives the linear conditions.
    """
    shells = list(shells)
    members = {s: integer_shell(dim, s) for s in shells}
    rows, rhs = [], []
    base = (2,) + (0,) * (dim - 1)
    rows.append([Fraction(_moment(members[s], base)) for s in shells]); rhs.append(Fraction(1))
    for rank in range(4, order + 1, 2):
        classes = _monomial_classes(dim, rank)
        ref = classes[0]
        ref_norm = prod(_double_factorial_odd(a) for a in ref)
        for cl in classes[1:]:
            norm = prod(_double_factorial_odd(a) for a in cl)
            rows.append([Fraction(_moment(members[s], cl), norm)
                         - Fraction(_moment(members[s], ref), ref_norm) for s in shells])
            rhs.append(Fraction(0))
    if len(rows) != len(shells):
        raise ValueError(f"{len(rows)} conditions for {len(shells)} shells")
    return _solve_exact(rows, rhs)


def stencil(name: str, dim: int = 3):
    """(vectors [m, dim] int64, weights [m] float64) of a forcing stencil.

    E4 are the 18 non-rest D3Q19 vectors in population order (Sec. II: the
    forcing vectors are the lattice velocities minus the rest one); wider
    stencils list their shells in increasing |xi|^2.
    """
    shells = STENCIL_SHELLS[name]
    W = forcing_weights(shells, STENCIL_ORDER[name], dim)
    wmap = dict(zip(shells, W))
    if name == "E4" and dim == 3:
        vecs = [tuple(v) for v in D3Q19[1:]]
    else:
        vecs = [v for s in shells for v in integer_shell(dim, s)]
    w = [float(wmap[sum(c * c for c in v)]) for v in vecs]
    return np.array(vecs, dtype=np.int64), np.array(w, dtype=np.float64)


def d3q19_weights() -> np.ndarray:
    """float64 w_i of D3Q19 in population order."""
    return np.array([float(w) for w in lattice_weights(D3Q19)], dtype=np.float64)


def d1q3_weights() -> np.ndarray:
    return np.array([float(w) for w in lattice_weights(D1Q3)], dtype=np.float64)
