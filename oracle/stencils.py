"""Finite-difference stencils of the spatial operator A (oracle; test
infrastructure only).

The paper does not print its stencils.  Sec. 5 states that the heat equation
is discretised with centred differences and the advection equation with an
upwind scheme, both periodic, and Tables 1-2 give the order kappa: 2, 4, 6
centred, 1 to 5 upwind.  The weights here follow from the definition of a
finite-difference formula: on the integer offsets o_0 < ... < o_p, the
weights w of the d-th derivative are the unique ones that are exact on the
monomials x^0 .. x^p,

    sum_j w_j o_j^k = d!  if k = d,  else 0,     k = 0 .. p,

solved here in exact rational arithmetic.  The derivative is then
h^-d sum_j w_j u_{i + o_j}.

Offsets (readings of "centred" and "upwind" of a given order):
  centred, order p (even):      -p/2 .. p/2;
  upwind,  order p, for c > 0:  lo .. lo + p with lo = -(floor(p/2) + 1),
      i.e. one more point on the upwind (left) side than on the other for
      odd p, two more for even p (the usual upwind-biased formulas);
      for c < 0 the stencil is mirrored: w'(o) = -w(-o).
The Laplacian of a problem with an upwind first derivative of order p uses
the centred second derivative of order p rounded up to even.
"""
import math
from fractions import Fraction

CENTRAL_ORDERS = (2, 4, 6)
UPWIND_ORDERS = (1, 2, 3, 4, 5)


def fd_weights(offsets, deriv):
    """Exact weights {offset: Fraction} of the `deriv`-th derivative on the
    given distinct integer offsets (moment conditions above)."""
    offsets = list(offsets)
    n = len(offsets)
    if len(set(offsets)) != n or not 0 <= deriv < n:
        raise ValueError("need distinct offsets and deriv < number of offsets")
    # augmented Vandermonde system, row k: o_j^k | d! [k == d]
    a = [[Fraction(o) ** k for o in offsets] + [Fraction(math.factorial(deriv) if k == deriv else 0)]
         for k in range(n)]
    for c in range(n):                       # Gauss-Jordan elimination, exact
        piv = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[piv] = a[piv], a[c]
        inv = 1 / a[c][c]
        a[c] = [x * inv for x in a[c]]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return {o: a[j][n] for j, o in enumerate(offsets)}


def central_offsets(order):
    if order not in CENTRAL_ORDERS:
        raise ValueError("centred order must be 2, 4 or 6")
    r = order // 2
    return list(range(-r, r + 1))


def upwind_offsets(order):
    if order not in UPWIND_ORDERS:
        raise ValueError("upwind order must be 1..5")
    lo = -(order // 2 + 1)
    return list(range(lo, lo + order + 1))


def d1_weights(order, upwind=False, c=1.0):
    """First-derivative weights {offset: Fraction} (nonzero only)."""
    if not upwind:
        w = fd_weights(central_offsets(order), 1)
    else:
        w = fd_weights(upwind_offsets(order), 1)
        if c < 0:
            w = {-o: -v for o, v in w.items()}
    return {o: v for o, v in w.items() if v != 0}


def laplacian_order(order, upwind=False):
    return order + (order % 2) if upwind else order


def d2_weights(order, upwind=False):
    """Second-derivative weights (centred, see the module note)."""
    w = fd_weights(central_offsets(laplacian_order(order, upwind)), 2)
    return {o: v for o, v in w.items() if v != 0}


def check_scheme(order, upwind):
    if upwind and order not in UPWIND_ORDERS:
        raise ValueError("upwind order must be 1..5")
    if not upwind and order not in CENTRAL_ORDERS:
        raise ValueError("centred order must be 2, 4 or 6")
