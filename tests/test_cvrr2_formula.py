"""The closed n-quantum CVRR2 form against repeated application of the 1-q step (no GPU).

Sec. 2.5.4: the contracted CVRR2 step
    (a c+1_i)_{k,n} = (a c)_{k,n+1_i} + a_i (a-1_i c)_{k+1,n}
applied lc times turns (a 0|c) = (a c)_{0,0} into prerequisites (e 0)_{k,n}.
The closed form printed in the paper is garbled; the reading used by the GPU
path (and derived by unrolling the step per axis) is
    (a 0|c) = sum_{u <= min(a,c)} prod_i C(a_i,u_i) C(c_i,u_i) u_i!  (a-u 0)_{|u|, c-u}.
This test expands the 1-q step symbolically, compares it with that closed
form for every a, c up to 6 quanta, and checks the paper's worked examples
(tests/golden/cvrr2_worked_examples.txt).
"""
import os
from functools import lru_cache
from math import comb, factorial

import pytest

from oracle.solid import cart_list

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cvrr2_worked_examples.txt")


@lru_cache(maxsize=None)
def expand_1q(a, c, k=0, n=(0, 0, 0)):
    """Symbolic expansion of (a c)_{k,n} into {(e, k', n'): coef} with c = 0 terms."""
    if sum(c) == 0:
        return {(a, k, n): 1}
    i = next(ax for ax in range(3) if c[ax] > 0)           # lower the first nonzero ket axis
    cm = tuple(c[j] - (j == i) for j in range(3))
    out = {}
    n1 = tuple(n[j] + (j == i) for j in range(3))
    for key, v in expand_1q(a, cm, k, n1).items():
        out[key] = out.get(key, 0) + v
    if a[i] > 0:
        am = tuple(a[j] - (j == i) for j in range(3))
        for key, v in expand_1q(am, cm, k + 1, n).items():
            out[key] = out.get(key, 0) + a[i] * v
    return {k_: v for k_, v in out.items() if v != 0}


def closed_form(a, c):
    out = {}
    for ux in range(min(a[0], c[0]) + 1):
        for uy in range(min(a[1], c[1]) + 1):
            for uz in range(min(a[2], c[2]) + 1):
                u = (ux, uy, uz)
                coef = 1
                for i in range(3):
                    coef *= comb(a[i], u[i]) * comb(c[i], u[i]) * factorial(u[i])
                key = (tuple(a[i] - u[i] for i in range(3)), sum(u), tuple(c[i] - u[i] for i in range(3)))
                out[key] = out.get(key, 0) + coef
    return out


@pytest.mark.parametrize("la", range(0, 7))
@pytest.mark.parametrize("lc", range(0, 7))
def test_closed_form_equals_repeated_step(la, lc):
    for a in cart_list(la):
        for c in cart_list(lc):
            assert expand_1q(a, c) == closed_form(a, c)


def _vec(s):
    return tuple(int(x) for x in s.split(","))


def test_worked_examples():
    lines = [l for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(lines) == 3
    for line in lines:
        a, c, terms = (p.strip() for p in line.split("|"))
        ref = {}
        for t in terms.split():
            coef, e, k, n = t.split(":")
            ref[(_vec(e), int(k), _vec(n))] = int(coef)
        assert closed_form(_vec(a), _vec(c)) == ref
        assert expand_1q(_vec(a), _vec(c)) == ref
