"""lr_choose_order (host arithmetic, no GPU): the chosen Lagrange order reads a sinusoid of the
band edge within the tolerance and the next lower compiled order does not, with the read error
measured through the oracle's centered Lagrange read (Sec. "Implementation") on the same
fractional offsets."""
import numpy as np
import pytest

import __graft_entry__  # noqa: F401
import oracle
import paper_2204_06633_gb300 as lr
from paper_2204_06633_gb300 import _build


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def read_error(p, f_dt):
    """max over eps of |exp(i w eps) - Lagrange read of exp(i w j)| through the oracle."""
    w = 2 * np.pi * f_dt
    j = np.arange(-200, 201)
    c, s = np.cos(w * j), np.sin(w * j)
    worst = 0.0
    for k in range(129):
        eps = k / 128.0
        re = oracle.lagrange_read(c, 200, eps, p)
        im = oracle.lagrange_read(s, 200, eps, p)
        worst = max(worst, abs(complex(np.cos(w * eps) - re, np.sin(w * eps) - im)))
    return worst


@pytest.mark.parametrize("f_dt,tol", [(0.1, 1e-6), (0.03, 1e-10), (0.01, 1e-12), (0.1, 1e-3), (1e-3, 1e-8)])
def test_chosen_order_is_the_smallest_that_meets_the_tolerance(f_dt, tol):
    p = lr.choose_order(f_dt, tol)
    assert lr.order_supported(p)
    assert read_error(p, f_dt) <= tol * (1 + 1e-6)
    lower = [q for q in range(1, p, 2) if lr.order_supported(q)]
    if lower:
        assert read_error(lower[-1], f_dt) > tol


def test_choose_order_rejects_bad_requests():
    for args in ((0.6, 1e-6), (-0.1, 1e-6), (0.1, 0.0)):
        with pytest.raises(lr.LRError):
            lr.choose_order(*args)
    with pytest.raises(lr.LRError) as e:
        lr.choose_order(0.45, 1e-15)   # no compiled order reaches it
    assert e.value.status == 2
