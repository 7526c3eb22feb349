"""The row-recurrence algebra of the mixed path's multi-row kernels, checked in float64 on
random complex quadratic exponents (no GPU).

A beamlet's field on the detector is exp(Q(tu, tv)) with the quadratic form (the
propagated beamlet of Eq. gauss_prop projected to pixel coordinates about its centre)
    Q = c0 + cu tu + cv tv + cuu tu^2 + cuv tu tv + cvv tv^2.
The row triples and quadruples evaluate the first row of a thread directly and the rows
8 r below as that value times P_r(tu) = S_r W(tu)^r, where
    R = exp(8 (cv + cvv (2 tv + 8))),  K = exp(128 cvv),  S_r = prod_{j<r} R K^j,
    W(tu) = exp(8 cuv tu),
and step P_r along a thread's columns (32 apart) by T^r with T = exp(256 cuv).  Without a
uv term W = T = 1 and P_r = S_r.  These are identities of the exponential of a quadratic;
the tests check them to float64 rounding, including the uv term's contribution, so that a
wrong power of K or of W (a plausible slip in the kernels' row terms) shows here.
"""
import numpy as np
import pytest

RNG = np.random.default_rng(240412457)


def rand_form(uv: bool):
    c = RNG.normal(scale=0.02, size=6) + 1j * RNG.normal(scale=0.05, size=6)
    c[0] = RNG.normal() + 1j * RNG.normal()
    if not uv:
        c[4] = 0.0
    return c


def Q(c, tu, tv):
    c0, cu, cv, cuu, cuv, cvv = c
    return c0 + cu * tu + cv * tv + cuu * tu * tu + cuv * tu * tv + cvv * tv * tv


def row_factor(c, tu, tv, r):
    """P_r(tu) as the kernels form it: S_r from R and K, times W(tu)^r."""
    cv, cuv, cvv = c[2], c[4], c[5]
    R = np.exp(8.0 * (cv + cvv * (2.0 * tv + 8.0)))
    K = np.exp(128.0 * cvv)
    S = np.prod([R * K ** j for j in range(r)]) if r else 1.0
    W = np.exp(8.0 * cuv * tu)
    return S * W ** r


@pytest.mark.parametrize("uv", [False, True])
def test_rows_below_are_the_first_row_times_the_row_factors(uv):
    for _ in range(20):
        c = rand_form(uv)
        tu, tv = RNG.uniform(-40, 40), RNG.uniform(-40, 40)
        E0 = np.exp(Q(c, tu, tv))
        for r in range(1, 4):
            want = np.exp(Q(c, tu, tv + 8.0 * r))
            got = E0 * row_factor(c, tu, tv, r)
            assert abs(got - want) <= 1e-12 * abs(want), (r, got, want)


@pytest.mark.parametrize("uv", [False, True])
def test_row_factors_step_along_the_row_by_powers_of_t(uv):
    for _ in range(20):
        c = rand_form(uv)
        tu0, tv = RNG.uniform(-40, 40), RNG.uniform(-40, 40)
        T = np.exp(256.0 * c[4])
        for r in range(1, 4):
            P = row_factor(c, tu0, tv, r)
            for col in range(1, 8):  # the thread's columns, 32 pixels apart
                P = P * T ** r
                want = row_factor(c, tu0 + 32.0 * col, tv, r)
                assert abs(P - want) <= 1e-12 * abs(want), (r, col)
        if not uv:
            assert T == 1.0


def test_the_uv_term_matters_to_the_row_factor():
    """With a uv term, dropping W (the no-uv kernels' row factor) is wrong by far more than
    rounding: the reason fields with a uv term need the per-column factors."""
    c = rand_form(True)
    tu, tv = 30.0, 5.0
    E0 = np.exp(Q(c, tu, tv))
    want = np.exp(Q(c, tu, tv + 16.0))
    cv, cvv = c[2], c[5]
    R = np.exp(8.0 * (cv + cvv * (2.0 * tv + 8.0)))
    K = np.exp(128.0 * cvv)
    no_w = E0 * R * R * K
    assert abs(no_w - want) > 1e-3 * abs(want)
