"""The FP64 quotient the kernels use on the hot path (div_nr: a float-seeded
reciprocal, one Newton step and a final residual correction, Markstein's
scheme) against CUDA's IEEE division a / b, on 2^20 random operand pairs over
the working range and on operands across the whole double range, including
divisors outside the float exponent range (where div_nr falls back to the
IEEE quotient), zeros, infinities and NaNs.

Bound: where the IEEE quotient is finite, div_nr is finite and within 2 ulp
of it, counted in the spacing of the doubles around it (subnormal spacing
included), for numerators of magnitude at least 2^-920; below that the
residual a - b q (about 2^-46 |a| before the correction) leaves the normal
range, the correction loses bits and the quotient keeps the error of the
refined reciprocal, within 2^8 ulp (the hot path's numerators -- WENO-5
weight sums, moment sums, transport terms -- are far above 2^-920).  Where
the IEEE quotient is NaN, so is div_nr's; where it is infinite (an
overflowing quotient, an infinite numerator), div_nr's is not finite either
-- the residual correction turns it into NaN -- which the kernels'
non-finite check flags in the same way; bit-identical where the divisor lies
outside the float exponent range."""
import numpy as np
import pytest

import paper_2503_15187_gb300 as ev

pytestmark = pytest.mark.gpu


def ordered(x):
    """Doubles mapped to integers in the order of their values (adjacent
    doubles differ by one), so that a difference counts ulps."""
    b = x.view(np.int64)
    return np.where(b >= 0, b, np.int64(-0x8000000000000000) - b)


def quotients(a, b):
    import torch
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    q, qi = ev.divide_fp64(ta, tb)
    return q.cpu().numpy(), qi.cpu().numpy()


def test_div_nr_within_two_ulp_on_the_working_range():
    rng = np.random.default_rng(20250315)
    n = 1 << 20
    a = rng.uniform(1, 2, n) * np.exp2(rng.integers(-60, 61, n)) * rng.choice([-1.0, 1.0], n)
    b = rng.uniform(1, 2, n) * np.exp2(rng.integers(-60, 61, n)) * rng.choice([-1.0, 1.0], n)
    q, qi = quotients(a, b)
    d = np.abs(ordered(q) - ordered(qi))
    print(f"div_nr, 2^20 pairs: max {d.max()} ulp, {np.mean(d > 0):.2%} differ from IEEE")
    assert d.max() <= 2


def test_div_nr_extremes_and_fallback():
    rng = np.random.default_rng(7)
    n = 1 << 18
    a = rng.uniform(1, 2, n) * np.exp2(rng.integers(-1070, 1023, n).astype(float)) * rng.choice([-1.0, 1.0], n)
    b = rng.uniform(1, 2, n) * np.exp2(rng.integers(-1070, 1023, n).astype(float)) * rng.choice([-1.0, 1.0], n)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 1.0, 3.0, 2.0 ** 120, 2.0 ** -120,
                        2.0 ** 121, 2.0 ** -121, 1.7976931348623157e308])
    sa, sb = np.meshgrid(special, special)
    a = np.concatenate([a, sa.ravel()])
    b = np.concatenate([b, sb.ravel()])
    with np.errstate(all="ignore"):
        q, qi = quotients(a, b)
    fin = np.isfinite(qi)
    assert np.all(np.isfinite(q[fin]))
    assert np.all(np.isnan(q[np.isnan(qi)]))
    assert np.all(~np.isfinite(q[np.isinf(qi)]))
    assert np.isinf(qi).sum() > 100                         # overflowing quotients were met
    d = np.abs(ordered(q[fin]) - ordered(qi[fin]))
    tiny = np.abs(a[fin]) < 2.0 ** -920
    print(f"div_nr, extremes: max {d[~tiny].max()} ulp over {(~tiny).sum()} finite quotients of numerators "
          f">= 2^-920, max {d[tiny].max() if tiny.any() else 0} ulp over {tiny.sum()} below")
    worst = np.argsort(d)[-5:]
    for j in worst:
        print(f"  a={a[fin][j]:.6e} b={b[fin][j]:.6e} ulp={d[j]}")
    assert d[~tiny].max() <= 2
    assert d.max() <= 256
    ex = (b.view(np.int64) >> 52) & 0x7FF
    out = (ex < 1023 - 120) | (ex > 1023 + 120)          # the IEEE fallback
    assert out.sum() > 1000
    both = out & ~np.isnan(qi)
    assert np.array_equal(q[both].view(np.int64), qi[both].view(np.int64))
