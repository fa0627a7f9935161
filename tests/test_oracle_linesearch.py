"""Pins for the oracle's globalization rules (no GPU): the filter acceptance test, the
barrier-parameter update and the inertia-correction schedule, against values worked out by
hand from Waechter & Biegler (2006), the line-search method cited in Sec. 2.2 of the paper.

Each case is chosen so that a wrong constant (gamma_theta, gamma_phi, s_theta, s_phi, delta,
eta_phi, kappa_mu, theta_mu, the delta_w factors) or a wrong branch flips the outcome.
"""
import types

import numpy as np
import pytest

from oracle import ipm
from oracle import kkt as K

TMIN, TMAX = 1e-4, 1e4


def acc(theta, phi, gphi, alpha, tht, pht, filt=(), tmin=TMIN, tmax=TMAX):
    return ipm.filter_accept(theta, phi, gphi, alpha, tht, pht, list(filt), tmin, tmax)


def test_sufficient_decrease_in_theta_pins_gamma_theta():
    # no switching (gphi >= 0): accept iff tht <= (1 - 1e-5) theta or pht <= phi - 1e-8 theta
    assert acc(1.0, 10.0, 0.0, 1.0, 1.0 - 2e-5, 10.5) == (True, False)
    assert acc(1.0, 10.0, 0.0, 1.0, 1.0 - 0.5e-5, 10.5)[0] is False


def test_sufficient_decrease_in_phi_pins_gamma_phi():
    assert acc(1.0, 10.0, 0.0, 1.0, 1.5, 10.0 - 2e-8) == (True, False)
    assert acc(1.0, 10.0, 0.0, 1.0, 1.5, 10.0 - 0.5e-8)[0] is False


def test_switching_condition_pins_s_theta():
    # gphi = -1: switching iff alpha > theta^1.1; theta = 0.5 -> 0.5^1.1 = 0.466516...
    # with theta_min = 10 the switching case takes the Armijo branch, whose decrease of
    # 1e-8 alpha is not met by pht = phi, so a switching trial is rejected
    kw = dict(tmin=10.0)
    assert acc(0.5, 10.0, -1.0, 0.48, 0.1, 10.0, **kw)[0] is False     # switching: Armijo fails
    assert acc(0.5, 10.0, -1.0, 0.45, 0.1, 10.0, **kw) == (True, False)  # no switching: theta drop


def test_switching_condition_pins_s_phi():
    # gphi = -2, theta = 1: switching iff alpha 2^2.3 > 1, i.e. alpha > 0.20306...
    kw = dict(tmin=10.0)
    assert acc(1.0, 10.0, -2.0, 0.21, 0.5, 10.0, **kw)[0] is False
    assert acc(1.0, 10.0, -2.0, 0.20, 0.5, 10.0, **kw) == (True, False)


def test_armijo_pins_eta_phi():
    # theta tiny (switching, theta <= theta_min): accept iff pht <= phi + 1e-8 alpha gphi
    assert acc(1e-6, 10.0, -1.0, 1.0, 1e-6, 10.0 - 2e-8) == (True, True)
    assert acc(1e-6, 10.0, -1.0, 1.0, 1e-6, 10.0 - 0.5e-8)[0] is False


def test_filter_entries_and_theta_max():
    # dominated by the entry (0.4, 10.5): rejected; passes (0.4, 12) through phi
    assert acc(1.0, 10.0, 0.0, 1.0, 0.5, 11.0, [(0.4, 10.5)])[0] is False
    assert acc(1.0, 10.0, 0.0, 1.0, 0.5, 11.0, [(0.4, 12.0)]) == (True, False)
    assert acc(1.0, 10.0, 0.0, 1.0, 0.3, 11.0, [(0.4, 10.5)]) == (True, False)
    assert acc(2e4, 10.0, 0.0, 1.0, 1.5e4, 5.0)[0] is False   # theta above theta_max
    assert acc(1.0, 10.0, 0.0, 1.0, 0.5, np.nan)[0] is False


def test_rounding_margin_of_phi_comparisons():
    # phi = 10: margin = 10 eps 10 = 2.2e-14.  A filter entry is passed by a trial whose phi
    # exceeds it by less than the margin, not by more.
    eps = np.finfo(np.float64).eps
    m = 10 * eps * 10.0
    assert acc(1.0, 10.0, 0.0, 1.0, 0.5, 11.0 + 0.4 * m, [(0.4, 11.0)]) == (True, False)
    assert acc(1.0, 10.0, 0.0, 1.0, 0.5, 11.0 + 3.0 * m, [(0.4, 11.0)])[0] is False
    # Armijo with a search direction whose phi change is below rounding: equal phi accepted
    assert acc(0.0, 10.0, -1e-20, 1.0, 0.0, 10.0 + 0.4 * m) == (True, True)
    assert acc(0.0, 10.0, -1e-20, 1.0, 0.0, 10.0 + 3.0 * m)[0] is False


def test_barrier_parameter_sequence():
    # mu0 = 0.1, tol = 1e-6: min(0.2 mu, mu^1.5) floored at tol / 10
    mu, seq = 0.1, []
    for _ in range(6):
        mu = ipm.barrier_update(mu, 1e-6)
        seq.append(mu)
    expect = [0.02, 0.0028284271247462, 1.5042412372345e-4, 1.84491446e-6, 1e-7, 1e-7]
    np.testing.assert_allclose(seq, expect, rtol=1e-7)


class _Scalar:
    """A 1x1 'matrix' a + delta, 'factored' iff positive."""

    def __init__(self):
        self.tried = []

    def factor(self, k):
        self.tried.append(k)
        return types.SimpleNamespace(ok=k > 0)


@pytest.mark.parametrize("a, last, expect, tries", [
    (-0.5, 0.0, 1.0, [0.0, 1e-4, 1e-2, 1.0]),            # first time: 1e-4, x100
    (-0.5, 1.0, 8.0 / 3.0, [0.0, 1.0 / 3.0, 8.0 / 3.0]),  # later: delta_last / 3, x8
    (-1e-3, 0.0, 1e-2, [0.0, 1e-4, 1e-2]),
    (2.0, 5.0, 0.0, [0.0]),                               # positive definite: no correction
])
def test_inertia_correction_schedule(a, last, expect, tries):
    s = _Scalar()
    dw, F, nf = K.inertia_schedule(lambda d: a + d, s, last)
    assert F.ok
    assert dw == pytest.approx(expect, rel=1e-12)
    np.testing.assert_allclose(np.array(s.tried) - a, tries, rtol=1e-12, atol=0)
    assert nf == len(tries)
