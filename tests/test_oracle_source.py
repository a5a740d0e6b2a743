"""Pins of the oracle's source time function (Section III's Gaussian pulse).

Reading (the printed G(t) lacks its minus sign): the dipole moment is
amplitude * G(t) with G(t) = exp(-(t - t0)^2 / (4 tau^2)), and the current it
drives is J(t) = amplitude * G'(t).  ``oracle.solver.dipole_current`` is
checked here against quantities fixed by that reading alone, none of which
retypes its formula:

* a central difference of the moment (a wrong factor in the exponent's
  derivative, such as 1/tau^2 for 1/(2 tau^2), or a flipped sign fails it);
* the integral of J from far before the pulse up to t, which must give back
  the moment amplitude * G(t) (adaptive quadrature, no derivative taken);
* the charge balance: J integrates to zero over the whole pulse, so no static
  charge is left behind;
* the extremes of G' in closed form: |J| peaks at t0 -+ sqrt(2) tau with the
  value amplitude * exp(-1/2) / (sqrt(2) tau), positive before t0.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.solver import dipole_current
from synthetic import Dipole


def moment(src, t):
    return src.amplitude * math.exp(-(t - src.t0) ** 2 / (4.0 * src.width ** 2))


@pytest.mark.parametrize("t0,width,amp", [(1.0, 0.25, 1.0), (0.6, 0.15, -2.5),
                                          (1.6, 0.4, 0.3)])
def test_current_is_central_difference_of_moment(t0, width, amp):
    src = Dipole(t0=t0, width=width, amplitude=amp)
    h = 1e-5 * width
    for t in np.linspace(t0 - 4 * width, t0 + 4 * width, 17):
        fd = (moment(src, t + h) - moment(src, t - h)) / (2 * h)
        j = dipole_current(src, t)
        scale = abs(amp) / width
        assert abs(j - fd) <= 1e-9 * scale, (t, j, fd)


@pytest.mark.parametrize("t0,width,amp", [(1.0, 0.25, 1.0), (0.6, 0.15, 2.0)])
def test_current_integrates_to_moment_and_to_zero(t0, width, amp):
    src = Dipole(t0=t0, width=width, amplitude=amp)
    t_start = t0 - 12 * width
    for t in (t0 - width, t0, t0 + 0.5 * width, t0 + 3 * width):
        val, _ = integrate.quad(lambda s: dipole_current(src, s), t_start, t,
                                epsabs=1e-13, epsrel=1e-12, limit=200)
        assert abs(val - moment(src, t)) <= 1e-10 * abs(amp), (t, val)
    total, _ = integrate.quad(lambda s: dipole_current(src, s), t_start, t0 + 12 * width,
                              epsabs=1e-13, epsrel=1e-12, limit=200)
    assert abs(total) <= 1e-10 * abs(amp)


def test_current_extremes_closed_form():
    src = Dipole(t0=1.0, width=0.25, amplitude=1.0)
    tau = src.width
    peak = src.amplitude * math.exp(-0.5) / (math.sqrt(2.0) * tau)
    t_lo, t_hi = src.t0 - math.sqrt(2.0) * tau, src.t0 + math.sqrt(2.0) * tau
    assert dipole_current(src, t_lo) == pytest.approx(peak, rel=1e-14)
    assert dipole_current(src, t_hi) == pytest.approx(-peak, rel=1e-14)
    ts = np.linspace(src.t0 - 6 * tau, src.t0 + 6 * tau, 20001)
    js = np.array([dipole_current(src, t) for t in ts])
    assert js.max() <= peak * (1 + 1e-12)
    assert abs(ts[np.argmax(js)] - t_lo) < 2 * (ts[1] - ts[0])
    assert dipole_current(src, src.t0) == 0.0
