"""Pins of the oracle's smoothing kernel and equation of state against facts
the paper and the mathematics fix (not against the oracle itself).

Wendland C2 (Section 4 kernel-template listing, w = (2q+1)(1-q/2)^4,
f = (q-2)^3) with the unit-integral and compact-support properties of
Section 2.1; Cole equation of state of Section 2.1.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

import oracle

H = 0.026


def test_unit_integral():
    # Section 2.1: the kernel is unitary, int W dV = 1 (3D, radial)
    val, err = integrate.quad(lambda r: 4 * math.pi * r * r * oracle.kernel_W(r, H), 0, 2 * H,
                              epsabs=1e-14, epsrel=1e-12, limit=200)
    assert abs(val - 1.0) <= 1e-12


def test_compact_support():
    # Section 2.1: W = 0 for r > kh with k = 2 (Wendland "radius 2")
    for r in (2 * H, 2.0001 * H, 3 * H):
        assert oracle.kernel_W(r, H) == 0.0
        assert oracle.kernel_F(r, H) == 0.0
    assert oracle.kernel_W(1.999 * H, H) > 0.0


def test_F_is_dW_dr_over_r():
    # Section 2.1: grad W = r F with F = (1/r) d omega / dr
    for q in np.linspace(0.05, 1.95, 39):
        r = q * H
        eps = 1e-6 * H
        dWdr = (oracle.kernel_W(r + eps, H) - oracle.kernel_W(r - eps, H)) / (2 * eps)
        F = oracle.kernel_F(r, H)
        assert abs(dWdr / r - F) <= 1e-8 * abs(F) + 1e-6


def test_F_moment_closed_form():
    # integration by parts of a unit kernel: int x . grad W dV = -3 int W dV = -3,
    # i.e. 4 pi int r^4 F dr = -3 (pins the gradient coefficient independently of W)
    val, _ = integrate.quad(lambda r: 4 * math.pi * r ** 4 * oracle.kernel_F(r, H), 0, 2 * H,
                            epsabs=1e-14, epsrel=1e-12, limit=200)
    assert abs(val + 3.0) <= 1e-11


def test_shape_matches_listing():
    # The listing's shape functions up to the normalisation constant:
    # W(q)/W(0) = (2q+1)(1-q/2)^4 and F(q)/F(0) = (q-2)^3 / (-8)
    W0, F0 = oracle.kernel_W(0.0, H), oracle.kernel_F(1e-300, H)
    for q in (0.1, 0.5, 1.0, 1.5, 1.9):
        assert oracle.kernel_W(q * H, H) / W0 == pytest.approx((2 * q + 1) * (1 - q / 2) ** 4, rel=1e-13)
        assert oracle.kernel_F(q * H, H) / F0 == pytest.approx((q - 2) ** 3 / -8.0, rel=1e-13)


def test_shape_matches_the_golden_values():
    # tests/golden/kernel_shapes.txt: exact values of the printed Wendland polynomials
    path = os.path.join(os.path.dirname(__file__), "golden", "kernel_shapes.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) >= 5
    W0, F0 = oracle.kernel_W(0.0, H), oracle.kernel_F(1e-300, H)
    w0, f0 = Fraction(rows[0][1]), Fraction(rows[0][2])
    for q, w, f in rows:
        q, w, f = Fraction(q), Fraction(w), Fraction(f)
        assert oracle.kernel_W(float(q) * H, H) / W0 == pytest.approx(float(w / w0), rel=1e-13, abs=1e-15)
        assert oracle.kernel_F(float(q) * H, H) / F0 == pytest.approx(float(f / f0), rel=1e-13, abs=1e-15)


def _exact_pressure(delta, rho0, c0, gamma):
    # (1+delta)^gamma - 1 in exact rational arithmetic
    d = Fraction(delta)
    B = Fraction(rho0) * Fraction(c0) ** 2 / gamma
    return float(B * ((1 + d) ** gamma - 1))


@pytest.mark.parametrize("delta", [0.0, 1e-9, -3e-7, 1e-4, -2e-3, 0.01, 0.05, -0.05])
def test_eos_binomial_exact(delta):
    # Section 2.1: P = B((rho/rho0)^gamma - 1), B = rho0 c0^2/gamma
    p = oracle.params(rho0=1000.0, c0=20.0, gamma=7.0)
    exact = _exact_pressure(delta, 1000.0, 20.0, 7)
    got = oracle.eos(p, delta)
    assert got == pytest.approx(exact, rel=1e-14, abs=1e-300)


def test_eos_sound_speed():
    # dP/drho at rest = c0^2 (definition of B)
    c0, rho0 = 17.155, 1000.0
    p = oracle.params(rho0=rho0, c0=c0, gamma=7.0)
    e = 1e-7
    dPdrho = (oracle.eos(p, e) - oracle.eos(p, -e)) / (2 * e * rho0)
    assert dPdrho == pytest.approx(c0 * c0, rel=1e-9)
