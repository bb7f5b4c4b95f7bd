"""Pin of the generators' initial density: the hydrostatic relative density
that the dam-break, resting-tank and sloshing generators assign must give,
through the equation of state, the hydrostatic pressure of its depth,

    P(delta_0(z)) = rho0 g (H - z)   (zero above the free surface),

Section 2.1 (Cole's equation of state) with the column at rest.  Both the
CUDA path and the oracle start from this array, so a mistake in it would be
invisible to GPU-vs-oracle parity; here it is checked against the
definition of hydrostatic pressure, with P from the oracle's equation of
state (itself pinned to the exact rational (1 + delta)^gamma - 1 elsewhere).

Tolerance: delta is stored in FP32, so P may be off by dP/ddelta times one
FP32 rounding of delta: rho0 c0^2 (1 + delta)^(gamma-1) 2^-24 |delta|."""
import math

import numpy as np

import oracle
from paper_2207_11328_gb300 import scenes


def _check(s, depth, c0, what):
    p = oracle.params(s, c0=c0)
    d = s.delta.astype(np.float64)
    P = np.array([oracle.eos(p, x) for x in d])
    expect = s.rho0 * abs(s.g[2]) * depth
    tol = 1.1 * s.rho0 * c0 * c0 * (1.0 + np.abs(d)) ** (s.gamma - 1) * 2.0 ** -24 * np.abs(d) \
        + 1e-9 * s.rho0 * abs(s.g[2]) * max(depth.max(), 1e-3)
    err = np.abs(P - expect)
    assert np.all(err <= tol), f"{what}: worst {err.max():.3e} Pa at depth {depth[np.argmax(err / tol)]:.4f} m"
    # the pressure really varies: a constant delta would fail the check above at depth
    assert depth.max() > 0 and P.max() > 0.5 * s.rho0 * abs(s.g[2]) * depth.max()
    # above the free surface (walls): zero density change, not a negative one
    assert np.all(s.delta[depth == 0.0] == 0.0)


def test_dam_break_initial_density_is_hydrostatic():
    dp = 0.02
    s = scenes.dam_break(dp=dp)
    H = int(round(0.3 / dp)) * dp          # top of the lattice column
    depth = np.maximum(H - s.pos[:, 2], 0.0)
    _check(s, depth, s.c0, "dam break")


def test_resting_tank_initial_density_is_hydrostatic():
    s = scenes.hydrostatic_tank(dp=0.02)
    H = int(round(0.3 / 0.02)) * 0.02
    depth = np.maximum(H - s.pos[:, 2], 0.0)
    _check(s, depth, s.c0, "resting tank")


def test_sloshing_tanks_initial_density_is_hydrostatic():
    # per tank: free surface tilted by 5 degrees about y through the tank centre,
    # z_s(x) = h_f + (x - L/2) tan 5deg, with h_f = c0^2 / (100 g) (c0 = 10 sqrt(g h_f))
    b = scenes.sloshing_batch(n_scenes=6, nmin=500, nmax=3000)
    g = abs(b.g[2])
    layers, margin = 3, 2.6 * b.dp
    for k, d in enumerate(b.scenes):
        m = b.scene == k
        one = scenes.subset(b, m)
        hf = d["c0"] ** 2 / (100.0 * g)
        L = d["size"][0] - 2 * (layers * b.dp + margin)
        x_local = one.pos[:, 0] - (d["origin"][0] + layers * b.dp + margin)
        zs = hf + (x_local - 0.5 * L) * math.tan(math.radians(5.0))
        depth = np.maximum(zs - one.pos[:, 2], 0.0)
        _check(one, depth, d["c0"], f"sloshing tank {k}")
