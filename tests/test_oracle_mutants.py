"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/sph_oracle.cpp (a flipped
sign, a dropped factor, a wrong coefficient or index, transposed operands, a
wrong branch), builds it on the CPU and runs the fast pins against it: at
least one pin must fail.  The oracle itself is never modified."""
import concurrent.futures as cf
import os
import subprocess

import pytest

import oracle
from paper_2207_11328_gb300 import scenes
from tests import test_oracle_integration as ti
from tests import test_oracle_kernel_eos as tk
from tests import test_oracle_models as tm
from tests import test_oracle_neighbors as tn
from tests import test_oracle_physics as tp

MUTANTS = [
    ("continuity sign", "drho += mc * udotx * F;", "drho -= mc * udotx * F;"),
    ("pressure term without m_j", "T coef = T(m[j]) * bracket * F;", "T coef = bracket * F;"),
    ("pressure sign", "for (int c = 0; c < 3; ++c) a[c] -= coef * d[c];",
     "for (int c = 0; c < 3; ++c) a[c] += coef * d[c];"),
    ("gradient coefficient", "return T(105.0 / (128.0 * kPi", "return T(105.0 / (64.0 * kPi"),
    ("kernel coefficient", "return T(21.0 / (16.0 * kPi", "return T(21.0 / (8.0 * kPi"),
    ("kernel shape", "* t * t * t * t * (q * 2.0 + T(1.0));", "* t * t * t * (q * 2.0 + T(1.0));"),
    ("EOS binomial index", "binom = binom * (double)(gam - k + 1) / (double)k;",
     "binom = binom * (double)(gam - k) / (double)k;"),
    ("EOS constant B", "double B = P.rho0 * P.c0 * P.c0 / P.gamma;", "double B = P.rho0 * P.c0 / P.gamma;"),
    ("laminar coefficient", "lu = omega * 2.0 * mubar * F;", "lu = omega * mubar * F;"),
    ("laminar sign", "a[c] += lu * uij[c] + lx * d[c];", "a[c] -= lu * uij[c] + lx * d[c];"),
    ("harmonic mean", "return a * b * 2.0 / (a + b);", "return a * b / (a + b);"),
    ("geometric mean", "if (op == 2) return sqrt(a * b);", "if (op == 2) return (a + b) * 0.5;"),
    ("Monaghan K", "lx = omega * 2.0 * mubar * F * udotx / r2 * 5.0;", "lx = omega * 2.0 * mubar * F * udotx / r2 * 10.0;"),
    ("Espanol-Revenga shear coefficient", "mubar * (5.0 / 3.0) - zetabar", "mubar * (4.0 / 3.0) - zetabar"),
    ("Espanol-Revenga bulk sign", "mubar * (5.0 / 3.0) - zetabar", "mubar * (5.0 / 3.0) + zetabar"),
    ("Espanol-Revenga projection", "(mubar / 3.0 + zetabar) * 5.0 * udotx / r2", "(mubar / 3.0 + zetabar) * 3.0 * udotx / r2"),
    ("formulation 2 density ratio", "T mc = form2 ? T(m[j]) * rho[i] / rho[j] : T(m[j]);",
     "T mc = form2 ? T(m[j]) * rho[j] / rho[i] : T(m[j]);"),
    ("formulation 2 pressure denominator", "eos_pressure(delta[j], P)) / (rho[i] * rho[j])",
     "eos_pressure(delta[j], P)) / (rho[i] * rho[i])"),
    ("diffusion sign", "(rho[i] - rho[j]) * F", "(rho[j] - rho[i]) * F"),
    ("diffusion volume", "* F * T(m[j]) / rho[j];", "* F * T(m[j]) / rho[i];"),
    ("diffusion factor 2", "T(2.0 * P.ddiff_coef * h * P.c0)", "T(P.ddiff_coef * h * P.c0)"),
    ("diffusion through boundary", "if (P.ddiff == 1 && fluid_i && fluid_j) {", "if (P.ddiff == 1 && fluid_i) {"),
    ("cubic spline inner piece", "q * q * q * 0.75);", "q * q * q * 0.5);"),
    ("cubic spline gradient outer piece", "(t * t * -0.75) / q;", "(t * t * -0.75);"),
    ("quadratic gradient", "* (q - T(2.0)) / q;", "* (q - T(2.0));"),
    ("Gaussian normalisation", "- (Q / 2.0 + Q * Q * Q / 3.0) * std::exp(-Q * Q);", "- (Q / 2.0) * std::exp(-Q * Q);"),
    ("Gaussian gradient factor", "-T(1.0 / (2.0 * kPi * h5 * gaussian_S(Q)))", "-T(1.0 / (4.0 * kPi * h5 * gaussian_S(Q)))"),
    ("viscosity switch", "if (P.visc_model == 0 && pv(udotx) < 0.0) {", "if (P.visc_model == 0 && pv(udotx) > 0.0) {"),
    ("viscosity density mean", "T rhobar = (rho[i] + rho[j]) * 0.5;", "T rhobar = (rho[i] + rho[j]);"),
    ("transposed separation", "d[a] = xi[a] - xj[a];", "d[a] = xj[a] - xi[a];"),
    ("minimum image", "double k = std::nearbyint(pv(d[a]) / L);", "double k = std::floor(pv(d[a]) / L);"),
    ("bins smaller than the radius", "int k = (int)std::floor(P.size[a] / R);",
     "int k = (int)std::floor(P.size[a] / R) + 1;"),
    ("gravity on boundary particles", "for (int c = 0; c < 3; ++c) a_out[c] = T(0.0);",
     "for (int c = 0; c < 3; ++c) a_out[c] = T(P.g[c]);"),
    ("boundary velocity used", "uij[c] = ui[c] - (fluid_j ? u[3 * j + c] : T(0.0));", "uij[c] = ui[c] - u[3 * j + c];"),
    ("predictor full step", "us[3 * i + c] = u[3 * i + c] + T(0.5 * dt) * a[3 * i + c];",
     "us[3 * i + c] = u[3 * i + c] + T(dt) * a[3 * i + c];"),
    ("corrector forward Euler position", "x[3 * i + c] = x[3 * i + c] + T(0.5 * dt) * (u[3 * i + c] + un);",
     "x[3 * i + c] = x[3 * i + c] + T(dt) * un;"),
    ("density integrated without 1/rho0", "delta[i] = delta[i] + T(dt / rho0) * drho[i];",
     "delta[i] = delta[i] + T(dt) * drho[i];"),
    ("CFL acceleration branch", "dt = std::min(dt, std::sqrt(P.h / std::sqrt(amax2)));",
     "dt = std::min(dt, P.h / std::sqrt(amax2));"),
    ("viscous time step scaled by the CFL factor", "dt = std::min(dt, kViscousDtCoef * P.h * P.h / P.nu);",
     "dt = std::min(dt, P.cfl * P.h * P.h / P.nu);"),
    ("dual sqrt derivative", "return Dual(s, a.d / (2.0 * s));", "return Dual(s, a.d / s);"),
    ("dual product rule", "return Dual(a.v * b.v, a.d * b.v + a.v * b.d);", "return Dual(a.v * b.v, a.d * b.v);"),
]


def _box8():
    s = scenes.periodic_box(n_per_axis=8, dp=0.02)
    return s, s.pos + scenes.seeded_normal(s.pos.shape, 0.1 * 0.02, 7)


# fast pins first; each returns normally or raises AssertionError
BATTERY = [
    tk.test_unit_integral, tk.test_F_moment_closed_form, tk.test_shape_matches_listing, tk.test_F_is_dW_dr_over_r,
    lambda: tk.test_eos_binomial_exact(0.01), tk.test_eos_sound_speed,
    lambda: tn.test_brute_matches_numpy(7), lambda: tn.test_grid_matches_brute(7), tn.test_lattice_interior_count_is_80,
    tp.test_continuity_linear_field, tp.test_continuity_sign_approaching_pair, tp.test_pressure_gradient_linear_density,
    tp.test_mass_factor_in_pressure_term, tp.test_artificial_viscosity_switch, tp.test_laminar_shear_closed_form,
    tp.test_boundary_particles, tp.test_cfl_dt_branches, tp.test_viscous_time_step_is_within_the_stable_range,
    lambda: tp.test_momentum_conserved_periodic(1, 0.0, 0.1),
    lambda: ti.test_jvp_matches_central_differences_smooth(_box8()),
    ti.test_first_dt_from_initial_forces_and_cfl,
    # model options (Table 1, Section 3)
    *[lambda k=k, Q=Q: tm.test_kernel_unit_integral(k, Q) for k, Q in tm.KERNELS],
    *[lambda k=k, Q=Q: tm.test_kernel_F_is_dW_dr_over_r(k, Q) for k, Q in tm.KERNELS],
    tm.test_averaging_operators_are_the_three_means,
    *[lambda m=m, f=f, e=e: tm.test_viscous_models_continuum_limit(0, 2.0, m, f, e)
      for m, f, e in [(2, "stretch", 6.0), (3, "shear", 2.0), (3, "stretch", 8.0 / 3.0)]],
    lambda: tm.test_bulk_viscosity_acts_on_divergence_only("stretch", 2.0),
    tm.test_formulation2_conserves_momentum, tm.test_formulation2_continuity_weights_volumes,
    tm.test_density_diffusion_laplacian, tm.test_density_diffusion_conserves_volume_weighted_mass,
    tm.test_density_diffusion_sign_and_fluid_pairs_only,
    # the slow pins last: most mistakes fail an earlier one
    ti.test_energy_non_increasing_with_artificial_viscosity, tp.test_artificial_viscosity_shear_decay,
    ti.test_predictor_corrector_second_order,
]


def _compile(src_text, path):
    src = path.with_suffix(".cpp")
    src.write_text(src_text)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                           str(src), "-o", str(path)])
    return str(path)


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    """Every mutant (and an unmutated copy) compiled once, in parallel."""
    with open(oracle._SRC) as f:
        source = f.read()
    d = tmp_path_factory.mktemp("mutants")
    jobs = {"(unmutated)": source}
    for name, old, new in MUTANTS:
        assert source.count(old) >= 1, f"mutation site not found: {name}"
        jobs[name] = source.replace(old, new, 1)
    with cf.ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        futs = {k: ex.submit(_compile, v, d / f"m{i}.so") for i, (k, v) in enumerate(jobs.items())}
        return {k: f.result() for k, f in futs.items()}


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, libs):
    with oracle.using(libs[name]):
        for pin in BATTERY:
            try:
                pin()
            except (AssertionError, RuntimeError):
                return
    pytest.fail(f"planted mistake '{name}' passed every pin")


def test_unmutated_copy_passes_the_battery(libs):
    with oracle.using(libs["(unmutated)"]):
        for pin in BATTERY:
            pin()
    assert os.path.exists(libs["(unmutated)"])
