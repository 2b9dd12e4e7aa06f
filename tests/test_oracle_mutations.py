"""Mutation check of the oracle's pins.

Each entry plants one plausible mistake (a dropped term, a wrong sign, factor,
index or operand) in a private copy of ``oracle/acm_oracle.c``, compiles it on
the CPU and runs the closed-form, invariant and physics pins against it.  Every
mistake must make at least one pin fail.  The brute-force whole-step test (which
retypes the force formulas) and the derived-parameter test are deliberately not
in the pin list, so that no mutation is caught only by a retyped formula; the
literal moment-matrix MRT phase step is in it (it builds Omega = M^-1 S M from
the lattice, not from the oracle's closed form).
"""
import os

import numpy as np
import pytest

import test_oracle_bruteforce as B
import test_oracle_d2q9 as D
import test_oracle_identities as I
import test_oracle_physics as Ph

MUTATIONS = [
    ("gradient without 1/c_s^2", "for (int a = 0; a < 3; ++a) grad[a] /= CS2;", ""),
    ("Laplacian factor 2 dropped", "return 2.0 * s / CS2;", "return s / CS2;"),
    ("theta coefficient", "(1.0 - 4.0 * (phi_theta", "(1.0 - 2.0 * (phi_theta"),
    ("phase forcing half-step sign", "- 0.5 * F[i]) + F[i];", "+ 0.5 * F[i]) + F[i];"),
    ("Gamma quadratic coefficient", "eu * eu / (2.0 * CS2 * CS2)", "eu * eu / (CS2 * CS2)"),
    ("phase relaxation literal 1/tau_phi", "d.omega_phi = 1.0 / (tau_phi + 0.5);", "d.omega_phi = 1.0 / tau_phi;"),
    ("normal not normalised", "double inv = 1.0 / sqrt(G2);", "double inv = 1.0;"),
    ("pressure force sign", "F_p[a] = -pstar * CS2 * grad_rho[a];", "F_p[a] = pstar * CS2 * grad_rho[a];"),
    ("chemical potential kappa sign", "- d.kappa * lap_phi;", "+ d.kappa * lap_phi;"),
    ("beta coefficient", "d.beta = 12.0 * P->sigma / P->xi;", "d.beta = 6.0 * P->sigma / P->xi;"),
    ("viscous force dropped", "F_mu[a] = -(nu / CS2) * s;", "F_mu[a] = 0.0 * s;"),
    ("viscous force sign", "F_mu[a] = -(nu / CS2) * s;", "F_mu[a] = (nu / CS2) * s;"),
    ("buoyancy sign", "F_b[a] = (rho - P->rho_ref) * P->gravity[a];",
     "F_b[a] = (P->rho_ref - rho) * P->gravity[a];"),
    ("tau interpolation transposed", "(phi_m - phi_L) * (d.tau_H - d.tau_L)", "(phi_m - phi_L) * (d.tau_L - d.tau_H)"),
    ("s_nu without the 1/2 shift", "double s_nu = 1.0 / (tau + 0.5);", "double s_nu = 1.0 / (tau + 1.0);"),
    ("density interpolation transposed", "P->rho_L + (phi_m - phi_L) * (P->rho_H - P->rho_L)",
     "P->rho_H + (phi_m - phi_L) * (P->rho_L - P->rho_H)"),
    ("velocity without half force", "u[a] = j[a] + F[a] / (2.0 * rho);", "u[a] = j[a] + F[a] / rho;"),
    ("first-moment forcing dropped", "m1s[a] = u[a] + F[a] / (2.0 * rho);", "m1s[a] = u[a];"),
    ("second moments relax toward j j", "s_nu * u[a] * u[b];", "s_nu * j[a] * j[b];"),
    ("Hermite trace term dropped", "(L.e[i][a] * L.e[i][b] - (a == b ? CS2 : 0.0)) * a2s[a][b]",
     "(L.e[i][a] * L.e[i][b]) * a2s[a][b]"),
    ("bounce-back without reversal", "fnext[(long)L->opp[i] * N + cell_index(P, x, y, z)] = fstar[i];",
     "fnext[(long)i * N + cell_index(P, x, y, z)] = fstar[i];"),
    ("stencil x and y transposed", "nb[(e[2] + 1) * 9 + (e[1] + 1) * 3 + (e[0] + 1)]",
     "nb[(e[2] + 1) * 9 + (e[0] + 1) * 3 + (e[1] + 1)]"),
    ("wall ghosts wrap instead of mirror", "    if (walled) {", "    if (0) {"),
    ("D3Q15 corner weight", "1.0 / 9.0, 0.0, 1.0 / 72.0}", "1.0 / 9.0, 0.0, 1.0 / 36.0}"),
    ("pressure output without rho", "p[c] = aux[1] * aux[0] * CS2;", "p[c] = aux[1] * CS2;"),
    ("MRT phase: first-moment rate transposed", "(1.0 - d.omega_phi) * L.w[i] * eJ / CS2",
     "d.omega_phi * L.w[i] * eJ / CS2"),
    ("MRT phase: unweighted projection", "(1.0 - d.omega_phi) * L.w[i] * eJ / CS2",
     "(1.0 - d.omega_phi) * eJ / 10.0"),
    ("MRT phase: forcing half-step dropped", "y[i] = heq[i] - h[i] - 0.5 * F[i];", "y[i] = heq[i] - h[i];"),
    ("D2Q9: Hermite tensors over three dimensions", "const int D = L.dim;", "const int D = 3;"),
    ("D2Q9 diagonal weight", "{4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0}", "{4.0 / 9.0, 1.0 / 9.0, 1.0 / 18.0}"),
]


def _pins(orc):
    """Pins ordered from fast to slow; each is a zero-argument callable."""
    P = []
    for q in (15, 19, 27):
        P.append(lambda q=q: I.test_lattice_moments(orc, q))
        P.append(lambda q=q: I.test_stencils_exact_on_quadratics(orc, q))
    P += [
        lambda: D.test_d2q9_lattice_moments(orc),
        lambda: D.test_d2q9_hydro_collision_moments(orc),
        lambda: I.test_stencil_walls_mirror(orc),
        lambda: I.test_phase_collision_moments(orc, 15),
        lambda: I.test_phase_normal_zero_gradient(orc, 15),
        lambda: I.test_hydro_collision_moments(orc, 19),
        lambda: I.test_hydro_collision_moments(orc, 27),
        lambda: I.test_hydro_forces_vanish_in_uniform_phase(orc),
        lambda: I.test_chemical_potential_vanishes_on_equilibrium_profile(orc, 27),
        lambda: I.test_mass_conservation(orc, (1, 1, 1), 27, 15),
        lambda: I.test_trivial_states(orc, 19),
        lambda: Ph.test_phase_diffusion_rate(orc, 0, 15),
        lambda: Ph.test_phase_diffusion_rate(orc, 1, 15),
        lambda: B.test_literal_mrt_phase_step(orc, 15),
        lambda: Ph.test_shear_wave_viscosity(orc, 19),
        lambda: Ph.test_planar_interface_steady(orc, 27, 15),
        lambda: Ph.test_interface_advection(orc),
        lambda: Ph.test_hydrostatic_balance(orc, 10.0),
        lambda: Ph.test_hydrostatic_balance(orc, 1000.0),
        lambda: Ph.test_two_layer_poiseuille_diffuse(orc, 1.0, 10.0, 0.5, 4.0, 19, 2e-3),
        lambda: Ph.test_two_layer_poiseuille_diffuse(orc, 10.0, 1.0, 0.05, 8.0, 19, 1.5e-2),
        lambda: Ph.test_two_layer_poiseuille_diffuse(orc, 1000.0, 100.0, 0.05, 4.0, 27, 1e-2),
        lambda: Ph.test_laplace_law_cylinder(orc),
        lambda: D.test_d2q9_shear_wave_viscosity(orc),
    ]
    return P


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(orc, tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(orc.__file__), "acm_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = tmp_path / "acm_oracle_mutated.c"
    mutated.write_text(src.replace(old, new))
    so = orc.compile_source(str(mutated), str(tmp_path / "libmutated.so"))
    caught = None
    with orc.using_library(so), np.errstate(all="ignore"):
        for i, pin in enumerate(_pins(orc)):
            try:
                pin()
            except Exception:  # an assertion, or NaN / overflow turned into an error
                caught = i
                break
    assert caught is not None, f"no pin catches: {name}"
