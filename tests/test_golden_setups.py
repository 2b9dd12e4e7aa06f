"""The paper's printed rising-bubble setups (tests/golden/rising_bubble_setups.txt,
Section 6) through the input recipe: the lattice parameters the recipe derives
reproduce each printed dimensionless group (Eo, Re_Gr, t_ref, Section 6.1
definitions), and the oracle's relaxation rates for them lie in the stable range
(0, 2) of the scheme (Section 3: s_nu = 1/(tau + 1/2), omega_phi = 1/(tau_phi + 1/2))."""
import math
import os

import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _setups():
    rows = []
    with open(os.path.join(HERE, "golden", "rising_bubble_setups.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            label, *vals = line.split()
            Eo, Re, D, t_ref, xi, M, rho_ratio, mu_ratio = (float(v) for v in vals)
            rows.append((label, Eo, Re, D, t_ref, xi, M, rho_ratio, mu_ratio))
    return rows


SETUPS = _setups()


def test_fixture_lists_every_printed_setup():
    labels = [r[0] for r in SETUPS]
    assert labels == ["fig6a", "fig6b", "fig6c", "fig6d", "fig6e", "fig6f", "field"]
    assert sum(1 for r in SETUPS if r[1] == 30.0 and r[0].startswith("fig6")) == 3  # Fig. 7's Eo


@pytest.mark.parametrize("row", SETUPS, ids=[r[0] for r in SETUPS])
def test_recipe_reproduces_the_printed_groups(row, orc):
    label, Eo, Re, D, t_ref, xi, M, rho_ratio, mu_ratio = row
    Mo = Eo ** 3 / Re ** 4  # Re_Gr = (Eo^3 / Mo)^(1/4)
    g, sigma, nu_H = W._bubble_params(D, Eo, Mo, t_ref)
    rho_H = 1.0
    mu_H = rho_H * nu_H
    assert math.sqrt(D / g) == pytest.approx(t_ref, rel=1e-12)                      # t_ref = sqrt(D / g)
    assert g * rho_H * D * D / sigma == pytest.approx(Eo, rel=1e-12)                # Eo
    assert rho_H * math.sqrt(g * D ** 3) / mu_H == pytest.approx(Re, rel=1e-12)     # Re_Gr
    prob = W.Problem(64, 64, 64, wall=(0, 1, 0), q_hydro=19, rho_H=rho_H, rho_ratio=rho_ratio, nu_H=nu_H,
                     mu_ratio=mu_ratio, sigma=sigma, xi=xi, mobility=M, gravity=(0.0, -g, 0.0))
    d = orc.derived(orc.make_problem(prob))
    for tau in (d["tau_H"], d["tau_L"]):
        assert 0.0 < 1.0 / (tau + 0.5) < 2.0
    assert 0.0 < d["omega_phi"] < 2.0
    assert d["omega_phi"] == pytest.approx(1.0 / (3.0 * M + 0.5), rel=1e-12)
    assert d["beta"] == pytest.approx(12.0 * sigma / xi, rel=1e-12) and d["kappa"] == pytest.approx(1.5 * sigma * xi, rel=1e-12)
