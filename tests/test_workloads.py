"""Seeded input recipes (host only): the batched rising-bubble draws."""
import numpy as np

import workloads as W


def test_batched_recipe():
    draws = W.batched()
    assert len(draws) == 64
    again = W.batched()
    for (p, phi, d), (p2, phi2, d2) in zip(draws, again):  # reproducible from the seed
        assert d == d2 and np.array_equal(phi, phi2)
    for prob, phi0, d in draws:
        assert d["size"] in W.BATCH_SIZES and (prob.nx, prob.ny, prob.nz) == d["size"]
        assert d["D"] == prob.nx / 4 and 1.0 <= d["Eo"] <= 50.0 and d["rho_ratio"] in (10.0, 100.0, 1000.0)
        assert prob.wall == (1, 1, 1) and prob.q_hydro == 27
        g = -prob.gravity[1]
        assert abs(np.sqrt(g * d["D"]) - 0.016) < 1e-12                       # u_s = sqrt(g D)
        assert abs(prob.rho_H * np.sqrt(g * d["D"] ** 3) / (prob.rho_H * prob.nu_H) - 30.0) < 1e-9  # Re_Gr
        assert abs(prob.rho_H * g * d["D"] ** 2 / prob.sigma - d["Eo"]) < 1e-9 * d["Eo"]          # Eo
        for nu in (prob.nu_H, prob.nu_L):
            assert 0.05 < 1.0 / (3.0 * nu + 0.5) < 1.98
        assert phi0.shape == prob.shape and phi0.dtype == np.float32
        # light bubble of diameter D at height 2 D, centred in x and z
        light = 1.0 - phi0.astype(np.float64)
        zc, yc, xc = (float((light * c).sum() / light.sum()) for c in np.meshgrid(
            *(np.arange(n) + 0.5 for n in prob.shape), indexing="ij"))
        assert abs(xc - prob.nx / 2) < 0.5 and abs(zc - prob.nz / 2) < 0.5 and abs(yc - 2 * d["D"]) < 0.5
