"""Pins for O1, the fine two-point-flux (lumped RT0) solve (Eqs. ellip.1-3)."""
import numpy as np
import pytest

import inputs
from inputs.problems import DIRICHLET, NEUMANN
from oracle.fine import solve_fine
from conftest import rel


def _balance(prob, out):
    """Cell-wise conservation residual: outward flux sum - q."""
    Fx, Fy = out["Fx"], out["Fy"]
    div = Fx[:, 1:] - Fx[:, :-1] + Fy[1:, :] - Fy[:-1, :]
    return div - prob.q


def test_linear_pressure_constant_K():
    # constant K, p=1 at x=0, p=0 at x=Lx, no flow in y: TPFA is exact for
    # linear p, so p_c = 1 - x_c / Lx and every x-face carries K * hy / Lx.
    prob = inputs.darcy_problem(12, 8, sigma2=0.0, Lx=2.0, Ly=0.5, bc="left_right")
    prob.K[:] = 2.5
    out = solve_fine(prob)
    xc = (np.arange(prob.nx) + 0.5) * prob.hx
    assert np.abs(out["p"] - (1.0 - xc / prob.Lx)[None, :]).max() < 1e-13
    assert np.abs(out["Fx"] - 2.5 * prob.hy / prob.Lx).max() < 1e-13
    assert np.abs(out["Fy"]).max() < 1e-13


def test_harmonic_series_resistance():
    # K varying only in x: each row is a series of resistances h/K_i, so
    # the flux per row is hy * (1 - 0) / sum_i(hx / K_i).
    nx, ny = 17, 5
    rng = np.random.default_rng(7)
    kx = np.exp(rng.normal(0, 1.5, nx))
    K = np.tile(kx, (ny, 1))
    prob = inputs.darcy_problem(nx, ny, K=K, Lx=1.0, Ly=0.3, bc="left_right")
    out = solve_fine(prob)
    flux = prob.hy / np.sum(prob.hx / kx)
    assert np.abs(out["Fx"] - flux).max() < 1e-13 * max(1.0, flux) + 1e-15
    # pressure drop across cell i is flux * (hx/K_i)/hy from the inlet value 1
    drop = np.concatenate([[0.5 * prob.hx / kx[0]],
                           0.5 * prob.hx / kx[:-1] + 0.5 * prob.hx / kx[1:]]) * flux / prob.hy
    p_expect = 1.0 - np.cumsum(drop)
    assert np.abs(out["p"][2] - p_expect).max() < 1e-12


@pytest.mark.parametrize("bc", ["left_right", "quarter_five_spot"])
def test_conservation_heterogeneous(bc):
    prob = inputs.darcy_problem(24, 20, sigma2=4.0, corr=0.2, seed=11, bc=bc)
    out = solve_fine(prob)
    scale = np.abs(out["Fx"]).max()
    assert np.abs(_balance(prob, out)).max() < 1e-12 * scale
    if bc == "quarter_five_spot":
        assert abs(out["p"].mean()) < 1e-13 * np.abs(out["p"]).max()
        # no-flow boundary
        assert np.abs(out["Fx"][:, [0, -1]]).max() == 0.0
        assert np.abs(out["Fy"][[0, -1], :]).max() == 0.0


def test_dirichlet_face_flux_matches_half_cell_law():
    prob = inputs.darcy_problem(9, 7, sigma2=1.0, corr=0.3, seed=2, bc="left_right")
    out = solve_fine(prob)
    # x=0 face: flux into the domain = 2 K hy / hx (g - p_c)
    expect = 2 * prob.K[:, 0] * prob.hy / prob.hx * (1.0 - out["p"][:, 0])
    assert np.abs(out["Fx"][:, 0] - expect).max() < 1e-14 * np.abs(expect).max()
