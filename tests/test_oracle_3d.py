"""Pins for the 3D oracle (oracle.mrcm3d).

Each check is fixed by mathematics or by the paper, not by the 3D oracle
itself: linear pressure and a layered medium's closed form for the fine
solve; two independently written assemblies (array operations in O1, cell
loops in the leaf problem) agreeing; MRCM equal to the fine solution when
every patch is one fine face; a one-cell-thick 3D slab equal to the pinned
2D oracle; strips exact for a uniform flow; Eqs. 13.2 / 14.2 and cell
conservation in the final fields; symmetric Robin-to-flux maps; the patch
counts of Table ntmmbfs.
"""
import os

import numpy as np
import pytest

import inputs
from oracle.mrcm import solve_mrcm
from oracle.mrcm3d import Decomposition3D, LeafProblem3D, solve_fine3d, solve_mrcm3d
from conftest import rel

BCS = ["left_right", "quarter_five_spot"]


def _faces(r):
    return np.concatenate([r["Fx"].ravel(), r["Fy"].ravel(), r["Fz"].ravel()])


def test_fine_linear_pressure_exact():
    # K = 1, p = 1 / 0 on x = 0 / 1, no flow elsewhere: p = 1 - x at the cell
    # centres and the flux density is 1 on every x-face
    prob = inputs.darcy_problem_3d(10, 6, 4, sigma2=0.0, bc="left_right")
    f = solve_fine3d(prob)
    hx, hy, hz = prob.h
    x = (np.arange(prob.nx) + 0.5) * hx
    assert np.abs(f["p"] - (1.0 - x)[None, None, :]).max() < 1e-13
    assert np.abs(f["Fx"] - hy * hz).max() < 1e-13 * hy * hz
    assert np.abs(f["Fy"]).max() < 1e-14 and np.abs(f["Fz"]).max() < 1e-14


def test_fine_layered_medium_closed_form():
    # K varies along x only: every x-face carries the same flux density
    # 1 / sum_i (h / K_i) (series resistances, half cells at both Dirichlet
    # faces), and p drops by that flux times each half-cell resistance
    nx, ny, nz = 12, 3, 5
    Kx = np.exp(np.random.default_rng(3).normal(0.0, 1.5, nx))
    K = np.broadcast_to(Kx[None, None, :], (nz, ny, nx))
    prob = inputs.darcy_problem_3d(nx, ny, nz, K=K, bc="left_right")
    f = solve_fine3d(prob)
    hx, hy, hz = prob.h
    u = 1.0 / np.sum(hx / Kx)
    assert np.abs(f["Fx"] / (hy * hz) - u).max() < 1e-11 * u
    p_expect = 1.0 - u * (np.cumsum(hx / Kx) - hx / (2 * Kx))
    assert np.abs(f["p"] - p_expect[None, None, :]).max() < 1e-11


@pytest.mark.parametrize("bc", BCS)
def test_fine_conservation(bc):
    prob = inputs.darcy_problem_3d(9, 7, 6, sigma2=2.0, corr=(0.3, 0.3, 0.1), seed=5, bc=bc)
    f = solve_fine3d(prob)
    div = (np.diff(f["Fx"], axis=2) + np.diff(f["Fy"], axis=1) + np.diff(f["Fz"], axis=0))
    assert np.abs(div - prob.q).max() < 1e-12 * np.abs(f["Fx"]).max()


def test_fine_equals_one_leaf_local_problem():
    # one leaf covering the grid has no patches: its local problem (built by
    # cell loops) is the fine problem (built by array operations)
    prob = inputs.darcy_problem_3d(7, 6, 5, sigma2=2.0, corr=(0.3, 0.3, 0.3), seed=2,
                                   bc="left_right", sub=(8, 8, 8))
    dec = Decomposition3D(prob)
    assert len(dec.leaves) == 1 and not dec.segments
    lp = LeafProblem3D(dec, 0)
    pl, _, faces = lp.solve(np.zeros(0), with_data=True)
    f = solve_fine3d(prob)
    p = np.zeros(prob.K.shape)
    lp.place(p, pl)
    assert rel(p, f["p"]) < 1e-13
    for (d, k, j, i), val in faces.items():
        F = (f["Fx"], f["Fy"], f["Fz"])[d]
        assert abs(val - F[k, j, i]) < 1e-13 * np.abs(f["Fx"]).max()


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("alpha", [1e-3, 1.0, 1e3])
def test_one_face_patches_equal_fine(bc, alpha):
    # a patch of one face turns the Robin pair into the two-point flux, so
    # MRCM equals O1 for every alpha
    prob = inputs.darcy_problem_3d(8, 6, 6, sigma2=2.0, corr=(0.3, 0.3, 0.2), seed=4, bc=bc,
                                   sub=(4, 3, 4), seg=(1, 1, 1), alpha=alpha)
    f, m = solve_fine3d(prob), solve_mrcm3d(prob)
    assert rel(m["p"], f["p"]) < 1e-11
    assert rel(_faces(m), _faces(f)) < 1e-11
    assert rel(m["Fa_y"], m["Fb_y"]) < 1e-11


@pytest.mark.parametrize("bc", BCS)
def test_one_cell_slab_equals_the_2d_oracle(bc):
    # nz = 1 with no flow through z: the 3D equations are the 2D ones times
    # the thickness hz, provided beta matches.  2D: beta = alpha2 L / Keff
    # (L the segment length); 3D: beta = alpha3 sqrt(L hz) / Keff.
    n, sub, seg, alpha2 = 24, 8, 4, 1.5
    p2 = inputs.darcy_problem(n, n, sigma2=2.0, corr=0.2, seed=7, bc=bc, sub=(sub, sub),
                              seg=(seg, seg), alpha=alpha2)
    hz = 1.0 / n
    L = seg / n
    alpha3 = alpha2 * L / np.sqrt(L * hz)
    p3 = inputs.darcy_problem_3d(n, n, 1, K=p2.K[None], bc=bc, sub=(sub, sub, 1),
                                 seg=(seg, seg, 1), alpha=alpha3, L=(1.0, 1.0, hz))
    p3.q = hz * p2.q[None]           # 2D sources are per unit depth
    m2, m3 = solve_mrcm(p2), solve_mrcm3d(p3)
    assert rel(m3["p"][0], m2["p"]) < 1e-12
    assert rel(m3["Fx"][0], hz * m2["Fx"]) < 1e-12
    assert rel(m3["Fy"][0], hz * m2["Fy"]) < 1e-12
    assert rel(m3["Fa_x"][0], hz * m2["Fa_x"]) < 1e-12
    assert np.abs(m3["Fz"]).max() < 1e-14


def test_strip_decomposition_exact_for_linear_pressure():
    # interfaces perpendicular to a uniform flow carry constant p and u
    prob = inputs.darcy_problem_3d(16, 8, 8, sigma2=0.0, bc="left_right", sub=(4, 8, 8),
                                   seg=(4, 4, 4))
    f, m = solve_fine3d(prob), solve_mrcm3d(prob)
    assert rel(m["p"], f["p"]) < 1e-13
    assert rel(_faces(m), _faces(f)) < 1e-13


@pytest.mark.parametrize("bc", BCS)
def test_interface_conditions_and_conservation(bc):
    prob = inputs.darcy_problem_3d(16, 12, 8, sigma2=2.0, corr=(0.3, 0.3, 0.1), seed=8, bc=bc,
                                   sub=(8, 6, 4), seg=(4, 3, 2), alpha=2.0)
    m = solve_mrcm3d(prob)
    dec = m["dec"]
    Fa = [m["Fa_x"], m["Fa_y"], m["Fa_z"]]
    Fb = [m["Fb_x"], m["Fb_y"], m["Fb_z"]]
    scale = np.abs(m["Fx"]).max()
    for t in dec.segments:
        keys = dec.face_keys(t)
        fa = sum(Fa[d][k, j, i] for d, k, j, i in keys)
        fb = -sum(Fb[d][k, j, i] for d, k, j, i in keys)
        assert abs(fa + fb) < 1e-12 * scale                                      # Eq. (13.2)
        assert abs(fa - fb - 2 * m["U"][t["id"]] * t["length"]) < 1e-12 * scale  # Eq. (14.2)
    for lf in dec.leaves:
        (i0, j0, k0), (i1, j1, k1) = lf["lo"], lf["hi"]
        Fx = Fa[0][k0:k1, j0:j1, i0:i1 + 1].copy(); Fx[:, :, 0] = Fb[0][k0:k1, j0:j1, i0]
        Fy = Fa[1][k0:k1, j0:j1 + 1, i0:i1].copy(); Fy[:, 0, :] = Fb[1][k0:k1, j0, i0:i1]
        Fz = Fa[2][k0:k1 + 1, j0:j1, i0:i1].copy(); Fz[0] = Fb[2][k0, j0:j1, i0:i1]
        div = np.diff(Fx, axis=2) + np.diff(Fy, axis=1) + np.diff(Fz, axis=0)
        assert np.abs(div - prob.q[k0:k1, j0:j1, i0:i1]).max() < 1e-12 * scale


def test_leaf_map_properties():
    prob = inputs.darcy_problem_3d(16, 8, 8, sigma2=2.0, corr=(0.3, 0.3, 0.2), seed=5,
                                   bc="left_right", sub=(8, 8, 4), seg=(4, 4, 2))
    dec = Decomposition3D(prob)
    for lf in dec.leaves:
        lp = LeafProblem3D(dec, lf["id"])
        R, rbar = lp.robin_to_flux()
        scale = np.abs(R).max()
        assert np.abs(R - R.T).max() < 1e-13 * scale
        assert np.linalg.eigvalsh(-0.5 * (R + R.T)).min() > -1e-12 * scale
        if not any(f[0] == "dir" for f in lp.faces.values()):
            assert np.abs(R.sum(axis=1)).max() < 1e-13 * scale


def test_patch_counts_reproduce_table_ntmmbfs():
    # Section 5.1: a x b x 1 subdomains (z never cut); one local solve per
    # patch of a subdomain plus its particular solution, with H-bar = H and
    # with H-bar = H/4 in x and y
    path = os.path.join(os.path.dirname(__file__), "golden", "ntmmbfs.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    for a, b, c, n1, n4, _ in rows[:3]:
        a, b, c = int(a), int(b), int(c)
        for seg, expect in (((4, 4, 4), int(n1)), ((1, 1, 4), int(n4))):
            prob = inputs.darcy_problem_3d(4 * a, 4 * b, 4 * c, sigma2=0.0, sub=(4, 4, 4), seg=seg)
            dec = Decomposition3D(prob)
            assert sum(len(lf["segs"]) + 1 for lf in dec.leaves) == expect
