"""Pins for O2 (global MRCM), the CPU Recursive MRCM and the leaf maps.

Each check is fixed by the paper's equations or by mathematics, not by the
oracle itself: MRCM equals the fine solution when every segment is one fine
face; the monolithic assembly of Eqs. 11.2-14.2 (no MMBFs) equals O2; the
recursion of Algorithm 1 equals the global system; the interface conditions
Eqs. 13.2 / 14.2 hold in the final fields; Robin-to-flux maps are symmetric
and annihilate constants on Dirichlet-free leaves.
"""
import numpy as np
import pytest

import inputs
from oracle.brute import solve_brute
from oracle.fine import solve_fine
from oracle.geometry import Decomposition
from oracle.local import LeafProblem
from oracle.mrcm import solve_mrcm
from oracle.recursive import RecursiveMRCM, solve_recursive
from conftest import rel

BCS = ["left_right", "quarter_five_spot"]


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("alpha", [1e-3, 1.0, 1e3])
def test_one_face_segments_equal_fine(bc, alpha):
    # U_H = u on a single face turns the Robin pair into the two-point flux
    # u (h/2K_a + h/2K_b) = p_a - p_b, so MRCM = O1 for every alpha.
    prob = inputs.darcy_problem(20, 14, sigma2=2.0, corr=0.2, seed=4, bc=bc,
                                sub=(6, 5), seg=(1, 1), alpha=alpha)
    f, m = solve_fine(prob), solve_mrcm(prob)
    assert rel(m["p"], f["p"]) < 1e-11
    assert rel(m["Fx"], f["Fx"]) < 1e-11
    assert rel(m["Fy"], f["Fy"]) < 1e-11
    # and the two one-sided skeleton fluxes coincide
    assert rel(m["Fa_x"], m["Fb_x"]) < 1e-11


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("seg,alpha", [((2, 2), 1.0), ((4, 4), 10.0), ((3, 2), 0.1), ((4, 1), 1.0)])
def test_brute_force_equals_global(bc, seg, alpha):
    prob = inputs.darcy_problem(16, 12, sigma2=3.0, corr=0.2, seed=9, bc=bc,
                                sub=(4, 4), seg=seg, alpha=alpha)
    m, b = solve_mrcm(prob), solve_brute(prob)
    assert rel(b["p"], m["p"]) < 1e-12


@pytest.mark.parametrize("bc", BCS)
def test_recursive_equals_global_and_tree_order(bc):
    prob = inputs.darcy_problem(40, 36, sigma2=3.0, corr=0.15, seed=21, bc=bc,
                                sub=(8, 8), seg=(4, 4), alpha=1.0)
    m = solve_mrcm(prob)
    for tie in ("x", "y"):
        r = solve_recursive(prob, tie=tie)
        for key in ("p", "Fx", "Fy", "Fa_x", "Fb_x", "Fa_y", "Fb_y"):
            assert rel(r[key], m[key]) < 1e-10, key


def test_node_maps_symmetric():
    prob = inputs.darcy_problem(32, 32, sigma2=2.0, corr=0.2, seed=3, bc="left_right",
                                sub=(8, 8), seg=(4, 4))
    rm = RecursiveMRCM(prob)
    rm.solve()
    stack = [rm.root]
    checked = 0
    while stack:
        nd = stack.pop()
        stack += nd.children
        if nd is not rm.root:
            assert np.abs(nd.R - nd.R.T).max() < 1e-12 * np.abs(nd.R).max()
            checked += 1
    assert checked == 2 * 16 - 2


def test_leaf_map_properties():
    prob = inputs.darcy_problem(24, 24, sigma2=2.0, corr=0.2, seed=5, bc="left_right",
                                sub=(8, 8), seg=(4, 4))
    dec = Decomposition(prob)
    for lf in dec.leaves:
        lp = LeafProblem(dec, lf["id"])
        R, rbar = lp.robin_to_flux()
        assert np.abs(R - R.T).max() < 1e-13 * np.abs(R).max()
        # -R is positive semi-definite (Robin-to-flux of a diffusion problem)
        assert np.linalg.eigvalsh(-0.5 * (R + R.T)).min() > -1e-12 * np.abs(R).max()
        has_dir = any(f[0] == "dir" for f in lp.faces.values())
        if not has_dir:
            # a uniform lambda gives p = lambda and no flux
            assert np.abs(R.sum(axis=1)).max() < 1e-13 * np.abs(R).max()
        # global balance of the particular solution: Robin outflow plus
        # boundary outflow equals the source inside the leaf
        _, _, faces = lp.solve(np.zeros(len(lp.segs)), with_data=True)
        out = 0.0
        for key, f in lp.faces.items():
            if f[0] in ("dir", "neu"):
                out += f[-1] * faces[key]
        q = prob.q[lp.j0:lp.j1, lp.i0:lp.i1].sum()
        assert abs(rbar.sum() + out - q) < 1e-12 * max(1.0, np.abs(rbar).sum())


def test_single_cell_leaf_closed_form():
    # a 1x1 leaf with four Robin faces: A = sum(rho), B = rho^T, hence
    # R = rho rho^T / sum(rho) - diag(rho)
    prob = inputs.darcy_problem(3, 3, sigma2=1.0, corr=0.5, seed=1, bc="left_right",
                                sub=(1, 1), seg=(1, 1), alpha=2.0)
    dec = Decomposition(prob)
    center = dec.leaf_id(1, 1)
    lp = LeafProblem(dec, center)
    R, _ = lp.robin_to_flux()
    K = prob.K[1, 1]
    rho = []
    for t in lp.segs:
        seg = dec.segments[t]
        hn, area = (prob.hx, prob.hy) if seg["axis"] == 0 else (prob.hy, prob.hx)
        rho.append(area / (hn / (2 * K) + seg["beta"]))
    rho = np.array(rho)
    expect = np.outer(rho, rho) / rho.sum() - np.diag(rho)
    assert np.abs(R - expect).max() < 1e-14 * np.abs(expect).max()


def test_robin_coefficient_worked_example():
    # Eq. (robin.beta)/(permeff) by hand on a 2-face segment of length 0.5:
    # K = 1, 4 in the left column and 2, 2 in the right one.
    K = np.array([[1.0, 2.0], [4.0, 2.0]])
    prob = inputs.darcy_problem(2, 2, K=K, Lx=1.0, Ly=0.5, sub=(1, 2), seg=(2, 2), alpha=3.0)
    dec = Decomposition(prob)
    assert len(dec.segments) == 1
    t = dec.segments[0]
    # harmonic means 2*1*2/3 = 4/3 and 2*4*2/6 = 8/3, mean 2
    assert abs(t["keff"] - 2.0) < 1e-15
    assert abs(t["length"] - 0.5) < 1e-15
    # beta = alpha * Hbar / Keff = 3 * 0.5 / 2
    assert abs(t["beta"] - 0.75) < 1e-15


@pytest.mark.parametrize("bc", BCS)
def test_interface_conditions_in_final_fields(bc):
    prob = inputs.darcy_problem(24, 16, sigma2=3.0, corr=0.2, seed=8, bc=bc,
                                sub=(8, 8), seg=(4, 4), alpha=2.0)
    m = solve_mrcm(prob)
    dec = m["dec"]
    scale = np.abs(m["Fx"]).max()
    for t in dec.segments:
        if t["axis"] == 0:
            fa = m["Fa_x"][t["lo"]:t["hi"], t["line"]]
            fb = m["Fb_x"][t["lo"]:t["hi"], t["line"]]
        else:
            fa = m["Fa_y"][t["line"], t["lo"]:t["hi"]]
            fb = m["Fb_y"][t["line"], t["lo"]:t["hi"]]
        # outward of a = +axis, outward of b = -axis
        Fa_out, Fb_out = fa.sum(), -fb.sum()
        assert abs(Fa_out + Fb_out) < 1e-12 * scale                           # Eq. (13.2)
        assert abs(Fa_out - Fb_out - 2 * m["U"][t["id"]] * t["length"]) < 1e-12 * scale  # Eq. (14.2)
    # cell-wise conservation inside every leaf with its own one-sided fluxes
    for lf in dec.leaves:
        j0, j1, i0, i1 = lf["j0"], lf["j1"], lf["i0"], lf["i1"]
        Fx = m["Fa_x"][j0:j1, i0:i1 + 1].copy()
        Fx[:, 0] = m["Fb_x"][j0:j1, i0]
        Fy = m["Fa_y"][j0:j1 + 1, i0:i1].copy()
        Fy[0, :] = m["Fb_y"][j0, i0:i1]
        div = Fx[:, 1:] - Fx[:, :-1] + Fy[1:, :] - Fy[:-1, :]
        assert np.abs(div - prob.q[j0:j1, i0:i1]).max() < 1e-12 * scale


def test_pure_neumann_pin_choice_does_not_matter():
    # O2 pins P of the first segment; the recursion pins the first segment
    # of the root interface.  After the zero-mean shift both agree.
    prob = inputs.darcy_problem(24, 24, sigma2=2.0, corr=0.2, seed=13, bc="quarter_five_spot",
                                sub=(8, 8), seg=(2, 2))
    m = solve_mrcm(prob)
    r = solve_recursive(prob, tie="y")
    assert rel(r["p"], m["p"]) < 1e-10
    assert abs(m["p"].mean()) < 1e-13 * np.abs(m["p"]).max()


def test_strip_decomposition_exact_for_linear_pressure():
    # interfaces perpendicular to a uniform flow: the exact linear pressure
    # and constant flux satisfy every local problem, so MRCM is exact
    prob = inputs.darcy_problem(24, 8, sigma2=0.0, bc="left_right", sub=(6, 8), seg=(4, 4), alpha=1.0)
    f, m = solve_fine(prob), solve_mrcm(prob)
    assert rel(m["p"], f["p"]) < 1e-13
    assert rel(m["Fx"], f["Fx"]) < 1e-13


def test_error_falls_with_alpha():
    # 2D decomposition, homogeneous K, 4-face segments, p=1 / p=0 left and
    # right: the fine solution is linear and flux-continuous, which the
    # flux-coupled (MHM) limit beta -> infinity reproduces (Section 2.1), so
    # the MRCM error decays like 1/alpha: about tenfold per decade.
    errs = []
    for alpha in (1e0, 1e1, 1e2, 1e3):
        prob = inputs.darcy_problem(32, 32, sigma2=0.0, bc="left_right",
                                    sub=(8, 8), seg=(4, 4), alpha=alpha)
        f, m = solve_fine(prob), solve_mrcm(prob)
        errs.append(rel(np.concatenate([m["Fx"].ravel(), m["Fy"].ravel()]),
                        np.concatenate([f["Fx"].ravel(), f["Fy"].ravel()])))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 5.0) and np.all(ratios < 20.0), errs


@pytest.mark.parametrize("bc", BCS)
def test_refinement_reaches_the_discrete_solution(bc):
    # Iterative refinement with double-double residuals of Eqs. 11.2-14.2:
    # the global system (O2) and the recursion (Algorithm 1) are different
    # FP64 solvers whose plain results differ at high contrast; refined, both
    # must give the same discrete solution to about one rounding unit, and
    # the residual must fall to the double-double level.
    prob = inputs.darcy_problem(96, 80, sigma2=4.0, corr=0.05, seed=77, bc=bc)
    m0, r0 = solve_mrcm(prob), solve_recursive(prob)
    m, r = solve_mrcm(prob, refine=3), solve_recursive(prob, refine=3)
    assert m["refine_history"][-1] < 1e-24 and r["refine_history"][-1] < 1e-24
    for key in ("p", "Fx", "Fy", "Fa_x", "Fb_y"):
        assert rel(m[key], r[key]) < 1e-14, key
        # the plain solves agree with the refined one only to their accuracy
        assert rel(m0[key], m[key]) < 1e-8


def test_refined_one_face_segments_equal_fine():
    prob = inputs.darcy_problem(24, 20, sigma2=3.0, corr=0.2, seed=4, bc="quarter_five_spot",
                                sub=(6, 5), seg=(1, 1), alpha=2.0)
    f, m = solve_fine(prob), solve_mrcm(prob, refine=2)
    for key in ("p", "Fx", "Fy"):
        assert rel(m[key], f[key]) < 1e-11


def test_node_segments_from_children_match_the_box_definition():
    # the recursion takes a node's outer segments from its children (their
    # segments minus gamma); they must be the segments with exactly one side
    # in the node's box, on a ragged grid with both split axes
    from oracle.recursive import outer_segments
    prob = inputs.darcy_problem(72, 52, sigma2=1.0, corr=0.2, seed=8, bc="left_right")
    rm = RecursiveMRCM(prob)
    stack, n = [rm.root], 0
    while stack:
        nd = stack.pop()
        stack += nd.children
        assert nd.segs == outer_segments(rm.dec, nd.box)
        n += 1
    assert n == 2 * len(rm.dec.leaves) - 1


def test_leaf_map_mode_gives_the_same_solution():
    # handing the per-leaf work to a map function (a process pool's at large
    # sizes) changes no arithmetic: the same refined solution
    from oracle.recursive import leaf_worker_init
    prob = inputs.darcy_problem(48, 40, sigma2=2.0, corr=0.1, seed=12, bc="quarter_five_spot")
    a = solve_recursive(prob, refine=2)
    leaf_worker_init(prob)
    b = solve_recursive(prob, refine=2, leaf_map=map)
    for k in ("p", "Fx", "Fy", "Fa_x", "Fb_y"):
        assert rel(b[k], a[k]) < 1e-13, k
