"""3D parity: the CUDA path (blocks of the patch shape merged into 16^3
subdomains by fine-face Robin couplings, subdomains coupled by patches)
against the 3D oracle (direct local solves of each subdomain and the global
interface system), FP64, rel-L2 <= 1e-10 in p, Fx, Fy, Fz.

At the full 256 x 256 x 64 size, where the oracle would take too long, the
test checks what holds at any size: the net inflow equals the net outflow,
every subdomain is balanced (the patch-integrated fluxes of its two sides
agree, Eq. 13.2), and every cell away from the subdomain boundaries is
conservative (its faces are exact fine-face couplings)."""
import numpy as np
import pytest

import inputs
from conftest import rel

pytestmark = pytest.mark.gpu


def _solve(prob, torch, precision=None, split=None, refine=None):
    from paper_2009_07965_gb300 import Solver3D, mrcm_set_mixed_split, mrcm_set_refinement
    import paper_2009_07965_gb300.binding as B
    dev = torch.device("cuda:0")
    K = torch.from_numpy(prob.K).to(dev)
    s = Solver3D(K, L=(prob.Lx, prob.Ly, prob.Lz), sub=prob.sub, seg=prob.seg, alpha=prob.alpha,
                 bc_type=prob.bc_type, precision=B.MRCM_FP64 if precision is None else precision)
    if split is not None:
        mrcm_set_mixed_split(s.ctx, split)
    if refine is not None:
        mrcm_set_refinement(s.ctx, refine, 0)
    s.build_basis()
    q = torch.from_numpy(prob.q).to(dev)
    g = torch.from_numpy(prob.bc_val).to(dev)
    p, Fx, Fy, Fz = s.solve(q, g)
    torch.cuda.synchronize()
    out = dict(p=p.cpu().numpy(), Fx=Fx.cpu().numpy(), Fy=Fy.cpu().numpy(), Fz=Fz.cpu().numpy())
    from paper_2009_07965_gb300 import mrcm_residual_history
    out["hist"] = mrcm_residual_history(s.ctx)
    s.close()
    return out


CASES = [
    # (n, sub, seg, L, sigma2, corr, seed, alpha)
    ((32, 32, 16), (16, 16, 16), (4, 4, 4), None, 2.0, (0.2, 0.2, 0.05), 1, 1.0),
    ((16, 24, 16), (8, 8, 8), (4, 4, 2), None, 2.0, (0.3, 0.3, 0.1), 2, 1.0),
    ((24, 16, 12), (8, 8, 4), (2, 4, 2), (1.0, 0.5, 0.25), 3.0, (0.2, 0.2, 0.2), 3, 3.0),
    ((16, 16, 16), (4, 4, 4), (4, 4, 4), None, 2.0, (0.3, 0.3, 0.3), 4, 0.5),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + "-seg" + "".join(map(str, c[2])))
def test_3d_matches_the_oracle(case, mrcm_lib):
    import torch
    from oracle.mrcm3d import solve_mrcm3d
    n, sub, seg, L, s2, corr, seed, alpha = case
    prob = inputs.darcy_problem_3d(*n, sigma2=s2, corr=corr, seed=seed, bc="left_right", sub=sub,
                                   seg=seg, alpha=alpha, L=L)
    g, o = _solve(prob, torch), solve_mrcm3d(prob)
    for key in ("p", "Fx", "Fy", "Fz"):
        assert rel(g[key], o[key]) < 1e-10, (key, rel(g[key], o[key]))


def test_3d_one_face_patches_equal_the_fine_solution(mrcm_lib):
    # single-cell blocks and one-face patches: every coupling is exact
    import torch
    from oracle.mrcm3d import solve_fine3d
    prob = inputs.darcy_problem_3d(12, 8, 8, sigma2=2.0, corr=(0.3, 0.3, 0.3), seed=6, bc="left_right",
                                   sub=(2, 2, 2), seg=(1, 1, 1), alpha=1.0)
    g, f = _solve(prob, torch), solve_fine3d(prob)
    for key in ("p", "Fx", "Fy", "Fz"):
        assert rel(g[key], f[key]) < 1e-10, key


def test_3d_box_workload_conservation(mrcm_lib):
    # the 256 x 256 x 64 workload of the benchmark, on its own inputs
    import torch
    prob = inputs.config_3d()
    g = _solve(prob, torch)
    Fx, Fy, Fz, q = g["Fx"], g["Fy"], g["Fz"], prob.q
    inflow, outflow = Fx[:, :, 0].sum(), Fx[:, :, -1].sum()
    assert inflow > 0 and abs(inflow - outflow) < 1e-10 * inflow
    assert np.abs(Fy[:, 0, :]).max() == 0 and np.abs(Fz[0]).max() == 0
    s = 16
    div = np.diff(Fx, axis=2) + np.diff(Fy, axis=1) + np.diff(Fz, axis=0) - q
    scale = np.abs(Fx).max()
    # cells with no face on a subdomain boundary
    inner = np.zeros(q.shape, dtype=bool)
    idx = [np.arange(m) % s for m in q.shape]
    kk, jj, ii = np.meshgrid(*idx, indexing="ij")
    inner = (ii > 0) & (ii < s - 1) & (jj > 0) & (jj < s - 1) & (kk > 0) & (kk < s - 1)
    assert np.abs(div[inner]).max() < 1e-10 * scale
    # every subdomain: net outflow = its source (zero)
    nz, ny, nx = q.shape
    for k0 in range(0, nz, s):
        for j0 in range(0, ny, s):
            for i0 in range(0, nx, s):
                net = (Fx[k0:k0 + s, j0:j0 + s, i0 + s].sum() - Fx[k0:k0 + s, j0:j0 + s, i0].sum()
                       + Fy[k0:k0 + s, j0 + s, i0:i0 + s].sum() - Fy[k0:k0 + s, j0, i0:i0 + s].sum()
                       + Fz[k0 + s, j0:j0 + s, i0:i0 + s].sum() - Fz[k0, j0:j0 + s, i0:i0 + s].sum())
                assert abs(net) < 1e-10 * inflow


def test_3d_settings_it_lacks_are_refused(mrcm_lib):
    # double-double residuals and FP32 block factors are 2D-only
    import torch
    from paper_2009_07965_gb300 import Solver3D, MrcmError, mrcm_set_residual, mrcm_set_mixed_leaves
    import paper_2009_07965_gb300.binding as B
    prob = inputs.darcy_problem_3d(16, 16, 16, sigma2=1.0, seed=1, sub=(8, 8, 8), seg=(4, 4, 4))
    s = Solver3D(torch.from_numpy(prob.K).cuda(), sub=prob.sub, seg=prob.seg, precision=B.MRCM_MIXED)
    with pytest.raises(MrcmError) as e:
        mrcm_set_residual(s.ctx, 1)
    assert e.value.code == -9
    with pytest.raises(MrcmError) as e:
        mrcm_set_mixed_leaves(s.ctx, 1)
    assert e.value.code == -9
    s.close()


MIXED = [CASES[0], CASES[1], CASES[2]]


@pytest.mark.parametrize("split", [1 << 30, 64])
@pytest.mark.parametrize("case", MIXED, ids=lambda c: "x".join(map(str, c[0])) + "-seg" + "".join(map(str, c[2])))
def test_3d_mixed_form_matches_the_oracle(case, split, mrcm_lib):
    # FP32 merges (all of them, or those up to 2g = 64), FP64 blocks, the
    # default two refinement steps with FP64 residuals: rel-L2 <= 1e-8
    import torch
    from oracle.mrcm3d import solve_mrcm3d
    import paper_2009_07965_gb300.binding as B
    n, sub, seg, L, s2, corr, seed, alpha = case
    prob = inputs.darcy_problem_3d(*n, sigma2=s2, corr=corr, seed=seed, bc="left_right", sub=sub,
                                   seg=seg, alpha=alpha, L=L)
    g = _solve(prob, torch, precision=B.MRCM_MIXED, split=split)
    o = solve_mrcm3d(prob)
    for key in ("p", "Fx", "Fy", "Fz"):
        assert rel(g[key], o[key]) < 1e-8, (key, rel(g[key], o[key]))
    hist = g["hist"]
    assert len(hist) == 2 and hist[-1] < 1e-2 * hist[0]


def test_3d_fp64_refinement_keeps_the_solution(mrcm_lib):
    # refining the FP64 form changes the single pass only at its rounding
    # level
    import torch
    from oracle.mrcm3d import solve_mrcm3d
    n, sub, seg, L, s2, corr, seed, alpha = CASES[0]
    prob = inputs.darcy_problem_3d(*n, sigma2=s2, corr=corr, seed=seed, bc="left_right", sub=sub,
                                   seg=seg, alpha=alpha, L=L)
    a, b = _solve(prob, torch), _solve(prob, torch, refine=2)
    o = solve_mrcm3d(prob)
    for key in ("p", "Fx", "Fy", "Fz"):
        assert rel(b[key], a[key]) < 1e-11, key
        assert rel(b[key], o[key]) < 1e-10, key


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_3d_every_side_and_source_against_the_oracle(precision, mrcm_lib):
    # Dirichlet on x-, y+ and z+, nonzero Neumann fluxes on x+, y- and z-, a
    # random source: every side's boundary-value block is read at its own
    # face positions (a transposed or shifted index fails here)
    import torch
    from oracle.mrcm3d import solve_mrcm3d
    import paper_2009_07965_gb300.binding as B
    from inputs.problems import DIRICHLET, NEUMANN
    prob = inputs.darcy_problem_3d(16, 12, 20, sigma2=2.0, corr=(0.3, 0.2, 0.2), seed=9, bc="left_right",
                                   sub=(8, 4, 4), seg=(4, 2, 2), alpha=1.5, L=(1.0, 0.5, 1.0))
    prob.bc_type = (DIRICHLET, NEUMANN, NEUMANN, DIRICHLET, NEUMANN, DIRICHLET)
    rng = np.random.default_rng(17)
    prob.bc_val = rng.uniform(-1.0, 1.0, prob.bc_val.shape)
    prob.q = rng.uniform(-0.01, 0.01, prob.q.shape)
    prec = B.MRCM_FP64 if precision == "fp64" else B.MRCM_MIXED
    g, o = _solve(prob, torch, precision=prec), solve_mrcm3d(prob)
    tol = 1e-10 if precision == "fp64" else 1e-8
    for key in ("p", "Fx", "Fy", "Fz"):
        assert rel(g[key], o[key]) < tol, (key, rel(g[key], o[key]))


def test_3d_single_leaf_nested_dissection_is_the_fine_solution(mrcm_lib):
    # one 16^3 leaf and no patches: the merges of its 64 blocks over one-face
    # segments must give the fine two-point-flux solution itself
    import torch
    from oracle.mrcm3d import solve_fine3d
    prob = inputs.darcy_problem_3d(16, 16, 16, sigma2=3.0, corr=(0.2, 0.2, 0.1), seed=21, bc="left_right",
                                   sub=(16, 16, 16), seg=(4, 4, 4), alpha=1.0)
    g, f = _solve(prob, torch), solve_fine3d(prob)
    for key in ("p", "Fx", "Fy", "Fz"):
        assert rel(g[key], f[key]) < 1e-10, (key, rel(g[key], f[key]))


def test_3d_one_sided_fluxes_against_the_oracle(mrcm_lib):
    # both one-sided skeleton fluxes (side a the lower block), FP64
    import torch
    from oracle.mrcm3d import solve_mrcm3d
    from paper_2009_07965_gb300 import Solver3D
    n, sub, seg, L, s2, corr, seed, alpha = CASES[1]
    prob = inputs.darcy_problem_3d(*n, sigma2=s2, corr=corr, seed=seed, bc="left_right", sub=sub,
                                   seg=seg, alpha=alpha, L=L)
    dev = torch.device("cuda:0")
    s = Solver3D(torch.from_numpy(prob.K).to(dev), L=(prob.Lx, prob.Ly, prob.Lz), sub=prob.sub, seg=prob.seg,
                 alpha=prob.alpha, bc_type=prob.bc_type)
    s.build_basis()
    s.solve(torch.from_numpy(prob.q).to(dev), torch.from_numpy(prob.bc_val).to(dev), want_iface=True)
    torch.cuda.synchronize()
    parts = [t.cpu().numpy() for t in s.iface_parts()]
    o = solve_mrcm3d(prob)
    for name, g in zip(("Fa_x", "Fb_x", "Fa_y", "Fb_y", "Fa_z", "Fb_z"), parts):
        assert rel(g, o[name]) < 1e-10, (name, rel(g, o[name]))
    s.close()


@pytest.mark.parametrize("case,precision", [(CASES[0], "fp64"), (CASES[2], "fp64"), (CASES[1], "mixed")],
                         ids=["32x32x16-fp64", "24x16x12-fp64", "16x24x16-mixed"])
def test_3d_all_neumann_quarter_five_spot(case, precision, mrcm_lib):
    # no-flow on every side, +1 / -1 in opposite corner cells: the pinned
    # root, the data check and the zero-mean shift in 3D
    import torch
    from oracle.mrcm3d import solve_mrcm3d
    import paper_2009_07965_gb300.binding as B
    n, sub, seg, L, s2, corr, seed, alpha = case
    prob = inputs.darcy_problem_3d(*n, sigma2=s2, corr=corr, seed=seed, bc="quarter_five_spot", sub=sub,
                                   seg=seg, alpha=alpha, L=L)
    prec = B.MRCM_FP64 if precision == "fp64" else B.MRCM_MIXED
    g, o = _solve(prob, torch, precision=prec), solve_mrcm3d(prob)
    tol = 1e-10 if precision == "fp64" else 1e-8
    assert abs(g["p"].mean()) < 1e-12 * np.abs(g["p"]).max()
    for key in ("p", "Fx", "Fy", "Fz"):
        assert rel(g[key], o[key]) < tol, (key, rel(g[key], o[key]))


def test_3d_incompatible_neumann_data_is_refused(mrcm_lib):
    import torch
    from paper_2009_07965_gb300 import Solver3D, MrcmError
    prob = inputs.darcy_problem_3d(16, 16, 16, sigma2=1.0, seed=3, bc="quarter_five_spot", sub=(8, 8, 8),
                                   seg=(4, 4, 4))
    dev = torch.device("cuda:0")
    s = Solver3D(torch.from_numpy(prob.K).to(dev), sub=prob.sub, seg=prob.seg, bc_type=prob.bc_type)
    s.build_basis()
    q = prob.q.copy()
    q[0, 0, 0] = 2.0                      # sources no longer balance the (zero) boundary flux
    with pytest.raises(MrcmError) as e:
        s.solve(torch.from_numpy(q).to(dev), torch.from_numpy(prob.bc_val).to(dev))
    assert e.value.code == -1
    s.close()
