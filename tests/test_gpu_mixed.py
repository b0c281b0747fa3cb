"""The mixed-precision form (MRCM_MIXED) against the FP64 oracle.

Leaf factorisations, multi-right-hand-side basis solves and the merges of
interface systems up to 2g = 512 run in FP32, the rest in FP64; the solve
refines with double-double residuals of Eqs. 11.2-14.2.  Target: rel-L2
<= 1e-8 in p, Fx, Fy and the one-sided skeleton fluxes against the
refined oracle, stated per result; the same with every merge in FP32; the
residual history must fall step by step.
"""
import numpy as np
import pytest

import inputs
from oracle.mrcm import solve_mrcm
from conftest import rel

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-8
KEYS = ("p", "Fx", "Fy", "Fa_x", "Fb_x", "Fa_y", "Fb_y")


def _mixed_solve(prob, split=None, refine=None, stream=None, leaves32=None, residual_dd=None):
    import torch
    import paper_2009_07965_gb300 as mr
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                  prob.bc_type, stream=stream, precision=mr.binding.MRCM_MIXED)
    if split is not None:
        mr.mrcm_set_mixed_split(s.ctx, split)
    if leaves32 is not None:
        mr.mrcm_set_mixed_leaves(s.ctx, leaves32)
    if residual_dd is not None:
        mr.mrcm_set_residual(s.ctx, residual_dd)
    if refine is not None:
        mr.mrcm_set_refinement(s.ctx, refine, check=True)
    else:
        mr.mrcm_set_refinement(s.ctx, 3, check=True)
    s.build_basis()
    s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda(), want_iface=True)
    fa_x, fb_x, fa_y, fb_y = s.iface_parts()
    out = dict(p=s.p, Fx=s.Fx, Fy=s.Fy, Fa_x=fa_x, Fb_x=fb_x, Fa_y=fa_y, Fb_y=fb_y)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    out["history"] = mr.mrcm_residual_history(s.ctx)
    s.close()
    return out


def _check(g, o, tol=TOL_MIXED):
    errs = {k: rel(g[k], o[k]) for k in KEYS}
    print("mixed rel errors", errs, "residuals", g["history"])
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, errs
    h = g["history"]
    assert h[-1] < h[0], h
    return errs


@pytest.mark.parametrize("bc", ["left_right", "quarter_five_spot"])
def test_mixed_ragged_leaves(mrcm_lib, bc):
    prob = inputs.darcy_problem(72, 60, sigma2=2.0, corr=0.15, seed=31, bc=bc)
    _check(_mixed_solve(prob), solve_mrcm(prob, refine=3))


def test_mixed_high_contrast_with_blocked_levels(mrcm_lib):
    # sigma^2 = 4 (contrast ~1e7): FP32 leaves and FP32 blocked sweeps
    # (2g up to 256 at 512^2), refined back to the FP64 solution
    prob = inputs.darcy_problem(512, 512, sigma2=4.0, corr=0.05, seed=2000, bc="quarter_five_spot")
    o = solve_mrcm(prob, refine=3)
    _check(_mixed_solve(prob), o)
    # FP32 leaves as well: every merge in FP32, and the top merges in FP64
    _check(_mixed_solve(prob, leaves32=1), o)
    _check(_mixed_solve(prob, leaves32=1, split=512), o)
    _check(_mixed_solve(prob, leaves32=1, split=64), o)


def test_mixed_rectangular_leaves_alpha(mrcm_lib):
    prob = inputs.darcy_problem(50, 30, sigma2=1.5, corr=0.1, seed=5, bc="left_right",
                                sub=(8, 16), seg=(2, 4), alpha=0.3, Lx=2.0, Ly=0.7)
    _check(_mixed_solve(prob), solve_mrcm(prob, refine=3))


def test_mixed_leaf_maps_are_fp32_accurate(mrcm_lib):
    # the leaf maps of the mixed form are FP32 approximations of the FP64
    # maps (not the same numbers, not garbage)
    import torch
    import paper_2009_07965_gb300 as mr
    prob = inputs.config_64()
    s64 = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                    prob.bc_type)
    s32 = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                    prob.bc_type, precision=mr.binding.MRCM_MIXED)
    mr.mrcm_set_mixed_leaves(s32.ctx, 1)
    s64.build_basis()
    s32.build_basis()
    for leaf in range(mr.mrcm_query(s64.ctx, "LEAVES")):
        a = mr.mrcm_node_operator(s64.ctx, leaf)
        b = mr.mrcm_node_operator(s32.ctx, leaf)
        e = rel(b, a)
        assert 0.0 < e < 1e-4, (leaf, e)
    s64.close()
    s32.close()


def test_mixed_with_fp64_leaves(mrcm_lib):
    """FP64 leaf factors (the default), FP32 merges up to a split and all of
    them: refined to the FP64 oracle; the leaf maps equal the FP64 form's."""
    import torch
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(512, 512, sigma2=4.0, corr=0.05, seed=2000, bc="quarter_five_spot")
    o = solve_mrcm(prob, refine=3)
    _check(_mixed_solve(prob, leaves32=0, split=512), o)
    _check(_mixed_solve(prob, leaves32=0), o)
    # double-double residuals instead of the form's FP64 ones
    _check(_mixed_solve(prob, leaves32=0, residual_dd=1), o)
    small = inputs.config_64()
    s64 = mr.Solver(torch.from_numpy(small.K).cuda(), small.Lx, small.Ly, small.sub, small.seg, small.alpha,
                    small.bc_type)
    sm = mr.Solver(torch.from_numpy(small.K).cuda(), small.Lx, small.Ly, small.sub, small.seg, small.alpha,
                   small.bc_type, precision=mr.binding.MRCM_MIXED)
    mr.mrcm_set_mixed_leaves(sm.ctx, 0)
    s64.build_basis()
    sm.build_basis()
    for leaf in range(mr.mrcm_query(s64.ctx, "LEAVES")):
        assert np.array_equal(mr.mrcm_node_operator(s64.ctx, leaf), mr.mrcm_node_operator(sm.ctx, leaf))
    with pytest.raises(mr.MrcmError) as e:
        mr.mrcm_set_mixed_leaves(s64.ctx, 0)               # not a mixed context
    assert e.value.code == -9
    s64.close()
    sm.close()
