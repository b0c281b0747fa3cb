"""Blocked tree heights with at least as many nodes as SMs and 2g <= 128 are
inverted per node (one CTA per interface system, in shared memory) instead
of by the cooperative blocked sweep.

A batch of 320 problems of 64 x 64 cells with one-face segments puts 320
roots of 2g = 128 (inverted: below the automatic factor threshold) and 640
nodes of 2g = 64 at two heights.  Each problem must match the FP64 oracle
(rel-L2 <= 1e-10 in p, Fx, Fy after refinement), and the single-problem
contexts (one node per height: the sweep) to rounding of a single pass;
the mixed form (FP32 inversions per node) must refine to 1e-8.
"""
import numpy as np
import pytest

import inputs
from oracle.mrcm import solve_mrcm
from conftest import rel

pytestmark = pytest.mark.gpu
COUNT = 320
CHECK = (0, 1, 57, 158, 319)


def _probs():
    return [inputs.darcy_problem(64, 64, sigma2=1.0 + (k % 4) * 0.5, corr=0.1, seed=700 + k, bc="left_right",
                                 seg=(1, 1)) for k in range(COUNT)]


def _batch(mr, probs, refine, precision=0):
    import torch
    b = mr.BatchSolver([torch.from_numpy(p.K).cuda() for p in probs], [(p.Lx, p.Ly) for p in probs],
                       [p.bc_type for p in probs], sub=probs[0].sub, seg=probs[0].seg, alpha=probs[0].alpha,
                       precision=precision)
    mr.mrcm_set_refinement(b.ctx, refine)
    b.build_basis()
    b.solve([torch.from_numpy(p.q).cuda() for p in probs], [torch.from_numpy(p.bc_val).cuda() for p in probs])
    out = [tuple(t.cpu().numpy().copy() for t in r) for r in b.split()]
    return b, out


def test_node_levels_match_the_oracle_and_the_sweep(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    probs = _probs()
    assert mr.mrcm_plan_query((64, 64), (1.0, 1.0), (16, 16), (1, 1), probs[0].bc_type, "MAX_GAMMA") == 128
    b, out = _batch(mr, probs, refine=3)
    for k in CHECK:
        o = solve_mrcm(probs[k], refine=3)
        p, fx, fy = out[k]
        errs = (rel(p, o["p"]), rel(fx, o["Fx"]), rel(fy, o["Fy"]))
        assert max(errs) <= 1e-10, (k, errs)
    # single passes: the batch (per-node inversions) against one-problem
    # contexts (the blocked sweep), to rounding
    b1, out1 = _batch(mr, probs, refine=0)
    for k in CHECK:
        prob = probs[k]
        s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                      prob.bc_type)
        mr.mrcm_set_refinement(s.ctx, 0)
        s.build_basis()
        s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda())
        ref = (s.p.cpu().numpy(), s.Fx.cpu().numpy(), s.Fy.cpu().numpy())
        d = [rel(a.reshape(r.shape), r) for a, r in zip(out1[k], ref)]
        assert max(d) <= 1e-9, (k, d)
        s.close()


def test_node_levels_in_fp32_refine_to_the_oracle(mrcm_lib):
    import paper_2009_07965_gb300 as mr
    probs = _probs()
    b, out = _batch(mr, probs, refine=6, precision=mr.binding.MRCM_MIXED)
    for k in CHECK[:3]:
        o = solve_mrcm(probs[k], refine=3)
        p, fx, fy = out[k]
        errs = (rel(p, o["p"]), rel(fx, o["Fx"]), rel(fy, o["Fy"]))
        assert max(errs) <= 1e-8, (k, errs)
