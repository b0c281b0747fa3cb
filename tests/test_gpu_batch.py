"""Batched ensembles (mrcm_setup_batch): several independent problems of
different sizes in one context, built and solved together (one launch per
tree height over every problem's tree).

Each problem's result must match the FP64 oracle's solution of that problem
alone (rel-L2 <= 1e-10 in p, Fx, Fy and the one-sided skeleton fluxes), and
the single-problem contexts of the CUDA path to rounding.  The problems have
different cell counts per side (truncated leaves at their own right and top
edges), different cell sizes, both split axes, a problem of a single leaf,
and both boundary-condition families allowed in a batch.
"""
import numpy as np
import pytest

import inputs
from oracle.mrcm import solve_mrcm
from conftest import rel

pytestmark = pytest.mark.gpu
TOL = 1e-10
KEYS = ("p", "Fx", "Fy", "Fa_x", "Fb_x", "Fa_y", "Fb_y")


def _problems():
    probs = [inputs.ensemble_member(r, nmin=20, nmax=90) for r in range(5)]
    probs.append(inputs.darcy_problem(12, 10, sigma2=1.0, corr=0.3, seed=3, bc="left_right"))   # one leaf
    probs.append(inputs.darcy_problem(50, 30, sigma2=2.0, corr=0.1, seed=5, bc="left_right", Lx=2.0, Ly=0.7,
                                      alpha=1.0))
    return probs


def _batch_solve(mr, probs, refine=3, stream=None):
    import torch
    Ks = [torch.from_numpy(p.K).cuda() for p in probs]
    b = mr.BatchSolver(Ks, [(p.Lx, p.Ly) for p in probs], [p.bc_type for p in probs], stream=stream)
    mr.mrcm_set_refinement(b.ctx, refine)
    b.build_basis()
    b.solve([torch.from_numpy(p.q).cuda() for p in probs], [torch.from_numpy(p.bc_val).cuda() for p in probs],
            want_iface=True)
    outs = []
    for (pp, fx, fy), (fa_x, fb_x, fa_y, fb_y) in zip(b.split(), b.iface_split()):
        outs.append({k: t.cpu().numpy().copy() for k, t in
                     zip(KEYS, (pp, fx, fy, fa_x, fb_x, fa_y, fb_y))})
    return b, outs


def test_batch_matches_the_oracle_per_problem(mrcm_lib):
    import paper_2009_07965_gb300 as mr
    probs = _problems()
    b, outs = _batch_solve(mr, probs)
    assert mr.mrcm_query(b.ctx, "GRIDS") == len(probs)
    assert mr.mrcm_query(b.ctx, "CELLS") == sum(p.nx * p.ny for p in probs)
    b.close()
    for prob, g in zip(probs, outs):
        o = solve_mrcm(prob, refine=3)
        errs = {k: rel(g[k], o[k]) for k in KEYS}
        assert all(e <= TOL for e in errs.values()), (prob.name, errs)


def test_batch_matches_single_problem_contexts(mrcm_lib):
    # the same per-problem arithmetic as a context of its own, up to the
    # summation order of the tree sweeps (their work split depends on the
    # level's composition)
    import paper_2009_07965_gb300 as mr
    from conftest import gpu_solve
    probs = _problems()
    b, outs = _batch_solve(mr, probs, refine=0)
    b.close()
    for prob, g in zip(probs, outs):
        s = gpu_solve(prob, refine=0)
        for k in KEYS:
            assert rel(g[k], s[k]) < 1e-13, (prob.name, k, rel(g[k], s[k]))
        s["solver"].close()


def test_batch_graph_replay_is_bitwise_repeatable(mrcm_lib):
    import paper_2009_07965_gb300 as mr
    import torch
    probs = _problems()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b, first = _batch_solve(mr, probs, refine=1, stream=st)
        qs = [torch.from_numpy(p.q).cuda() for p in probs]
        bcs = [torch.from_numpy(p.bc_val).cuda() for p in probs]
        for _ in range(2):
            b.build_basis()
            b.solve(qs, bcs, want_iface=True)
        again = [{k: t.cpu().numpy() for k, t in zip(("p", "Fx", "Fy"), o)} for o in b.split()]
        assert mr.mrcm_query(b.ctx, "GRAPH_REPLAYS") >= 2
        st.synchronize()
        b.close()
    for a, c in zip(first, again):
        for k in ("p", "Fx", "Fy"):
            assert np.array_equal(a[k], c[k])


def test_batch_refuses_all_neumann_members(mrcm_lib):
    import paper_2009_07965_gb300 as mr
    import torch
    probs = [inputs.darcy_problem(32, 32, sigma2=1.0, seed=1, bc="left_right"),
             inputs.darcy_problem(32, 32, sigma2=1.0, seed=2, bc="quarter_five_spot")]
    with pytest.raises(mr.MrcmError) as e:
        mr.BatchSolver([torch.from_numpy(p.K).cuda() for p in probs], [(1.0, 1.0)] * 2,
                       [p.bc_type for p in probs])
    assert e.value.code == -9
