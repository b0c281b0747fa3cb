"""Failure handling of the CUDA path, made without faulting the GPU.

- MRCM_ERR_TIMEOUT: the bounded inter-CTA waits of the cooperative launches
  (blocked interface sweep, solve tree sweeps) are given a limit of zero
  polls, so that they run out; the call must return MRCM_ERR_TIMEOUT and the
  context must give the normal results once the default limit is back.
- MRCM_ERR_INVALID_ARG for all-Neumann data whose sources do not balance
  the boundary outflow (no solution exists, Section 2), while balanced data
  solve normally on the same context.
"""
import numpy as np
import pytest

import inputs
from conftest import rel

pytestmark = pytest.mark.gpu


def _solver(prob, stream=None):
    import torch
    import paper_2009_07965_gb300 as mr
    return mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                     prob.bc_type, stream=stream)


@pytest.mark.parametrize("graphs", [False, True])
def test_bounded_waits_time_out_and_the_context_recovers(mrcm_lib, graphs):
    import torch
    import paper_2009_07965_gb300 as mr
    from paper_2009_07965_gb300 import MrcmError
    # 256^2: blocked interface systems (2g up to 128) run in the cooperative
    # sweep, and the solve's tree sweeps wait between heights
    prob = inputs.darcy_problem(256, 256, sigma2=2.0, corr=0.1, seed=61, bc="quarter_five_spot")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = _solver(prob, stream=st)
        mr.mrcm_use_graphs(s.ctx, graphs)
        q, bc = torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda()
        s.build_basis()
        s.solve(q, bc)
        ref = [t.cpu().numpy().copy() for t in (s.p, s.Fx, s.Fy)]
        # limit 0: a wait gives up at its first unmet check, so every CTA
        # of a launch but the last to arrive at a grid barrier gives up
        mr.mrcm_set_wait_limit(s.ctx, 0)
        with pytest.raises(MrcmError) as e:
            s.build_basis()
        assert e.value.code == -8                    # MRCM_ERR_TIMEOUT
        mr.mrcm_set_wait_limit(s.ctx, -1)            # default limit
        s.build_basis()                              # everything recomputed
        mr.mrcm_set_wait_limit(s.ctx, 0)
        with pytest.raises(MrcmError) as e:
            s.solve(q, bc)
        assert e.value.code == -8
        mr.mrcm_set_wait_limit(s.ctx, -1)
        s.solve(q, bc)
        out = [t.cpu().numpy() for t in (s.p, s.Fx, s.Fy)]
        st.synchronize()
        s.close()
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)


def test_inconsistent_neumann_data_are_rejected(mrcm_lib):
    import torch
    from paper_2009_07965_gb300 import MrcmError
    prob = inputs.darcy_problem(96, 80, sigma2=1.0, corr=0.2, seed=5, bc="quarter_five_spot")
    s = _solver(prob)
    s.build_basis()
    bc = torch.from_numpy(prob.bc_val).cuda()
    q = prob.q.copy()
    q[40, 50] = 1e-9                                 # sum q = 1e-9 = 5e-10 sum |q|
    with pytest.raises(MrcmError) as e:
        s.solve(torch.from_numpy(q).cuda(), bc)
    assert e.value.code == -1
    # balanced again by a boundary outflow of the same amount on the y+ side
    g = prob.bc_val.copy()
    g[2 * prob.ny + prob.nx + 7] = 1e-9 / prob.hx
    s.solve(torch.from_numpy(q).cuda(), torch.from_numpy(g).cuda())
    # and the original data still solve (the context stays usable)
    s.solve(torch.from_numpy(prob.q).cuda(), bc)
    assert np.isfinite(s.p.cpu().numpy()).all()
    s.close()
