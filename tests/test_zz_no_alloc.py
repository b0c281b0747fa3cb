"""The allocation-free merge entry point agrees with the regular build.

mrcm_merge_pair_noalloc serves callers that cannot allocate device memory
where they merge (for example code running inside another framework's
execution step, whose framework owns the device memory).  It keeps its LU
workspace in a fixed device array inside the library.  This test merges the
children of two tree nodes with it, twice in a row, and compares each merged
map with the one mrcm_build_basis produced for that node.  The file sorts
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import inputs
from conftest import rel

pytestmark = pytest.mark.gpu


def _inputs_for_node(mr, ctx, prob, node):
    """Children maps, index map and D of one node, from the regular build."""
    import torch
    info = mr.mrcm_node_info(ctx, node)
    c1, c2 = info["c1"], info["c2"]
    s1 = mr.mrcm_node_segments(ctx, c1)
    s2 = mr.mrcm_node_segments(ctx, c2)
    pos2 = {t: k for k, t in enumerate(s2)}
    gamma = [t for t in s1 if t in pos2]
    gpos1 = [k for k, t in enumerate(s1) if t in pos2]
    gpos2 = [pos2[t] for t in gamma]
    opos1 = [k for k, t in enumerate(s1) if t not in pos2]
    gset = set(gamma)
    opos2 = [k for k, t in enumerate(s2) if t not in gset]
    # D_t = |t| / (2 beta_t) = Keff_t / (2 alpha), Keff the mean harmonic
    # permeability of the segment's faces
    D = []
    for t in gamma:
        si = mr.mrcm_segment_info(ctx, t)
        hm = []
        for e in range(si["len"]):
            if si["axis"] == 0:
                ka, kb = prob.K[si["lo"] + e, si["line"] - 1], prob.K[si["lo"] + e, si["line"]]
            else:
                ka, kb = prob.K[si["line"] - 1, si["lo"] + e], prob.K[si["line"], si["lo"] + e]
            hm.append(2.0 * ka * kb / (ka + kb))
        keff = sum(hm) / len(hm)
        D.append(keff / (2.0 * prob.alpha))
    dev = torch.device("cuda:0")
    R1 = torch.from_numpy(mr.mrcm_node_operator(ctx, c1)).to(dev)
    R2 = torch.from_numpy(mr.mrcm_node_operator(ctx, c2)).to(dev)
    index_map = torch.tensor(gpos1 + gpos2 + opos1 + opos2, dtype=torch.int32, device=dev)
    Dt = torch.tensor(D, dtype=torch.float64, device=dev)
    return R1, len(s1), R2, len(s2), index_map, len(gamma), Dt


def test_noalloc_merge_matches_build(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(64, 48, sigma2=2.0, corr=0.1, seed=23, bc="left_right")
    dev = torch.device("cuda:0")
    s = mr.Solver(torch.from_numpy(prob.K).to(dev), prob.Lx, prob.Ly, prob.sub, prob.seg,
                  prob.alpha, prob.bc_type)
    s.build_basis()
    torch.cuda.synchronize()
    ctx = s.ctx
    nodes = [v for v in range(mr.mrcm_query(ctx, "NODES"))
             if mr.mrcm_node_info(ctx, v)["height"] >= 1 and mr.mrcm_node_info(ctx, v)["parent"] >= 0]
    # a low merge and the largest non-root merge
    picks = [nodes[0], max(nodes, key=lambda v: mr.mrcm_node_info(ctx, v)["g"])]
    for node in picks + picks:          # two calls in a row per node, interleaved
        R1, m1, R2, m2, index_map, g, Dt = _inputs_for_node(mr, ctx, prob, node)
        m = m1 + m2 - 2 * g
        R_out = torch.full((m, m), float("nan"), dtype=torch.float64, device=dev)
        X_out = torch.full((2 * g, m), float("nan"), dtype=torch.float64, device=dev)
        mr.mrcm_merge_pair_noalloc(R1, m1, R2, m2, index_map, g, Dt, R_out, X_out,
                                   torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        R_ref = mr.mrcm_node_operator(ctx, node)
        assert rel(R_out.cpu().numpy(), R_ref) < 1e-12, (node, rel(R_out.cpu().numpy(), R_ref))
        # X (2g x m, row-major) against -M^-1 C formed on the host from the
        # same children maps, index map and D
        X_ref = _host_X(R1.cpu().numpy(), R2.cpu().numpy(), index_map.cpu().numpy(), g, Dt.cpu().numpy())
        assert rel(X_out.cpu().numpy(), X_ref) < 1e-12, (node, rel(X_out.cpu().numpy(), X_ref))
    s.close()


def _host_X(R1, R2, index_map, g, D):
    m1, m2 = R1.shape[0], R2.shape[0]
    o1 = m1 - g
    gpos1, gpos2 = index_map[:g], index_map[g:2 * g]
    opos1, opos2 = index_map[2 * g:2 * g + o1], index_map[2 * g + o1:]
    M = np.block([[R1[np.ix_(gpos1, gpos1)] + np.diag(D), -np.diag(D)],
                  [-np.diag(D), R2[np.ix_(gpos2, gpos2)] + np.diag(D)]])
    C = np.zeros((2 * g, len(opos1) + len(opos2)))
    C[:g, :o1] = R1[np.ix_(gpos1, opos1)]
    C[g:, o1:] = R2[np.ix_(gpos2, opos2)]
    return -np.linalg.solve(M, C)


def test_noalloc_reports_a_singular_interface_system(mrcm_lib):
    # zero children maps on gamma and D = 0 make the interface matrix zero:
    # the call must report MRCM_ERR_SINGULAR (on a host-made input; the
    # kernel only divides by the zero pivots, which faults nothing)
    import torch
    import paper_2009_07965_gb300 as mr
    from paper_2009_07965_gb300 import MrcmError
    dev = torch.device("cuda:0")
    g = 2
    R = torch.zeros(4, 4, dtype=torch.float64, device=dev)
    idx = torch.tensor([0, 1, 0, 1, 2, 3, 2, 3], dtype=torch.int32, device=dev)
    D = torch.zeros(g, dtype=torch.float64, device=dev)
    Ro = torch.zeros(4, 4, dtype=torch.float64, device=dev)
    Xo = torch.zeros(4, 4, dtype=torch.float64, device=dev)
    with pytest.raises(MrcmError) as e:
        mr.mrcm_merge_pair_noalloc(R, 4, R, 4, idx, g, D, Ro, Xo)
    assert e.value.code == -5
    # the shared array keeps no state that spoils the next call
    R1 = -torch.eye(4, dtype=torch.float64, device=dev)
    mr.mrcm_merge_pair_noalloc(R1, 4, R1, 4, idx, g, torch.ones(g, dtype=torch.float64, device=dev), Ro, Xo)


def test_noalloc_rejects_oversized_and_bad_maps(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    from paper_2009_07965_gb300 import MrcmError
    dev = torch.device("cuda:0")
    g = 129                            # 2g = 258 > MRCM_NOALLOC_MAX_G2
    R = torch.zeros(300, 300, dtype=torch.float64, device=dev)
    idx = torch.zeros(2 * g + 2 * (300 - g), dtype=torch.int32, device=dev)
    D = torch.ones(g, dtype=torch.float64, device=dev)
    out = torch.zeros(400, 400, dtype=torch.float64, device=dev)
    with pytest.raises(MrcmError) as e:
        mr.mrcm_merge_pair_noalloc(R, 300, R, 300, idx, g, D, out, out)
    assert e.value.code == -1
    # an index outside child 1's map is refused on the device
    g = 2
    R1 = torch.eye(4, dtype=torch.float64, device=dev)
    bad = torch.tensor([0, 1, 0, 1, 2, 7, 2, 3], dtype=torch.int32, device=dev)
    D = torch.ones(g, dtype=torch.float64, device=dev)
    Ro = torch.zeros(4, 4, dtype=torch.float64, device=dev)
    Xo = torch.zeros(4, 4, dtype=torch.float64, device=dev)
    with pytest.raises(MrcmError) as e:
        mr.mrcm_merge_pair_noalloc(R1, 4, R1, 4, bad, g, D, Ro, Xo)
    assert e.value.code == -1
