"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: relative L2 <= 1e-10 in pressure and in each flux array (the
FP64 target), on problems that span several leaves, ragged (truncated)
leaves, both boundary-condition families, one-face segments (64 Robin
responses per leaf) and per-node Robin-to-flux maps.  Both sides refine
their solution with residuals of Eqs. 11.2-14.2 evaluated in double-double
arithmetic, so both approximate the same discrete solution to near FP64
accuracy even where the permeability contrast makes a plain FP64 solve
accurate to only ~1e-6 in the fluxes.
"""
import numpy as np
import pytest

import inputs
from oracle.fine import solve_fine
from oracle.geometry import Decomposition
from oracle.local import LeafProblem
from oracle.mrcm import solve_mrcm as _solve_mrcm
from oracle.recursive import RecursiveMRCM
from conftest import gpu_solve, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10
KEYS = ("p", "Fx", "Fy", "Fa_x", "Fb_x", "Fa_y", "Fb_y")
REFINE = 3


def solve_mrcm(prob):
    return _solve_mrcm(prob, refine=REFINE)


def _compare(g, o, keys=KEYS, tol=TOL):
    errs = {k: rel(g[k], o[k]) for k in keys}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, errs
    return errs


def test_square64_left_right(mrcm_lib):
    prob = inputs.config_64()
    _compare(gpu_solve(prob), solve_mrcm(prob))


@pytest.mark.parametrize("bc", ["left_right", "quarter_five_spot"])
def test_ragged_leaves(mrcm_lib, bc):
    prob = inputs.darcy_problem(40, 36, sigma2=2.0, corr=0.15, seed=31, bc=bc)
    _compare(gpu_solve(prob), solve_mrcm(prob))


@pytest.mark.parametrize("bc", ["left_right", "quarter_five_spot"])
def test_one_face_segments_equal_fine(mrcm_lib, bc):
    # 64 Robin responses per 16x16 leaf; MRCM then equals the fine solution
    prob = inputs.darcy_problem(48, 40, sigma2=2.0, corr=0.2, seed=3, bc=bc, seg=(1, 1), alpha=5.0)
    g = gpu_solve(prob)
    _compare(g, solve_mrcm(prob))
    f = solve_fine(prob)
    for k in ("p", "Fx", "Fy"):
        assert rel(g[k], f[k]) < 1e-10


def test_rectangular_leaves_and_segments(mrcm_lib):
    prob = inputs.darcy_problem(50, 30, sigma2=1.5, corr=0.1, seed=5, bc="left_right",
                                sub=(8, 16), seg=(2, 4), alpha=0.3, Lx=2.0, Ly=0.7)
    _compare(gpu_solve(prob), solve_mrcm(prob))


@pytest.mark.parametrize("alpha", [1e-3, 1e3])
def test_alpha_range(mrcm_lib, alpha):
    prob = inputs.darcy_problem(64, 48, sigma2=1.0, corr=0.1, seed=7, bc="quarter_five_spot",
                                alpha=alpha)
    _compare(gpu_solve(prob, refine=REFINE), solve_mrcm(prob))


def test_tiny_leaves(mrcm_lib):
    prob = inputs.darcy_problem(12, 10, sigma2=1.0, corr=0.3, seed=2, bc="left_right",
                                sub=(1, 2), seg=(1, 1), alpha=2.0)
    _compare(gpu_solve(prob), solve_mrcm(prob))


def _oracle_seg_key(dec, t):
    s = dec.segments[t]
    return (s["axis"], s["line"], s["lo"])


def test_node_maps_match_recursive_oracle(mrcm_lib):
    import torch
    prob = inputs.darcy_problem(64, 48, sigma2=2.0, corr=0.1, seed=17, bc="left_right")
    g = gpu_solve(prob, want_iface=False)
    ctx = g["solver"].ctx
    # node particular fluxes of the plain solve (refinement passes overwrite
    # them with those of the correction data)
    mrcm_lib.mrcm_set_refinement(ctx, 0)
    g["solver"].solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda())
    rm = RecursiveMRCM(prob)
    rm.solve()
    dec = rm.dec
    by_box = {}
    stack = [rm.root]
    while stack:
        nd = stack.pop()
        stack += nd.children
        by_box[tuple(nd.box)] = nd
    nnodes = mrcm_lib.mrcm_query(ctx, "NODES")
    assert nnodes == len(by_box)
    checked = 0
    for v in range(nnodes):
        info = mrcm_lib.mrcm_node_info(ctx, v)
        nd = by_box[(info["I0"], info["I1"], info["J0"], info["J1"])]
        if info["parent"] < 0:
            continue
        R_gpu, rbar_gpu = mrcm_lib.mrcm_node_operator(ctx, v, with_rbar=True)
        keys = []
        for t in mrcm_lib.mrcm_node_segments(ctx, v):
            si = mrcm_lib.mrcm_segment_info(ctx, t)
            keys.append((si["axis"], si["line"], si["lo"]))
        okey = {_oracle_seg_key(dec, t): k for k, t in enumerate(nd.segs)}
        perm = [okey[k] for k in keys]
        R_o = nd.R[np.ix_(perm, perm)]
        assert rel(R_gpu, R_o) < 1e-11, (v, rel(R_gpu, R_o))
        assert rel(rbar_gpu, nd.rbar[perm]) < 1e-10
        checked += 1
    assert checked == nnodes - 1


def test_leaf_maps_match_oracle(mrcm_lib):
    prob = inputs.config_64()
    g = gpu_solve(prob, want_iface=False)
    ctx = g["solver"].ctx
    dec = Decomposition(prob)
    for leaf in range(len(dec.leaves)):
        lp = LeafProblem(dec, leaf)
        R_o, _ = lp.robin_to_flux()
        R_g = mrcm_lib.mrcm_node_operator(ctx, leaf)
        keys = []
        for t in mrcm_lib.mrcm_node_segments(ctx, leaf):
            si = mrcm_lib.mrcm_segment_info(ctx, t)
            keys.append((si["axis"], si["line"], si["lo"]))
        okey = {_oracle_seg_key(dec, t): k for k, t in enumerate(lp.segs)}
        perm = [okey[k] for k in keys]
        assert rel(R_g, R_o[np.ix_(perm, perm)]) < 1e-12
        # symmetric and annihilating constants on Dirichlet-free leaves
        assert np.abs(R_g - R_g.T).max() < 1e-12 * np.abs(R_g).max()


def test_repeat_solves_bitwise_identical(mrcm_lib):
    import torch
    prob = inputs.darcy_problem(64, 64, sigma2=2.0, corr=0.1, seed=9, bc="quarter_five_spot")
    g = gpu_solve(prob, want_iface=False)
    s = g["solver"]
    q = torch.from_numpy(prob.q).cuda()
    bc = torch.from_numpy(prob.bc_val).cuda()
    s.build_basis()
    p2, fx2, fy2 = [x.cpu().numpy() for x in s.solve(q, bc)]
    assert np.array_equal(p2, g["p"]) and np.array_equal(fx2, g["Fx"]) and np.array_equal(fy2, g["Fy"])


def test_graph_replay_matches_direct_launches(mrcm_lib):
    # on a side stream mrcm_build_basis / mrcm_solve replay CUDA graphs; the
    # replay (also with new input buffers and with phase timing) must give
    # the direct launches' results bit for bit
    import paper_2009_07965_gb300 as mr
    import torch
    prob = inputs.darcy_problem(128, 128, sigma2=3.0, corr=0.1, seed=31, bc="quarter_five_spot")
    st = torch.cuda.Stream()
    res = {}
    for graphs in (False, True):
        with torch.cuda.stream(st):
            s = mr.Solver(torch.from_numpy(prob.K).cuda(), sub=prob.sub, seg=prob.seg, alpha=prob.alpha,
                          bc_type=prob.bc_type, stream=st)
            mr.mrcm_use_graphs(s.ctx, graphs)
            out = []
            for it in range(3):
                if it == 2:
                    mr.mrcm_enable_timing(s.ctx, True)
                s.build_basis()
                for scale in (1.0, 2.5, 1.0):
                    q = torch.from_numpy(scale * prob.q).cuda()          # a new buffer every call
                    bc = torch.from_numpy(scale * prob.bc_val).cuda()
                    s.solve(q, bc)
                    out.append([t.cpu().numpy().copy() for t in (s.p, s.Fx, s.Fy)])
            assert mr.mrcm_query(s.ctx, "GRAPH_REPLAYS") == (12 if graphs else 0)
            if graphs:
                ms = mr.mrcm_phase_times(s.ctx)
                assert ms["leaf_build"] > 0 and ms["finish"] > 0
            st.synchronize()
            s.close()
        res[graphs] = out
    assert len(res[False]) == len(res[True]) == 9
    for a, b in zip(res[False], res[True]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    for k in (3, 6):
        for x, y in zip(res[True][0], res[True][k]):
            assert np.array_equal(x, y)
    assert not np.array_equal(res[True][0][0], res[True][1][0])


def test_errors_are_reported(mrcm_lib):
    import torch
    from paper_2009_07965_gb300 import Solver, MrcmError
    K = torch.ones(32, 32, dtype=torch.float64, device="cuda")
    s = Solver(K)
    q = torch.zeros(32, 32, dtype=torch.float64, device="cuda")
    bc = torch.zeros(2 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(MrcmError) as e:
        s.solve(q, bc)
    assert e.value.code == -4            # NOT_BUILT
    K[3, 5] = -1.0
    s.set_permeability(K)
    with pytest.raises(MrcmError) as e:
        s.build_basis()
    assert e.value.code == -3            # BAD_K
    K[3, 5] = float("nan")
    s.set_permeability(K)
    with pytest.raises(MrcmError) as e:
        s.build_basis()
    assert e.value.code == -3
    K[3, 5] = 1.0
    s.set_permeability(K)
    s.build_basis()
    s.solve(q, bc)                       # the context stays usable
    with pytest.raises(MrcmError) as e:
        Solver(K, sub=(16, 16), seg=(3, 4))
    assert e.value.code == -2            # SHAPE


def test_refinement_converges(mrcm_lib):
    import paper_2009_07965_gb300 as mr
    import torch
    prob = inputs.darcy_problem(256, 256, sigma2=4.0, corr=0.05, seed=2000, bc="quarter_five_spot")
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), sub=prob.sub, seg=prob.seg, alpha=prob.alpha,
                  bc_type=prob.bc_type)
    mr.mrcm_set_refinement(s.ctx, 3, check=True)
    s.build_basis()
    s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda())
    hist = mr.mrcm_residual_history(s.ctx)
    assert len(hist) == 4
    assert hist[-1] < 1e-13 and hist[-1] <= hist[0], hist
    g = {k: v.cpu().numpy() for k, v in zip(("p", "Fx", "Fy"), (s.p, s.Fx, s.Fy))}
    _compare(g, solve_mrcm(prob), keys=("p", "Fx", "Fy"))


def test_unrefined_solve_is_close_to_the_refined_one(mrcm_lib):
    # the quasi-definite interface inverses keep the plain FP64 solve of a
    # high-contrast field close to the discrete solution; one refinement
    # step (the default) then reaches the rounding level
    import paper_2009_07965_gb300 as mr
    import torch
    prob = inputs.darcy_problem(256, 256, sigma2=4.0, corr=0.05, seed=2001, bc="quarter_five_spot")
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), sub=prob.sub, seg=prob.seg, alpha=prob.alpha,
                  bc_type=prob.bc_type)
    s.build_basis()
    q, bc = torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda()
    out = {}
    for k in (0, 1, 3):
        mr.mrcm_set_refinement(s.ctx, k)
        s.solve(q, bc)
        out[k] = [t.cpu().numpy().copy() for t in (s.p, s.Fx, s.Fy)]
    for a, b in zip(out[0], out[3]):
        assert rel(a, b) < 1e-9
    for a, b in zip(out[1], out[3]):
        assert rel(a, b) < 1e-14


@pytest.mark.parametrize("bc", ["left_right", "quarter_five_spot"])
def test_single_pass_matches_oracle(mrcm_lib, bc):
    # the paper's single pass (no refinement step; outputs formed in plain
    # FP64, the all-Neumann mean shift on the high parts) against the oracle
    # at the FP64 form's 1e-10 rel-L2, one-sided fluxes included
    import paper_2009_07965_gb300 as mr
    import torch
    prob = inputs.darcy_problem(160, 144, sigma2=4.0, corr=0.05, seed=77, bc=bc)
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                  prob.bc_type)
    mr.mrcm_set_refinement(s.ctx, 0)
    s.build_basis()
    s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda(), want_iface=True)
    fa_x, fb_x, fa_y, fb_y = s.iface_parts()
    g = dict(p=s.p, Fx=s.Fx, Fy=s.Fy, Fa_x=fa_x, Fb_x=fb_x, Fa_y=fa_y, Fb_y=fb_y)
    g = {k: v.cpu().numpy() for k, v in g.items()}
    _compare(g, solve_mrcm(prob), tol=1e-10)


def test_heights_with_more_nodes_than_ctas(mrcm_lib):
    # one-cell segments: at 512^2 the first blocked height (2g = 64) has 256
    # nodes, more than the sweep's CTAs, so CTAs take several form, look-ahead
    # and back-form items in a row; MRCM with one-face segments equals the fine
    # solution, and a repeated build gives the same bits
    import paper_2009_07965_gb300 as mr
    import torch
    prob = inputs.darcy_problem(512, 512, sigma2=2.0, corr=0.1, seed=41, bc="quarter_five_spot", seg=(1, 1),
                                alpha=5.0)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                      prob.bc_type, stream=st)
        q, bc = torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda()
        outs = []
        for _ in range(2):
            s.build_basis()
            s.solve(q, bc)
            outs.append([t.cpu().numpy().copy() for t in (s.p, s.Fx, s.Fy)])
        st.synchronize()
        s.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    f = solve_fine(prob)
    for k, g in zip(("p", "Fx", "Fy"), outs[0]):
        assert rel(g, f[k]) < 1e-10, (k, rel(g, f[k]))


def test_square512_same_recipe_as_benchmark(mrcm_lib):
    # the benchmark recipe (sigma^2 = 4, corr 0.05, quarter-five-spot) at
    # 512^2: 1024 leaves, 10 levels, interface systems up to 2g = 256
    prob = inputs.darcy_problem(512, 512, sigma2=4.0, corr=0.05, seed=2000, bc="quarter_five_spot")
    _compare(gpu_solve(prob), solve_mrcm(prob))


@pytest.mark.slow
def test_square1024_quarter_five_spot_full_size(mrcm_lib):
    # the benchmark workload (1024^2, sigma^2 = 4, 4096 leaves, 12 levels)
    prob = inputs.config_1024()
    g = gpu_solve(prob, want_iface=True)
    errs = _compare(g, solve_mrcm(prob))
    print("1024^2 rel errors", errs)


def test_kernel_reciprocal_within_an_ulp(mrcm_lib):
    # the Newton-Raphson reciprocal of the pivot chains against CUDA's
    # division (torch on the same device): within one ulp over a wide range
    # of magnitudes, both signs, powers of two, and the fallback range
    import paper_2009_07965_gb300 as mr
    import torch
    rng = np.random.default_rng(11)
    x = np.concatenate([
        np.exp(rng.uniform(-80.0, 80.0, 200000)) * rng.choice([-1.0, 1.0], 200000),
        2.0 ** np.arange(-125, 126, dtype=np.float64),
        np.array([1.0, -1.0, 3.0, 1e-40, -1e-40, 1e40, 7.5e37, 1.5e-37, 0.9999999999999999, 1.0000000000000002]),
    ])
    xd = torch.from_numpy(x).cuda()
    r = mr.mrcm_check_reciprocal(xd).cpu().numpy()
    ref = (1.0 / xd).cpu().numpy()
    err = np.abs(r - ref) / np.spacing(np.abs(ref))
    assert err.max() <= 1.0, (err.max(), x[np.argmax(err)])


def test_autotuned_launch_shapes_give_the_same_bits(mrcm_lib):
    # the tuner times every launch shape of the blocked levels and keeps the
    # fastest; all shapes compute the same numbers, so the solution after
    # tuning (graph replay included) is bit-identical to the untuned one
    import paper_2009_07965_gb300 as mr
    import torch
    prob = inputs.darcy_problem(512, 512, sigma2=3.0, corr=0.05, seed=47, bc="quarter_five_spot")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                      prob.bc_type, stream=st)
        q, bc = torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda()
        s.build_basis()
        s.solve(q, bc)
        before = [t.cpu().numpy().copy() for t in (s.p, s.Fx, s.Fy)]
        levels = mr.mrcm_query(s.ctx, "LEVELS")
        assert all(v == 0 for h in range(1, levels + 1) for v in mr.mrcm_tune_info(s.ctx, h).values())
        mr.mrcm_autotune(s.ctx, 2)
        chosen = [mr.mrcm_tune_info(s.ctx, h) for h in range(1, levels + 1)]
        assert any(c["sweep_per_sm"] in (1, 2, 3) for c in chosen), chosen
        for _ in range(2):
            s.build_basis()
            s.solve(q, bc)
            after = [t.cpu().numpy() for t in (s.p, s.Fx, s.Fy)]
            for a, b in zip(before, after):
                assert np.array_equal(a, b)
        st.synchronize()
        s.close()
    with pytest.raises(mr.MrcmError) as e:
        s2 = mr.Solver(torch.from_numpy(prob.K).cuda())
        mr.mrcm_autotune(s2.ctx, 1)                   # not built
    assert e.value.code == -4
