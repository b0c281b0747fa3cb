"""The root interface system kept as a block LDL^T factor (the default,
MRCM_ROOT_FACTOR) or as an explicit inverse (MRCM_ROOT_INVERSE).

The two forms solve the same equations (Algorithm 1's top merge, Section
3.2), so:
- with refinement both match the FP64 oracle at the parity tolerance
  (rel-L2 <= 1e-10 in p, Fx, Fy and the one-sided skeleton fluxes);
- their single-pass solutions agree to rounding;
on roots whose system size 2g is not a multiple of the factor's 16-wide
blocks or of the sweeps' 64-wide solve blocks, on pinned roots (all-Neumann
problems: the regularised form), on batched roots (several trees' roots in
one launch) and on an FP32 root of the mixed form.  The factor form's flops
are booked under its own phase.
"""
import numpy as np
import pytest

import inputs
from oracle.mrcm import solve_mrcm
from conftest import rel

pytestmark = pytest.mark.gpu
KEYS = ("p", "Fx", "Fy", "Fa_x", "Fb_x", "Fa_y", "Fb_y")


def _solve(mr, prob, form, refine, precision=0, split=None):
    import torch
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                  prob.bc_type, precision=precision)
    mr.mrcm_set_root_form(s.ctx, form)
    if split is not None:
        mr.mrcm_set_mixed_split(s.ctx, split)
    mr.mrcm_set_refinement(s.ctx, refine)
    s.build_basis()
    s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda(), want_iface=True)
    torch.cuda.synchronize()
    out = dict(p=s.p.cpu().numpy(), Fx=s.Fx.cpu().numpy(), Fy=s.Fy.cpu().numpy())
    fa_x, fb_x, fa_y, fb_y = s.iface_parts()
    out.update(Fa_x=fa_x.cpu().numpy(), Fb_x=fb_x.cpu().numpy(), Fa_y=fa_y.cpu().numpy(),
               Fb_y=fb_y.cpu().numpy())
    return s, out


def _root_g2(mr, s):
    return mr.mrcm_query(s.ctx, "MAX_GAMMA")


CASES = {
    # 2g of the root: 68 (four 16-blocks and a ragged one), pinned
    "qfs_200x136": dict(nx=200, ny=136, sigma2=2.0, corr=0.1, seed=11, bc="quarter_five_spot"),
    # 2g = 272: four full solve blocks and a 16-row one
    "lr_200x136_seg1": dict(nx=200, ny=136, sigma2=2.0, corr=0.1, seed=12, bc="left_right", seg=(1, 1),
                            alpha=5.0),
    # rectangular leaves and segments, 2g = 2 * 60 / 2
    "lr_rect": dict(nx=150, ny=120, sigma2=1.5, corr=0.1, seed=13, bc="left_right", sub=(8, 16), seg=(2, 4),
                    alpha=0.3, Lx=2.0, Ly=0.7),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_factor_root_matches_the_oracle_and_the_inverse(mrcm_lib, name):
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(**CASES[name])
    sf, gf = _solve(mr, prob, mr.binding.MRCM_ROOT_FACTOR, refine=3)
    assert _root_g2(mr, sf) > 32                     # a blocked root
    o = solve_mrcm(prob, refine=3)
    errs = {k: rel(gf[k], o[k]) for k in KEYS}
    assert all(e <= 1e-10 for e in errs.values()), errs
    # single passes of the two forms agree to rounding
    sf1, gf1 = _solve(mr, prob, mr.binding.MRCM_ROOT_FACTOR, refine=0)
    si1, gi1 = _solve(mr, prob, mr.binding.MRCM_ROOT_INVERSE, refine=0)
    d = {k: rel(gf1[k], gi1[k]) for k in ("p", "Fx", "Fy")}
    assert all(e <= 1e-9 for e in d.values()), d
    # flops: the root's sweep is booked as the factorisation
    ff = mr.mrcm_phase_flops(sf1.ctx)
    fi = mr.mrcm_phase_flops(si1.ctx)
    assert ff["root_factor"] > 0 and fi["root_factor"] == 0
    assert ff["gj_sweep"] < fi["gj_sweep"]
    n = _root_g2(mr, sf1)
    assert abs(ff["root_factor"] - n * (n * n - 1) / 3.0) < 1e-6 * n ** 3
    for s in (sf, sf1, si1):
        s.close()


def test_factor_root_phase_is_timed(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(**CASES["lr_200x136_seg1"])
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                  prob.bc_type)
    mr.mrcm_set_root_form(s.ctx, mr.binding.MRCM_ROOT_FACTOR)
    mr.mrcm_enable_timing(s.ctx, 1)
    s.build_basis()
    s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda())
    ms = mr.mrcm_phase_times(s.ctx)
    assert ms["root_factor"] > 0 and ms["tree_up"] > 0 and ms["tree_down"] > 0
    s.close()


def test_batched_roots_in_one_factor_launch(mrcm_lib):
    """Equal-sized problems put every root at the top height (count > 1)."""
    import torch
    import paper_2009_07965_gb300 as mr
    # (all-Neumann problems run in contexts of their own)
    probs = [inputs.darcy_problem(96, 80, sigma2=1.0 + k, corr=0.1, seed=40 + k, bc="left_right", seg=(2, 2))
             for k in range(3)]
    outs = {}
    for form in (mr.binding.MRCM_ROOT_FACTOR, mr.binding.MRCM_ROOT_INVERSE):
        Ks = [torch.from_numpy(p.K).cuda() for p in probs]
        b = mr.BatchSolver(Ks, [(p.Lx, p.Ly) for p in probs], [p.bc_type for p in probs], sub=probs[0].sub,
                           seg=probs[0].seg, alpha=probs[0].alpha)
        mr.mrcm_set_root_form(b.ctx, form)
        mr.mrcm_set_refinement(b.ctx, 3)
        b.build_basis()
        b.solve([torch.from_numpy(p.q).cuda() for p in probs], [torch.from_numpy(p.bc_val).cuda() for p in probs])
        outs[form] = [tuple(t.cpu().numpy().copy() for t in r) for r in b.split()]
        if form == mr.binding.MRCM_ROOT_FACTOR:
            assert mr.mrcm_phase_flops(b.ctx)["root_factor"] > 0
    for k, prob in enumerate(probs):
        o = solve_mrcm(prob, refine=3)
        for form in outs:
            p, fx, fy = outs[form][k]
            errs = (rel(p, o["p"]), rel(fx, o["Fx"]), rel(fy, o["Fy"]))
            assert max(errs) <= 1e-10, (k, form, errs)


def test_fp32_root_factor_refines_to_the_oracle(mrcm_lib):
    """The mixed form with every merge in FP32, the root's factor included."""
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(**CASES["lr_200x136_seg1"])
    s, g = _solve(mr, prob, mr.binding.MRCM_ROOT_FACTOR, refine=6, precision=mr.binding.MRCM_MIXED,
                  split=1 << 20)
    o = solve_mrcm(prob, refine=3)
    errs = {k: rel(g[k], o[k]) for k in ("p", "Fx", "Fy")}
    assert all(e <= 1e-8 for e in errs.values()), errs
    s.close()


def test_auto_form_keeps_small_roots_inverted(mrcm_lib):
    """The default factors roots from 2g = 1024 on; this root has 2g = 272."""
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(**CASES["lr_200x136_seg1"])
    s, g = _solve(mr, prob, mr.binding.MRCM_ROOT_AUTO, refine=3)
    assert mr.mrcm_phase_flops(s.ctx)["root_factor"] == 0
    o = solve_mrcm(prob, refine=3)
    assert max(rel(g[k], o[k]) for k in ("p", "Fx", "Fy")) <= 1e-10
    s.close()


def test_root_form_switch_needs_a_rebuild(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(**CASES["qfs_200x136"])
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                  prob.bc_type)
    s.build_basis()
    mr.mrcm_set_root_form(s.ctx, mr.binding.MRCM_ROOT_INVERSE)
    with pytest.raises(mr.MrcmError) as e:
        s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda())
    assert e.value.code == -4                       # MRCM_ERR_NOT_BUILT
    with pytest.raises(mr.MrcmError) as e:
        mr.mrcm_set_root_form(s.ctx, 7)
    assert e.value.code == -1
    s.build_basis()
    s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda())
    s.close()
