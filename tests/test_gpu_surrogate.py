"""The learned basis surrogate: training targets from the plain method, the
network's BF16 kernels against a CPU FP32 reference, training on the GPU,
and the residual gate with the plain local solve as fallback.

- Basis fields psi_s = A^-1 B e_s of interior leaves against the oracle's
  local solves (Eqs. 11Hhatbasisa/b), to float accuracy.
- Convolution forward, weight gradient and input gradient (forward kernel
  on flipped weights) against the oracle's FP64 arithmetic (oracle.cnn) on
  the same BF16-rounded operands.
- Training with the library's kernels lowers the loss.
- The gate accepts exact fields and refuses wrong ones; with accepted exact
  fields the solution equals the plain one to float accuracy; with a trained
  network and tau = 1e-4 (the workload's threshold) the result stays within
  the surrogate form's 1e-3 of the oracle, and the accepted fraction is
  reported (what the network gains over the method without it).
"""
import numpy as np
import pytest

import inputs
from oracle.cnn import conv3x3, conv3x3_wgrad, conv3x3_xgrad
from oracle.geometry import Decomposition
from oracle.local import LeafProblem
from oracle.mrcm import solve_mrcm
from conftest import rel

pytestmark = pytest.mark.gpu
SHAPES = [(16, 32, 0), (16, 32, 1), (32, 32, 1), (32, 16, 1)]


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def _leaf_key_perm(mr, ctx, dec, lp, leaf):
    keys = []
    for t in mr.mrcm_node_segments(ctx, leaf):
        si = mr.mrcm_segment_info(ctx, t)
        keys.append((si["axis"], si["line"], si["lo"]))
    okey = {(dec.segments[t]["axis"], dec.segments[t]["line"], dec.segments[t]["lo"]): k
            for k, t in enumerate(lp.segs)}
    return [okey[k] for k in keys]


def test_leaf_fields_match_the_oracle(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(80, 80, sigma2=2.0, corr=0.1, seed=21, bc="left_right")
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha, prob.bc_type)
    s.build_basis()
    ids = mr.mrcm_interior_leaves(s.ctx)
    assert len(ids) == 9
    idt = torch.tensor(ids, dtype=torch.int32, device="cuda")
    psi = torch.empty((len(ids), 256, 16), dtype=torch.float32, device="cuda")
    mr.mrcm_leaf_fields(s.ctx, idt, psi)
    psi = psi.cpu().numpy()
    dec = Decomposition(prob)
    for item, leaf in enumerate(ids):
        lp = LeafProblem(dec, leaf)
        p, _, _ = lp.solve(np.eye(len(lp.segs)), with_data=False, want_faces=False)
        perm = _leaf_key_perm(mr, s.ctx, dec, lp, leaf)
        assert rel(psi[item], p[:, perm]) < 1e-6, (leaf, rel(psi[item], p[:, perm]))
        # the discrete maximum principle: responses in [0, 1]
        assert psi[item].min() > -1e-6 and psi[item].max() < 1 + 1e-6
    s.close()


@pytest.mark.parametrize("cin,cout,pad", SHAPES)
def test_conv_forward_matches_cpu_reference(mrcm_lib, cin, cout, pad):
    import torch
    import paper_2009_07965_gb300 as mr
    rng = np.random.default_rng(cin + cout + pad)
    n, hin = 5, 16 if pad else 18
    xb = _bf16(rng.standard_normal((n, hin, hin, cin)))
    wb = _bf16(rng.standard_normal((cout, 3, 3, cin)) * 0.2)
    b = rng.standard_normal(cout).astype(np.float32)
    y = torch.empty((n, 16, 16, cout), dtype=torch.float32, device="cuda")
    ybf = torch.empty((n, 16, 16, cout), dtype=torch.bfloat16, device="cuda")
    for relu in (False, True):
        mr.mrcm_cnn_conv_forward(xb.cuda(), n, cin, cout, pad, relu, wb.cuda(), torch.from_numpy(b).cuda(), ybf, y)
        ref = conv3x3(xb.float().numpy(), wb.float().numpy(), b, pad)
        if relu:
            ref = np.maximum(ref, 0.0)
        assert rel(y.cpu().numpy(), ref) < 1e-5, (relu, rel(y.cpu().numpy(), ref))
        assert rel(ybf.float().cpu().numpy(), ref) < 1e-2


@pytest.mark.parametrize("cin,cout,pad", [(16, 32, 0), (32, 32, 1), (32, 16, 1)])
def test_conv_gradients_match_cpu_reference(mrcm_lib, cin, cout, pad):
    import torch
    import paper_2009_07965_gb300 as mr
    rng = np.random.default_rng(7 * cin + cout)
    n, hin = 6, 16 if pad else 18
    xb = _bf16(rng.standard_normal((n, hin, hin, cin)))
    wb = _bf16(rng.standard_normal((cout, 3, 3, cin)) * 0.2)
    dyb = _bf16(rng.standard_normal((n, 16, 16, cout)))
    dw = torch.zeros((cout, 3, 3, cin), dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    mr.mrcm_cnn_conv_wgrad(xb.cuda(), dyb.cuda(), n, cin, cout, pad, dw, db)
    ref, ref_db = conv3x3_wgrad(xb.float().numpy(), dyb.float().numpy(), pad)
    assert rel(dw.cpu().numpy(), ref) < 1e-5, rel(dw.cpu().numpy(), ref)
    assert rel(db.cpu().numpy(), ref_db) < 1e-5
    if pad:
        # input gradient: the forward kernel on flipped weights
        w2 = torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device="cuda")
        mr.mrcm_cnn_flip_weights(wb.cuda(), cout, cin, w2)
        dx = torch.empty((n, 16, 16, cin), dtype=torch.float32, device="cuda")
        mr.mrcm_cnn_conv_forward(dyb.cuda(), n, cout, cin, 1, False, w2, None, None, dx)
        ref_dx = conv3x3_xgrad(dyb.float().numpy(), wb.float().numpy())
        assert rel(dx.cpu().numpy(), ref_dx) < 1e-5, rel(dx.cpu().numpy(), ref_dx)


def _training_set(mr, probs):
    import torch
    xs, ys = [], []
    for prob in probs:
        s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha,
                      prob.bc_type)
        s.build_basis()
        idt = torch.tensor(mr.mrcm_interior_leaves(s.ctx), dtype=torch.int32, device="cuda")
        x = torch.empty((idt.numel(), 18, 18, 16), dtype=torch.bfloat16, device="cuda")
        y = torch.empty((idt.numel(), 256, 16), dtype=torch.float32, device="cuda")
        mr.mrcm_leaf_patches(s.ctx, idt, x)
        mr.mrcm_leaf_fields(s.ctx, idt, y)
        xs.append(x)
        ys.append(y.view(-1, 16, 16, 16))
        s.close()
    return torch.cat(xs), torch.cat(ys)


def test_training_lowers_the_loss(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    from paper_2009_07965_gb300.surrogate import BasisSurrogate
    probs = [inputs.darcy_problem(256, 256, sigma2=2.0, corr=0.1, seed=300 + k, bc="left_right") for k in range(2)]
    x, y = _training_set(mr, probs)
    net = BasisSurrogate(seed=1)
    losses = []
    g = torch.Generator(device="cpu").manual_seed(0)
    for it in range(300):
        idx = torch.randint(0, x.shape[0], (64,), generator=g).cuda()
        losses.append(net.train_step(x[idx].contiguous(), y[idx].contiguous(), lr=2e-3))
    first, last = np.mean(losses[:10]), np.mean(losses[-10:])
    print("surrogate training loss", first, "->", last)
    assert last < 0.3 * first, (first, last)


def test_gate_accepts_exact_fields_and_refuses_wrong_ones(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    prob = inputs.darcy_problem(96, 96, sigma2=2.0, corr=0.1, seed=5, bc="left_right")
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha, prob.bc_type)
    q, bc = torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda()
    s.build_basis()
    s.solve(q, bc)
    plain = [t.cpu().numpy().copy() for t in (s.p, s.Fx, s.Fy)]
    idt = torch.tensor(mr.mrcm_interior_leaves(s.ctx), dtype=torch.int32, device="cuda")
    n = idt.numel()
    psi = torch.empty((n, 256, 16), dtype=torch.float32, device="cuda")
    mr.mrcm_leaf_fields(s.ctx, idt, psi)
    res = torch.empty(n, dtype=torch.float64, device="cuda")
    mr.mrcm_leaf_gate(s.ctx, idt, psi, res)
    assert float(res.max()) < 1e-5, float(res.max())         # float storage of exact fields
    bad = torch.zeros_like(psi)
    res_bad = torch.empty_like(res)
    mr.mrcm_leaf_gate(s.ctx, idt, bad, res_bad)
    assert float(res_bad.min()) > 0.99                       # zero fields: residual = ||B e_s||
    acc = torch.empty(n, dtype=torch.int32, device="cuda")
    mr.mrcm_leaf_apply(s.ctx, idt, psi, res, 1e-4, acc)
    assert int(acc.sum()) == n
    s.solve(q, bc)
    for a, b in zip((s.p, s.Fx, s.Fy), plain):
        assert rel(a.cpu().numpy(), b) < 1e-5
    s.close()


def test_trained_surrogate_with_fallback_against_the_oracle(mrcm_lib):
    import torch
    import paper_2009_07965_gb300 as mr
    from paper_2009_07965_gb300.surrogate import BasisSurrogate
    probs = [inputs.darcy_problem(256, 256, sigma2=1.0, corr=0.1, seed=400 + k, bc="left_right") for k in range(2)]
    x, y = _training_set(mr, probs)
    net = BasisSurrogate(seed=2)
    g = torch.Generator(device="cpu").manual_seed(1)
    for it in range(400):
        idx = torch.randint(0, x.shape[0], (64,), generator=g).cuda()
        net.train_step(x[idx].contiguous(), y[idx].contiguous(), lr=2e-3)
    prob = inputs.darcy_problem(128, 128, sigma2=1.0, corr=0.1, seed=499, bc="left_right")
    s = mr.Solver(torch.from_numpy(prob.K).cuda(), prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha, prob.bc_type)
    mr.mrcm_set_refinement(s.ctx, 3)
    s.build_basis()
    idt = torch.tensor(mr.mrcm_interior_leaves(s.ctx), dtype=torch.int32, device="cuda")
    o = solve_mrcm(prob, refine=3)
    for tau in (1e-4, 1e-2):
        try:
            acc, res = net.apply(s.ctx, idt, tau)
            s.solve(torch.from_numpy(prob.q).cuda(), torch.from_numpy(prob.bc_val).cuda())
        except mr.MrcmError as e:
            # maps far from a Robin-to-flux map can break the interface
            # systems' quasi-definite form: reported, not hidden
            print(f"surrogate tau={tau}: refused by the merges ({e})")
            assert tau > 1e-4
            s.build_basis()
            continue
        out = {k: t.cpu().numpy() for k, t in (("p", s.p), ("Fx", s.Fx), ("Fy", s.Fy))}
        errs = {k: rel(out[k], o[k]) for k in out}
        print(f"surrogate tau={tau}: accepted {acc.mean():.3f} of {acc.size} interior leaves, median residual "
              f"{np.median(res):.3e}, rel errors vs oracle {errs}")
        if tau == 1e-4:
            assert max(errs.values()) <= 1e-3, errs
        s.build_basis()                              # back to the plain maps
    s.close()
