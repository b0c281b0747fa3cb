"""The seeded input generators (shared by the oracle and the GPU path): the
workloads' stated statistics hold.  log K = sigma * xi with xi a zero-mean,
unit-variance Gaussian field of exponential covariance exp(-|r| / lambda),
sampled by circulant embedding; the problems' sources and boundary data have
the stated form."""
import numpy as np
import pytest

from inputs.fields import gaussian_random_field, lognormal_permeability
import inputs


def test_field_is_a_function_of_its_seed():
    a, _ = gaussian_random_field(64, 48, 1 / 64, 1 / 64, 0.1, 7)
    b, _ = gaussian_random_field(64, 48, 1 / 64, 1 / 64, 0.1, 7)
    c, _ = gaussian_random_field(64, 48, 1 / 64, 1 / 64, 0.1, 8)
    assert a.shape == (48, 64) and a.flags.c_contiguous
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_field_has_unit_variance_and_exponential_covariance():
    # ensemble over seeds: pointwise mean ~0 and variance ~1, and the lag-k
    # covariance along each axis ~exp(-k h / lambda)
    n, h, lam = 96, 1 / 96, 0.08
    fields = [gaussian_random_field(n, n, h, h, lam, 100 + s)[0] for s in range(60)]
    x = np.stack(fields)
    assert abs(x.mean()) < 0.05
    assert abs(x.var() - 1.0) < 0.08
    for k in (1, 4, 8):
        cx = float((x[:, :, :-k] * x[:, :, k:]).mean())
        cy = float((x[:, :-k, :] * x[:, k:, :]).mean())
        want = np.exp(-k * h / lam)
        assert abs(cx - want) < 0.06, (k, cx, want)
        assert abs(cy - want) < 0.06, (k, cy, want)


def test_embedding_clips_nothing_at_the_workload_lengths():
    for n, lam in ((256, 0.05), (512, 0.02)):
        _, clipped = gaussian_random_field(n, n, 1 / n, 1 / n, lam, 1)
        assert clipped < 1e-3


def test_lognormal_permeability_scales_the_field_by_sigma():
    xi, _ = gaussian_random_field(80, 60, 1 / 80, 1 / 80, 0.1, 11)
    K = lognormal_permeability(80, 60, 1 / 80, 1 / 80, 4.0, 0.1, 11)
    assert np.all(K > 0)
    assert np.allclose(np.log(K), 2.0 * xi, rtol=0, atol=1e-12)


@pytest.mark.parametrize("bc", ["left_right", "quarter_five_spot"])
def test_problem_sources_and_boundary_data(bc):
    p = inputs.darcy_problem(40, 24, sigma2=1.0, corr=0.1, seed=3, bc=bc)
    assert p.K.shape == (24, 40) and p.q.shape == (24, 40)
    assert p.bc_val.shape == (2 * 40 + 2 * 24,)
    if bc == "quarter_five_spot":
        # pure Neumann: sources balance, no-flow everywhere
        assert p.q.sum() == 0.0 and p.q[0, 0] == 1.0 and p.q[-1, -1] == -1.0
        assert np.all(p.bc_val == 0.0)
    else:
        assert np.all(p.q == 0.0)
        assert np.all(p.bc_val[:24] == 1.0) and np.all(p.bc_val[24:48] == 0.0)


def test_golden_4096_matches_this_generator():
    # the oracle's stored 4096^2 solution was computed for the field this
    # generator makes (fingerprint equal up to the rounding of the FFT and
    # exp of the machine), and its refinement reached the rounding level
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "square4096_qfs_oracle.npz"))
    K = inputs.config_4096().K
    fp = np.array([K.sum(), (K * K).sum(), np.log(K).sum(), K.min(), K.max()])
    assert np.allclose(fp, g["K_fingerprint"], rtol=1e-10, atol=0.0)
    assert int(g["n"]) == 4096 and int(g["refine"]) == 3
    assert g["history"][-1] < 1e-20 * max(1.0, g["history"][0])
    for k in ("p", "Fx", "Fy", "Fa_x", "Fb_x", "Fa_y", "Fb_y"):
        assert len(g[f"{k}_idx"]) == len(g[f"{k}_val"]) >= 9000
        assert np.all(np.isfinite(g[f"{k}_val"])) and float(g[f"{k}_norm"]) > 0
