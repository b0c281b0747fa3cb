import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: larger CPU oracle runs")


def rel(a, b):
    import numpy as np
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


import pytest as _pytest


@_pytest.fixture(scope="session")
def mrcm_lib():
    """Builds libmrcm.so once per session (nvcc, sm_103a) and imports the binding."""
    from paper_2009_07965_gb300 import build
    build.build()
    import paper_2009_07965_gb300 as pkg
    return pkg


def gpu_solve(prob, want_iface=True, refine=None):
    """Run the CUDA path on one Problem through the C ABI; numpy results.
    refine: refinement steps of the solve (None: the library default)."""
    import numpy as np
    import torch
    from paper_2009_07965_gb300 import Solver, mrcm_set_refinement
    dev = torch.device("cuda:0")
    K = torch.from_numpy(prob.K).to(dev)
    s = Solver(K, prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha, prob.bc_type)
    if refine is not None:
        mrcm_set_refinement(s.ctx, refine)
    s.build_basis()
    q = torch.from_numpy(prob.q).to(dev)
    g = torch.from_numpy(prob.bc_val).to(dev)
    s.solve(q, g, want_iface=want_iface)
    torch.cuda.synchronize()
    out = dict(p=s.p.cpu().numpy(), Fx=s.Fx.cpu().numpy(), Fy=s.Fy.cpu().numpy(), solver=s)
    if want_iface:
        fa_x, fb_x, fa_y, fb_y = s.iface_parts()
        out.update(Fa_x=fa_x.cpu().numpy(), Fb_x=fb_x.cpu().numpy(),
                   Fa_y=fa_y.cpu().numpy(), Fb_y=fb_y.cpu().numpy())
    return out
