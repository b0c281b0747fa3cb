"""The C-ABI library loads and exports what include/mrcm.h declares; host-only
calls (error strings, planning) work without a GPU."""
import os
import re

import numpy as np
import pytest

import inputs
from oracle.geometry import Decomposition
from oracle.recursive import build_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "mrcm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrcm_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(mrcm_lib):
    import ctypes
    lib = ctypes.CDLL(mrcm_lib.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(mrcm_lib.EXPORTS) == declared


def test_error_strings(mrcm_lib):
    for code in range(-9, 1):
        assert mrcm_lib.mrcm_error_string(code)
    assert mrcm_lib.mrcm_error_string(-5).startswith("singular")


def _tree_height(node):
    if not node.children:
        return 0
    return 1 + max(_tree_height(c) for c in node.children)


@pytest.mark.parametrize("n,sub,seg,bc", [((64, 64), (16, 16), (4, 4), (1, 1, 0, 0)),
                                          ((40, 36), (16, 16), (4, 4), (0, 0, 0, 0)),
                                          ((50, 30), (8, 16), (2, 4), (1, 1, 0, 0)),
                                          ((48, 48), (16, 16), (1, 1), (1, 1, 0, 0)),
                                          ((1024, 1024), (16, 16), (4, 4), (0, 0, 0, 0))])
def test_plan_matches_oracle_decomposition(mrcm_lib, n, sub, seg, bc):
    q = lambda k: mrcm_lib.mrcm_plan_query(n, (1.0, 1.0), sub, seg, bc, k)
    prob = inputs.darcy_problem(n[0], n[1], sigma2=0.0, sub=sub, seg=seg)
    dec = Decomposition(prob) if n[0] * n[1] <= 4096 else None
    nl = -(-n[0] // sub[0]) * -(-n[1] // sub[1])
    assert q("LEAVES") == nl
    assert q("NODES") == 2 * nl - 1
    if dec is not None:
        assert q("SEGMENTS") == len(dec.segments)
        assert q("LEVELS") == _tree_height(build_tree(dec))
    assert q("BUILD_FLOPS") > q("LEAF_FLOPS") > 0


def test_plan_counts_for_the_paper_layout(mrcm_lib):
    # 2D analogue of Table ntmmbfs: interior segments per leaf side = H/Hbar
    for (a, b) in [(4, 8), (8, 8), (16, 32)]:
        for r in (1, 4):
            segs = mrcm_lib.mrcm_plan_query((16 * a, 16 * b), (1, 1), (16, 16), (16 // r, 16 // r),
                                            (1, 1, 0, 0), "SEGMENTS")
            assert segs == r * ((a - 1) * b + a * (b - 1))


def test_setup_rejects_bad_shapes_without_a_device(mrcm_lib):
    from paper_2009_07965_gb300.binding import MrcmError
    with pytest.raises(MrcmError) as e:
        mrcm_lib.mrcm_plan_query((64, 64), (1, 1), (16, 16), (3, 4), (1, 1, 0, 0), "LEAVES")
    assert e.value.code == -2
    with pytest.raises(MrcmError) as e:
        mrcm_lib.mrcm_plan_query((64, 64), (1, 1), (32, 32), (4, 4), (1, 1, 0, 0), "LEAVES")
    assert e.value.code == -2
    with pytest.raises(MrcmError) as e:
        mrcm_lib.mrcm_plan_query((64, 64), (1, 1), (16, 16), (4, 4), (1, 2, 0, 0), "LEAVES")
    assert e.value.code == -1


def test_unsupported_requests_are_refused_before_any_device_work(mrcm_lib):
    # The surrogate precision (2D and 3D)
    # and 3D batches are refused with MRCM_ERR_UNSUPPORTED, 3D shapes that the
    # blocks cannot tile with MRCM_ERR_SHAPE, after validating the host
    # arguments and before touching the device (the permeability pointer is
    # never read)
    import ctypes
    from paper_2009_07965_gb300 import binding as B
    lib = B._lib()
    ctx = ctypes.c_void_p()
    fake_K = ctypes.c_void_p(16)
    sub, seg, bc = B._ints((16, 16, 16), 3), B._ints((4, 4, 4), 3), B._ints((1, 1, 0, 0, 0, 0), 6)
    g3 = B.mrcm_grid(3, (ctypes.c_int * 3)(64, 64, 64), (ctypes.c_double * 3)(1.0, 1.0, 1.0))
    assert lib.mrcm_setup(ctypes.byref(ctx), ctypes.byref(g3), fake_K, sub, seg, 1.0, bc, B.MRCM_SURROGATE,
                          None) == -9
    two = (B.mrcm_grid * 2)(g3, g3)
    bc2 = B._ints((1, 1, 0, 0, 0, 0) * 2, 12)
    assert lib.mrcm_setup_batch(ctypes.byref(ctx), 2, two, bc2, fake_K, sub, seg, 1.0, B.MRCM_FP64,
                                None) == -9
    ragged = B.mrcm_grid(3, (ctypes.c_int * 3)(64, 64, 40), (ctypes.c_double * 3)(1.0, 1.0, 1.0))
    assert lib.mrcm_setup(ctypes.byref(ctx), ctypes.byref(ragged), fake_K, sub, seg, 1.0, bc, B.MRCM_FP64,
                          None) == -2
    flat = B._ints((8, 8, 1), 3)
    assert lib.mrcm_setup(ctypes.byref(ctx), ctypes.byref(g3), fake_K, sub, flat, 1.0, bc, B.MRCM_FP64,
                          None) == -2
    assert not ctx.value
    g2 = B.mrcm_grid(2, (ctypes.c_int * 3)(64, 64, 1), (ctypes.c_double * 3)(1.0, 1.0, 1.0))
    assert lib.mrcm_setup(ctypes.byref(ctx), ctypes.byref(g2), fake_K, sub, seg, 1.0, bc, B.MRCM_SURROGATE,
                          None) == -9
    assert lib.mrcm_setup(ctypes.byref(ctx), ctypes.byref(g2), fake_K, sub, seg, 1.0, bc, 7, None) == -1
    assert not ctx.value


def test_plan_of_the_3d_box_workload(mrcm_lib):
    # 256 x 256 x 64 cells, 16^3 subdomains, 4 x 4 patches: 64 x 64 x 16
    # blocks of 4^3 cells; a face between blocks of one subdomain is one
    # segment, the side between blocks of two subdomains one patch; the
    # bisection tree has log2(65536) = 16 levels
    Nb, Ns = (64, 64, 16), (16, 16, 4)
    segs = 0
    for d in range(3):
        others = Nb[0] * Nb[1] * Nb[2] // Nb[d]
        patch_sides = (Ns[d] - 1) * others
        fine_sides = (Nb[d] - 1) * others - patch_sides
        segs += patch_sides + 16 * fine_sides
    q = lambda what: mrcm_lib.mrcm_plan_query((256, 256, 64), (1.0, 1.0, 0.25), (16, 16, 16), (4, 4, 4),
                                               (1, 1, 0, 0, 0, 0), what)
    assert q("LEAVES") == 64 * 64 * 16
    assert q("SEGMENTS") == segs
    assert q("LEVELS") == 16
    assert q("NODES") == 2 * 64 * 64 * 16 - 1
    assert q("CELLS") == 256 * 256 * 64
