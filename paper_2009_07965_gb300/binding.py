"""ctypes binding of libmrcm (include/mrcm.h): argument marshalling only.

The functions below carry the C names and pass plain pointers and sizes
through; device buffers are torch CUDA tensors (float64, contiguous).  The
library must have been built (paper_2009_07965_gb300.build.build()); there
is no fallback path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrcm.so")

MRCM_BC_NEUMANN, MRCM_BC_DIRICHLET = 0, 1
MRCM_FP64, MRCM_MIXED, MRCM_SURROGATE = 0, 1, 2
MRCM_ROOT_FACTOR, MRCM_ROOT_INVERSE, MRCM_ROOT_AUTO = 0, 1, 2
ERRORS = {0: "MRCM_OK", -1: "MRCM_ERR_INVALID_ARG", -2: "MRCM_ERR_SHAPE", -3: "MRCM_ERR_BAD_K",
          -4: "MRCM_ERR_NOT_BUILT", -5: "MRCM_ERR_SINGULAR", -6: "MRCM_ERR_CUDA",
          -7: "MRCM_ERR_OOM", -8: "MRCM_ERR_TIMEOUT", -9: "MRCM_ERR_UNSUPPORTED"}
Q = dict(LEAVES=0, SEGMENTS=1, LEVELS=2, NODES=3, WORKSPACE_BYTES=4, MAX_GAMMA=5,
         BUILD_FLOPS=6, SOLVE_FLOPS=7, LEAF_FLOPS=8, KERNEL_LAUNCHES_BUILD=9,
         KERNEL_LAUNCHES_SOLVE=10, GRAPH_REPLAYS=11, MODEL_BUILD_FLOPS=12, MODEL_SWEEP_FLOPS=13,
         GRIDS=14, CELLS=15)

# every symbol include/mrcm.h declares
EXPORTS = ["mrcm_setup", "mrcm_setup_batch", "mrcm_plan_query", "mrcm_set_permeability", "mrcm_build_basis", "mrcm_solve", "mrcm_query",
           "mrcm_node_info", "mrcm_node_segments", "mrcm_segment_info", "mrcm_node_operator",
           "mrcm_destroy", "mrcm_error_string", "mrcm_enable_timing", "mrcm_phase_times", "mrcm_use_graphs",
           "mrcm_last_cuda_error",
           "mrcm_merge_pair_noalloc", "mrcm_set_refinement", "mrcm_set_residual", "mrcm_residual_history",
           "mrcm_phase_flops", "mrcm_group_times", "mrcm_check_reciprocal", "mrcm_set_wait_limit",
           "mrcm_probe_peak", "mrcm_set_mixed_split", "mrcm_set_mixed_leaves", "mrcm_set_root_form", "mrcm_autotune", "mrcm_tune_info",
           "mrcm_interior_leaves", "mrcm_leaf_fields", "mrcm_leaf_patches", "mrcm_leaf_gate", "mrcm_leaf_apply",
           "mrcm_cnn_conv_forward", "mrcm_cnn_conv_wgrad", "mrcm_cnn_flip_weights", "mrcm_cnn_relu_grad",
           "mrcm_cnn_mse_grad", "mrcm_cnn_adam"]
PHASES = ["coef", "leaf_build", "merge_small", "gj_sweep", "merge_form", "merge_x", "merge_r",
          "leaf_particular", "tree_up", "tree_down", "leaf_pressure", "residual", "finish", "root_factor"]
# kernel family behind each phase (for reports)
PHASE_KERNELS = {"coef": "face_coef_kernel", "leaf_build": "leaf_build_kernel",
                 "merge_small": "merge_small_kernel", "gj_sweep": "gj_sweep_kernel",
                 "merge_form": "gj_sweep_kernel (form and back-form folded in)", "merge_x": "merge_x_kernel",
                 "merge_r": "merge_rupdate_kernel", "leaf_particular": "leaf_particular_kernel",
                 "tree_up": "tree_up_kernel", "tree_down": "tree_down_kernel",
                 "leaf_pressure": "leaf_pressure_kernel", "residual": "residual_cells/segments_kernel",
                 "finish": "face_flux_kernel", "root_factor": "ldl_sweep_kernel"}


class MrcmError(RuntimeError):
    def __init__(self, code, call):
        self.code = code
        msg = f"{call} failed: {ERRORS.get(code, code)} ({_lib().mrcm_error_string(code).decode()})"
        self.cuda_error = None
        if code in (-6, -7):                 # MRCM_ERR_CUDA, MRCM_ERR_OOM
            self.cuda_error = mrcm_last_cuda_error()
            msg += f" [{self.cuda_error[1]}]"
        super().__init__(msg)


class mrcm_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2009_07965_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        IP = ctypes.POINTER(ctypes.c_int)
        lib.mrcm_setup.argtypes = [ctypes.POINTER(P), ctypes.POINTER(mrcm_grid), P, IP, IP, D, IP, I, P]
        lib.mrcm_setup.restype = I
        lib.mrcm_setup_batch.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(mrcm_grid), IP, P, IP, IP, D, I, P]
        lib.mrcm_setup_batch.restype = I
        lib.mrcm_plan_query.argtypes = [ctypes.POINTER(mrcm_grid), IP, IP, IP, I,
                                        ctypes.POINTER(ctypes.c_longlong)]
        lib.mrcm_plan_query.restype = I
        lib.mrcm_set_permeability.argtypes = [P, P]
        lib.mrcm_set_permeability.restype = I
        lib.mrcm_build_basis.argtypes = [P]
        lib.mrcm_build_basis.restype = I
        lib.mrcm_solve.argtypes = [P, P, P, P, P, P, P, P]
        lib.mrcm_solve.restype = I
        lib.mrcm_query.argtypes = [P, I, ctypes.POINTER(ctypes.c_longlong)]
        lib.mrcm_query.restype = I
        lib.mrcm_node_info.argtypes = [P, I, IP]
        lib.mrcm_node_info.restype = I
        lib.mrcm_node_segments.argtypes = [P, I, IP]
        lib.mrcm_node_segments.restype = I
        lib.mrcm_segment_info.argtypes = [P, I, IP]
        lib.mrcm_segment_info.restype = I
        lib.mrcm_node_operator.argtypes = [P, I, P, P]
        lib.mrcm_node_operator.restype = I
        lib.mrcm_enable_timing.argtypes = [P, I]
        lib.mrcm_enable_timing.restype = I
        lib.mrcm_use_graphs.argtypes = [P, I]
        lib.mrcm_use_graphs.restype = I
        lib.mrcm_phase_times.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
        lib.mrcm_phase_times.restype = I
        lib.mrcm_merge_pair_noalloc.argtypes = [P, I, P, I, P, I, P, P, P, P]
        lib.mrcm_merge_pair_noalloc.restype = I
        lib.mrcm_phase_flops.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
        lib.mrcm_phase_flops.restype = I
        lib.mrcm_group_times.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), I]
        lib.mrcm_group_times.restype = I
        lib.mrcm_check_reciprocal.argtypes = [P, P, ctypes.c_longlong, P]
        lib.mrcm_check_reciprocal.restype = I
        lib.mrcm_set_refinement.argtypes = [P, I, I]
        lib.mrcm_set_refinement.restype = I
        lib.mrcm_set_residual.argtypes = [P, I]
        lib.mrcm_set_residual.restype = I
        LL, F = ctypes.c_longlong, ctypes.c_float
        lib.mrcm_interior_leaves.argtypes = [P, IP, I]
        lib.mrcm_interior_leaves.restype = I
        lib.mrcm_leaf_fields.argtypes = [P, P, I, P]
        lib.mrcm_leaf_fields.restype = I
        lib.mrcm_leaf_patches.argtypes = [P, P, I, P]
        lib.mrcm_leaf_patches.restype = I
        lib.mrcm_leaf_gate.argtypes = [P, P, I, P, P]
        lib.mrcm_leaf_gate.restype = I
        lib.mrcm_leaf_apply.argtypes = [P, P, I, P, P, D, P]
        lib.mrcm_leaf_apply.restype = I
        lib.mrcm_cnn_conv_forward.argtypes = [P, I, I, I, I, I, P, P, P, P, P]
        lib.mrcm_cnn_conv_forward.restype = I
        lib.mrcm_cnn_conv_wgrad.argtypes = [P, P, I, I, I, I, P, P, P]
        lib.mrcm_cnn_conv_wgrad.restype = I
        lib.mrcm_cnn_flip_weights.argtypes = [P, I, I, P, P]
        lib.mrcm_cnn_flip_weights.restype = I
        lib.mrcm_cnn_relu_grad.argtypes = [P, P, LL, I, P, P]
        lib.mrcm_cnn_relu_grad.restype = I
        lib.mrcm_cnn_mse_grad.argtypes = [P, P, I, P, P, P]
        lib.mrcm_cnn_mse_grad.restype = I
        lib.mrcm_cnn_adam.argtypes = [P, P, P, P, P, LL, F, F, F, F, I, P]
        lib.mrcm_cnn_adam.restype = I
        lib.mrcm_autotune.argtypes = [P, I]
        lib.mrcm_autotune.restype = I
        lib.mrcm_tune_info.argtypes = [P, I, IP]
        lib.mrcm_tune_info.restype = I
        lib.mrcm_set_mixed_split.argtypes = [P, I]
        lib.mrcm_set_mixed_split.restype = I
        lib.mrcm_set_root_form.argtypes = [P, I]
        lib.mrcm_set_root_form.restype = I
        lib.mrcm_set_mixed_leaves.argtypes = [P, I]
        lib.mrcm_set_mixed_leaves.restype = I
        lib.mrcm_probe_peak.argtypes = [I, D, ctypes.POINTER(ctypes.c_double), P]
        lib.mrcm_probe_peak.restype = I
        lib.mrcm_set_wait_limit.argtypes = [P, ctypes.c_longlong]
        lib.mrcm_set_wait_limit.restype = I
        lib.mrcm_residual_history.argtypes = [P, ctypes.POINTER(ctypes.c_double), I]
        lib.mrcm_residual_history.restype = I
        lib.mrcm_destroy.argtypes = [P]
        lib.mrcm_destroy.restype = None
        lib.mrcm_error_string.argtypes = [I]
        lib.mrcm_error_string.restype = ctypes.c_char_p
        lib.mrcm_last_cuda_error.argtypes = [ctypes.c_char_p, I]
        lib.mrcm_last_cuda_error.restype = I
        _LIB = lib
    return _LIB


def _check(code, call):
    if code != 0:
        raise MrcmError(code, call)


def _ptr(t):
    """Device (or host) address of a tensor / array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    return int(t)


def _ints(vals, n):
    vals = list(vals) + [0] * (n - len(vals))
    return (ctypes.c_int * n)(*vals)


def mrcm_setup(n, L, K, sub_cells=(16, 16), seg_cells=(4, 4), alpha=1.0,
               bc_type=(1, 1, 0, 0), precision=MRCM_FP64, stream=0):
    """n = (nx, ny) or (nx, ny, nz) cells, L the physical size per axis."""
    dim = len(n)
    g = mrcm_grid(dim, (ctypes.c_int * 3)(n[0], n[1], n[2] if dim == 3 else 1),
                  (ctypes.c_double * 3)(L[0], L[1], L[2] if dim == 3 else 1.0))
    ctx = ctypes.c_void_p()
    _check(_lib().mrcm_setup(ctypes.byref(ctx), ctypes.byref(g), _ptr(K), _ints(sub_cells, 3),
                             _ints(seg_cells, 3), float(alpha), _ints(bc_type, 6), int(precision),
                             stream), "mrcm_setup")
    return ctx


def mrcm_setup_batch(ns, Ls, bc_types, K, sub_cells=(16, 16), seg_cells=(4, 4), alpha=1.0,
                     precision=MRCM_FP64, stream=0):
    """One context for several problems: ns[k] = (nx, ny), Ls[k] = (Lx, Ly),
    bc_types[k] = (x-, x+, y-, y+); K holds their permeabilities
    concatenated in problem order."""
    count = len(ns)
    grids = (mrcm_grid * count)()
    for k, (n, L) in enumerate(zip(ns, Ls)):
        grids[k] = mrcm_grid(2, (ctypes.c_int * 3)(n[0], n[1], 1), (ctypes.c_double * 3)(L[0], L[1], 1.0))
    bcs = []
    for b in bc_types:
        bcs += list(b) + [0] * (6 - len(b))
    ctx = ctypes.c_void_p()
    _check(_lib().mrcm_setup_batch(ctypes.byref(ctx), count, grids, _ints(bcs, 6 * count), _ptr(K),
                                   _ints(sub_cells, 3), _ints(seg_cells, 3), float(alpha), int(precision),
                                   stream), "mrcm_setup_batch")
    return ctx


def mrcm_plan_query(n, L, sub_cells, seg_cells, bc_type, what):
    dim = len(n)
    g = mrcm_grid(dim, (ctypes.c_int * 3)(n[0], n[1], n[2] if dim == 3 else 1),
                  (ctypes.c_double * 3)(L[0], L[1], L[2] if dim == 3 else 1.0))
    v = ctypes.c_longlong()
    key = Q[what] if isinstance(what, str) else int(what)
    _check(_lib().mrcm_plan_query(ctypes.byref(g), _ints(sub_cells, 3), _ints(seg_cells, 3),
                                  _ints(bc_type, 6), key, ctypes.byref(v)), "mrcm_plan_query")
    return v.value


def mrcm_set_permeability(ctx, K):
    _check(_lib().mrcm_set_permeability(ctx, _ptr(K)), "mrcm_set_permeability")


def mrcm_build_basis(ctx):
    _check(_lib().mrcm_build_basis(ctx), "mrcm_build_basis")


def mrcm_solve(ctx, q, bc_val, p, Fx, Fy, Fz=None, iface=None):
    _check(_lib().mrcm_solve(ctx, _ptr(q), _ptr(bc_val), _ptr(p), _ptr(Fx), _ptr(Fy), _ptr(Fz),
                             _ptr(iface)), "mrcm_solve")


def mrcm_query(ctx, what):
    v = ctypes.c_longlong()
    key = Q[what] if isinstance(what, str) else int(what)
    _check(_lib().mrcm_query(ctx, key, ctypes.byref(v)), "mrcm_query")
    return v.value


def mrcm_node_info(ctx, node):
    info = (ctypes.c_int * 11)()
    _check(_lib().mrcm_node_info(ctx, node, info), "mrcm_node_info")
    keys = ["height", "m", "g", "c1", "c2", "parent", "leaf", "I0", "I1", "J0", "J1"]
    return dict(zip(keys, list(info)))


def mrcm_node_segments(ctx, node):
    m = mrcm_node_info(ctx, node)["m"]
    buf = (ctypes.c_int * max(m, 1))()
    _check(_lib().mrcm_node_segments(ctx, node, buf), "mrcm_node_segments")
    return list(buf)[:m]


def mrcm_segment_info(ctx, seg):
    info = (ctypes.c_int * 6)()
    _check(_lib().mrcm_segment_info(ctx, seg, info), "mrcm_segment_info")
    return dict(zip(["axis", "line", "lo", "len", "a", "b"], list(info)))


def mrcm_node_operator(ctx, node, with_rbar=False):
    import numpy as np
    m = mrcm_node_info(ctx, node)["m"]
    R = np.zeros((m, m))
    rbar = np.zeros(m) if with_rbar else None
    _check(_lib().mrcm_node_operator(ctx, node, R.ctypes.data if m else R.ctypes.data,
                                     rbar.ctypes.data if with_rbar else None), "mrcm_node_operator")
    return (R, rbar) if with_rbar else R


def mrcm_enable_timing(ctx, on=True):
    _check(_lib().mrcm_enable_timing(ctx, 1 if on else 0), "mrcm_enable_timing")


def mrcm_last_cuda_error():
    """(cudaError_t code, name) behind the last CUDA failure on this thread."""
    buf = ctypes.create_string_buffer(64)
    code = _lib().mrcm_last_cuda_error(buf, 64)
    return code, buf.value.decode()


def mrcm_use_graphs(ctx, on=True):
    _check(_lib().mrcm_use_graphs(ctx, 1 if on else 0), "mrcm_use_graphs")


def mrcm_phase_times(ctx):
    ms = (ctypes.c_double * len(PHASES))()
    _check(_lib().mrcm_phase_times(ctx, ms), "mrcm_phase_times")
    return dict(zip(PHASES, list(ms)))


def mrcm_group_times(ctx, cap=4096):
    """[(phase name, ms)] of the timed launch groups of the last build and solve."""
    ph = (ctypes.c_int * cap)()
    ms = (ctypes.c_double * cap)()
    n = _lib().mrcm_group_times(ctx, ph, ms, cap)
    _check(min(n, 0), "mrcm_group_times")
    return [(PHASES[ph[k]], ms[k]) for k in range(min(n, cap))]


def mrcm_check_reciprocal(x, out=None):
    """The kernels' reciprocal of every entry of a float64 CUDA tensor."""
    import torch
    x = x.contiguous()
    out = torch.empty_like(x) if out is None else out
    stream = torch.cuda.current_stream(x.device).cuda_stream
    _check(_lib().mrcm_check_reciprocal(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        x.numel(), ctypes.c_void_p(stream)), "mrcm_check_reciprocal")
    return out


def mrcm_set_refinement(ctx, steps, check=False):
    _check(_lib().mrcm_set_refinement(ctx, int(steps), 1 if check else 0), "mrcm_set_refinement")


def mrcm_set_residual(ctx, dd):
    """Refinement residuals in double-double (1; FP64 form default) or FP64 (0; mixed form default)."""
    _check(_lib().mrcm_set_residual(ctx, 1 if dd else 0), "mrcm_set_residual")


PROBES = dict(DFMA=0, DMMA=1, FFMA=2, TF32=3, BF16=4, DFMA_DMMA=5)


def mrcm_probe_peak(kind, seconds=0.3, stream=None):
    """Measured TFLOP/s of one arithmetic pipe (kind: a PROBES key)."""
    out = ctypes.c_double()
    _check(_lib().mrcm_probe_peak(PROBES[kind] if isinstance(kind, str) else int(kind), float(seconds),
                                  ctypes.byref(out), stream), "mrcm_probe_peak")
    return out.value


def mrcm_interior_leaves(ctx):
    """Ids of the full interior leaves (host list)."""
    n = _lib().mrcm_interior_leaves(ctx, None, 0)
    _check(min(n, 0), "mrcm_interior_leaves")
    buf = (ctypes.c_int * max(n, 1))()
    _lib().mrcm_interior_leaves(ctx, buf, n)
    return list(buf)[:n]


def mrcm_leaf_fields(ctx, ids, psi):
    _check(_lib().mrcm_leaf_fields(ctx, _ptr(ids), int(ids.numel()), _ptr(psi)), "mrcm_leaf_fields")


def mrcm_leaf_patches(ctx, ids, x):
    _check(_lib().mrcm_leaf_patches(ctx, _ptr(ids), int(ids.numel()), _ptr(x)), "mrcm_leaf_patches")


def mrcm_leaf_gate(ctx, ids, psi, res):
    _check(_lib().mrcm_leaf_gate(ctx, _ptr(ids), int(ids.numel()), _ptr(psi), _ptr(res)), "mrcm_leaf_gate")


def mrcm_leaf_apply(ctx, ids, psi, res, tau, accepted):
    _check(_lib().mrcm_leaf_apply(ctx, _ptr(ids), int(ids.numel()), _ptr(psi), _ptr(res), float(tau),
                                  _ptr(accepted)), "mrcm_leaf_apply")


def mrcm_cnn_conv_forward(x, count, cin, cout, pad, relu, w, b, y_bf16=None, y_f32=None, stream=None):
    _check(_lib().mrcm_cnn_conv_forward(_ptr(x), int(count), cin, cout, pad, 1 if relu else 0, _ptr(w), _ptr(b),
                                        _ptr(y_bf16), _ptr(y_f32), stream), "mrcm_cnn_conv_forward")


def mrcm_cnn_conv_wgrad(x, dy, count, cin, cout, pad, dw, db=None, stream=None):
    _check(_lib().mrcm_cnn_conv_wgrad(_ptr(x), _ptr(dy), int(count), cin, cout, pad, _ptr(dw), _ptr(db), stream),
           "mrcm_cnn_conv_wgrad")


def mrcm_cnn_flip_weights(w, cout, cin, w2, stream=None):
    _check(_lib().mrcm_cnn_flip_weights(_ptr(w), cout, cin, _ptr(w2), stream), "mrcm_cnn_flip_weights")


def mrcm_cnn_relu_grad(dpost, y, n, mask, dpre, stream=None):
    _check(_lib().mrcm_cnn_relu_grad(_ptr(dpost), _ptr(y), int(n), 1 if mask else 0, _ptr(dpre), stream),
           "mrcm_cnn_relu_grad")


def mrcm_cnn_mse_grad(pred, target, count, dpred, loss, stream=None):
    _check(_lib().mrcm_cnn_mse_grad(_ptr(pred), _ptr(target), int(count), _ptr(dpred), _ptr(loss), stream),
           "mrcm_cnn_mse_grad")


def mrcm_cnn_adam(p, g, m1, m2, p_bf16, n, lr, beta1, beta2, eps, step, stream=None):
    _check(_lib().mrcm_cnn_adam(_ptr(p), _ptr(g), _ptr(m1), _ptr(m2), _ptr(p_bf16), int(n), float(lr), float(beta1),
                                float(beta2), float(eps), int(step), stream), "mrcm_cnn_adam")


def mrcm_autotune(ctx, reps=3):
    _check(_lib().mrcm_autotune(ctx, int(reps)), "mrcm_autotune")


def mrcm_tune_info(ctx, height):
    out = (ctypes.c_int * 3)()
    _check(_lib().mrcm_tune_info(ctx, int(height), out), "mrcm_tune_info")
    return dict(sweep_per_sm=out[0], x_rows=out[1], r_tile=out[2])


def mrcm_set_mixed_split(ctx, max_g2_fp32):
    _check(_lib().mrcm_set_mixed_split(ctx, int(max_g2_fp32)), "mrcm_set_mixed_split")


def mrcm_set_mixed_leaves(ctx, fp32):
    """Mixed form: leaf factors in FP32 (1) or FP64 (0, default); the basis must be rebuilt."""
    _check(_lib().mrcm_set_mixed_leaves(ctx, int(fp32)), "mrcm_set_mixed_leaves")


def mrcm_set_root_form(ctx, form):
    """MRCM_ROOT_FACTOR (0), MRCM_ROOT_INVERSE (1) or MRCM_ROOT_AUTO (2, default); the basis must be rebuilt."""
    _check(_lib().mrcm_set_root_form(ctx, int(form)), "mrcm_set_root_form")


def mrcm_set_wait_limit(ctx, polls):
    _check(_lib().mrcm_set_wait_limit(ctx, int(polls)), "mrcm_set_wait_limit")


def mrcm_residual_history(ctx, cap=17):
    buf = (ctypes.c_double * cap)()
    n = _lib().mrcm_residual_history(ctx, buf, cap)
    if n < 0:
        raise MrcmError(n, "mrcm_residual_history")
    return list(buf)[:min(n, cap)]


def mrcm_phase_flops(ctx):
    f = (ctypes.c_double * len(PHASES))()
    _check(_lib().mrcm_phase_flops(ctx, f), "mrcm_phase_flops")
    return dict(zip(PHASES, list(f)))


def mrcm_destroy(ctx):
    if ctx:
        _lib().mrcm_destroy(ctx)


def mrcm_error_string(code):
    return _lib().mrcm_error_string(code).decode()


def mrcm_merge_pair_noalloc(R1, m1, R2, m2, index_map, g, D, R_out, X_out, stream=0):
    """Allocation-free merge of two maps (device tensors in, device tensors out)."""
    _check(_lib().mrcm_merge_pair_noalloc(_ptr(R1), int(m1), _ptr(R2), int(m2), _ptr(index_map),
                                          int(g), _ptr(D), _ptr(R_out), _ptr(X_out), stream),
           "mrcm_merge_pair_noalloc")
