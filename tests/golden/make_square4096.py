#!/usr/bin/env python3
"""Writes the oracle's sampled solution of the 4096^2 quarter-five-spot
field (tests/golden/square4096_qfs_oracle.npz).

The field is the one of inputs.config_4096(): 4096 x 4096 cells, log-normal
K with sigma^2 = 3 and correlation length 0.02 (seed 5000), no-flow
boundary, +1 / -1 sources in opposite corner cells, 16 x 16 leaves, 4-cell
segments, alpha = 1.  The solution is computed by the oracle alone: the CPU
Recursive MRCM (oracle.recursive, Algorithm 1 with dense FP64 merges) with
its per-leaf work spread over a process pool, refined three times with
double-double residuals of Eqs. 11.2-14.2 (oracle.refine), then the
all-Neumann zero-mean shift.  The global sparse factorisation of the
non-recursive oracle does not fit this size in memory; the recursive oracle
agrees with it to 1e-10 on every size where both run (tests).

Stored (a seeded sample; the full arrays are ~0.7 GB): flat indices and
values of p, Fx, Fy and of the one-sided skeleton fluxes Fa_x, Fb_x, Fa_y,
Fb_y, the full arrays' L2 norms, the refinement history and a fingerprint of
K (sum, sum of squares, sum of log K, min, max) so that a reader can check
that its own generator produced the same field up to rounding.

Usage: python tests/golden/make_square4096.py [--n 4096] [--procs P] [--out PATH]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SAMPLES = dict(p=20000, Fx=20000, Fy=20000, Fa_x=10000, Fb_x=10000, Fa_y=10000, Fb_y=10000)


def sample_indices(n, out, rng):
    """Flat indices per output: uniform over the array, the corner cells and
    faces next to the sources, and for the one-sided fluxes skeleton faces
    only (elsewhere they equal the face flux)."""
    idx = {}
    ny, nx = out["p"].shape
    corners = np.array([0, nx - 1, (ny - 1) * nx, ny * nx - 1])
    idx["p"] = np.unique(np.concatenate([rng.choice(nx * ny, SAMPLES["p"], replace=False), corners]))
    for key in ("Fx", "Fy"):
        size = out[key].size
        idx[key] = np.unique(np.concatenate([rng.choice(size, SAMPLES[key], replace=False),
                                             np.arange(8), size - 1 - np.arange(8)]))
    # skeleton faces: x-faces at multiples of 16 (interior), y-faces likewise
    sx = np.arange(16, nx, 16)
    jx = rng.integers(0, ny, SAMPLES["Fa_x"])
    ix = rng.choice(sx, SAMPLES["Fa_x"])
    skel_x = np.unique(jx * (nx + 1) + ix)
    sy = np.arange(16, ny, 16)
    jy = rng.choice(sy, SAMPLES["Fa_y"])
    iy = rng.integers(0, nx, SAMPLES["Fa_y"])
    skel_y = np.unique(jy * nx + iy)
    idx["Fa_x"] = idx["Fb_x"] = skel_x
    idx["Fa_y"] = idx["Fb_y"] = skel_y
    return idx


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--procs", type=int, default=len(os.sched_getaffinity(0)))
    ap.add_argument("--refine", type=int, default=3)
    ap.add_argument("--out", default=os.path.join(HERE, "square4096_qfs_oracle.npz"))
    args = ap.parse_args()
    import inputs
    from oracle.recursive import RecursiveMRCM, leaf_worker_init

    t0 = time.time()
    prob = inputs.config_4096(args.n)
    print(f"field {args.n}^2 generated in {time.time() - t0:.1f} s", flush=True)
    ctx = mp.get_context("spawn")
    # one BLAS thread per worker (the workers' 256 x 256 factorisations are
    # many and small); the parent keeps its threads for the large merges
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    pool = ctx.Pool(args.procs, initializer=leaf_worker_init, initargs=(prob,))
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    with pool:
        def leaf_map(fn, items):
            return pool.map(fn, items, chunksize=64)
        t1 = time.time()
        rm = RecursiveMRCM(prob, leaf_map=leaf_map)
        print(f"basis built in {time.time() - t1:.1f} s", flush=True)
        t2 = time.time()
        out = rm.solve(refine=args.refine)
        print(f"solved and refined in {time.time() - t2:.1f} s; history {out['refine_history']}", flush=True)
    rng = np.random.default_rng(4096)
    idx = sample_indices(args.n, out, rng)
    K = prob.K
    data = dict(n=args.n, refine=args.refine, history=np.array(out["refine_history"]),
                K_fingerprint=np.array([K.sum(), (K * K).sum(), np.log(K).sum(), K.min(), K.max()]))
    for key, ii in idx.items():
        arr = out[key].reshape(-1)
        data[f"{key}_idx"] = ii.astype(np.int64)
        data[f"{key}_val"] = arr[ii]
        data[f"{key}_norm"] = np.linalg.norm(out[key])
    np.savez_compressed(args.out, **data)
    print(f"wrote {args.out} ({os.path.getsize(args.out) / 1e6:.2f} MB) in {time.time() - t0:.1f} s total")


if __name__ == "__main__":
    main()
