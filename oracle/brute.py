"""Monolithic dense solve of the MRCM equations on tiny grids.

Assembles Eqs. (11.2), (12.2), (13.2) and (14.2) directly -- no MMBFs, no
Robin-to-flux maps, no recursion -- and solves them with one dense solve, so
that it pins the basis/Schur algebra of oracle.mrcm and oracle.recursive
without sharing their steps.  Lumped RT0 (see oracle.fine).

Unknowns: every leaf's cell pressures, the outward flux F^i_e of every
skeleton face e seen from each of its two leaves, and (U_t, P_t) per
segment.  Equations:
  Eq. (12.2), per cell: sum of its outward fluxes = q_c, interior faces by
      two-point fluxes, skeleton faces by the unknown F^i_e, boundary faces
      by the Dirichlet / Neumann data;
  Eq. (11.2) tested with the RT0 basis function of a skeleton face, lumped:
      (h_d / (2 K_c)) F_e/|e| - p_c + P_t - beta_t U_t (n_t.n^i)
      + beta_t F_e/|e| = 0;
  Eq. (13.2), per segment: sum over both sides of F^i_e = 0;
  Eq. (14.2), per segment: sum over both sides of
      beta_t (F^i_e - U_t |e| (n_t.n^i)) (n_t.n^i) = 0.
Pure Neumann: the Eq. (13.2) row of the first segment becomes P_1 = 0, then
the pressure is shifted to zero mean.
"""
import numpy as np

from inputs.problems import DIRICHLET
from .geometry import Decomposition


def solve_brute(prob):
    dec = Decomposition(prob)
    nx, ny, hx, hy, K = prob.nx, prob.ny, prob.hx, prob.hy, prob.K
    ncell = nx * ny
    cell = lambda i, j: i + nx * j
    leaf_of = np.zeros((ny, nx), dtype=np.int64)
    for lf in dec.leaves:
        leaf_of[lf["j0"]:lf["j1"], lf["i0"]:lf["i1"]] = lf["id"]
    # skeleton face unknowns: (segment, face index within segment, side)
    fidx = {}
    for t in dec.segments:
        for k, (ca, cb) in enumerate(dec.face_cells(t)):
            fidx[(t["id"], k, 0)] = ncell + len(fidx)
            fidx[(t["id"], k, 1)] = ncell + len(fidx)
    nseg = len(dec.segments)
    iU = lambda t: ncell + len(fidx) + t
    iP = lambda t: ncell + len(fidx) + nseg + t
    N = ncell + len(fidx) + 2 * nseg
    A = np.zeros((N, N))
    b = np.zeros(N)
    bcs = prob.bc_slices()
    # Eq. (12.2): cell balances
    for j in range(ny):
        for i in range(nx):
            c = cell(i, j)
            b[c] += prob.q[j, i]
            for (ni, nj, axis, outsign) in [(i - 1, j, 0, -1), (i + 1, j, 0, 1),
                                            (i, j - 1, 1, -1), (i, j + 1, 1, 1)]:
                hn, area = (hx, hy) if axis == 0 else (hy, hx)
                if 0 <= ni < nx and 0 <= nj < ny:
                    if leaf_of[nj, ni] == leaf_of[j, i]:
                        T = area / (hn / (2 * K[j, i]) + hn / (2 * K[nj, ni]))
                        A[c, c] += T
                        A[c, cell(ni, nj)] -= T
                    else:
                        # skeleton face: its own flux unknown
                        if axis == 0:
                            fi = i if outsign < 0 else i + 1
                            t = dec.xface_seg[j, fi]
                            k = j - dec.segments[t]["lo"]
                        else:
                            fj = j if outsign < 0 else j + 1
                            t = dec.yface_seg[fj, i]
                            k = i - dec.segments[t]["lo"]
                        side = 0 if outsign > 0 else 1      # +axis outward => side a
                        A[c, fidx[(t, k, side)]] += 1.0
                else:
                    s = (0 if outsign < 0 else 1) if axis == 0 else (2 if outsign < 0 else 3)
                    kk = j if axis == 0 else i
                    gval = prob.bc_val[bcs[s]][kk]
                    if prob.bc_type[s] == DIRICHLET:
                        tau = 2.0 * K[j, i] * area / hn
                        A[c, c] += tau
                        b[c] += tau * gval
                    else:
                        b[c] -= area * gval
    row = ncell
    # Eq. (11.2) on skeleton faces
    for t in dec.segments:
        hn, area = (hx, hy) if t["axis"] == 0 else (hy, hx)
        beta = t["beta"]
        for k, (ca, cb) in enumerate(dec.face_cells(t)):
            for side, (jj, ii) in enumerate((ca, cb)):
                s_in = 1.0 if side == 0 else -1.0
                f = fidx[(t["id"], k, side)]
                A[row, f] = hn / (2 * K[jj, ii]) / area + beta / area
                A[row, cell(ii, jj)] = -1.0
                A[row, iP(t["id"])] = 1.0
                A[row, iU(t["id"])] = -beta * s_in
                row += 1
    # Eq. (13.2) and Eq. (14.2) per segment
    for t in dec.segments:
        nf = t["hi"] - t["lo"]
        area = hy if t["axis"] == 0 else hx
        r13 = row; r14 = row + 1
        for k in range(nf):
            for side in (0, 1):
                s_in = 1.0 if side == 0 else -1.0
                A[r13, fidx[(t["id"], k, side)]] += 1.0
                A[r14, fidx[(t["id"], k, side)]] += t["beta"] * s_in
                A[r14, iU(t["id"])] -= t["beta"] * area * s_in * s_in
        row += 2
    assert row == N
    if prob.pure_neumann and nseg > 0:
        r13 = ncell + len(fidx)
        A[r13, :] = 0.0
        A[r13, iP(0)] = 1.0
        b[r13] = 0.0
    x = np.linalg.solve(A, b)
    p = x[:ncell].reshape(ny, nx)
    if prob.pure_neumann:
        p = p - p.mean()
    return dict(p=p, x=x, fidx=fidx, dec=dec)
