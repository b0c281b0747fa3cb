"""O2: the non-recursive MRCM with a global interface system (parity target).

Follows Section 3 of the paper step by step:
  1. for every leaf, the MMBFs of Eqs. (11Hhatbasisa)/(11Hhatbasisb) -- one
     local solve with U_H = phi^j and one with P_H = psi^j per interface
     segment j of the leaf -- plus the particular solution (Eqs. addu/addp);
  2. the global interface system A X = b of Eq. (linsys) with the entries of
     Eq. (brhs): rows tested with phi^r come from Eq. (14.2), rows tested
     with psi^r from Eq. (13.2); unknowns X = (U_1..U_n, P_1..P_n);
  3. the final local solutions of Eq. (final) as linear combinations of the
     MMBFs with the coefficients X.

Reading for the pure-Neumann case (every side no-flow): the system then has
the constant null vector (P += c); the Eq. (13.2) row of the first segment is
replaced by P_1 = 0 and the pressure (cell values and P) is shifted
afterwards to zero area-weighted mean.

Returned arrays: p (ny, nx); Fx (ny, nx+1), Fy (ny+1, nx) integrated face
fluxes in the +axis direction, on skeleton faces the mean of the two
one-sided values; Fa_x, Fb_x, Fa_y, Fb_y the one-sided values (side a =
lower leaf, side b = upper leaf) in the +axis direction, equal to F off the
skeleton; U, P per segment; the leaf Robin-to-flux data (R, rbar).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .geometry import Decomposition
from .local import LeafProblem


def mmbf_traces(lp, dec):
    """Step 1 for one leaf: the segment flux traces of the 2m MMBFs (U-type
    columns first, then P-type) and of the particular solution."""
    m = len(lp.segs)
    lam = np.zeros((m, 2 * m))
    for k, t in enumerate(lp.segs):
        seg = dec.segments[t]
        lam[k, k] = -seg["beta"] * dec.side(t, lp.leaf["id"])   # U_H = phi^t
        lam[k, m + k] = 1.0                                      # P_H = psi^t
    _, traces, _ = lp.solve(lam, with_data=False)
    _, part, _ = lp.solve(np.zeros(m), with_data=True)
    return lam, traces, part


def solve_mrcm(prob, return_leaf_ops=False):
    dec = Decomposition(prob)
    nseg = len(dec.segments)
    leaves = [LeafProblem(dec, lf["id"]) for lf in dec.leaves]
    rows, cols, vals = [], [], []
    b = np.zeros(2 * nseg)
    for lp in leaves:
        i = lp.leaf["id"]
        m = len(lp.segs)
        _, traces, part = mmbf_traces(lp, dec)
        for kr, r in enumerate(lp.segs):
            s_ir = dec.side(r, i)
            beta_r = dec.segments[r]["beta"]
            length_r = dec.segments[r]["length"]
            for kj, j in enumerate(lp.segs):
                for typ in (0, 1):                # 0: U_j column, 1: P_j column
                    F = traces[kr, typ * m + kj]
                    col = j + typ * nseg
                    # Eq. (brhs), first case: (beta (Phi.n^i - varphi^j n^i.n), phi^r n^i.n)
                    phi_term = length_r * s_ir if (typ == 0 and j == r) else 0.0
                    rows.append(r); cols.append(col)
                    vals.append(beta_r * (F - phi_term) * s_ir)
                    # Eq. (brhs), second case: (Phi.n^i, psi^r)
                    rows.append(nseg + r); cols.append(col); vals.append(F)
            b[r] -= beta_r * part[kr] * s_ir
            b[nseg + r] -= part[kr]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(2 * nseg, 2 * nseg))
    if prob.pure_neumann and nseg > 0:
        A = A.tolil()
        A[nseg, :] = 0.0
        A[nseg, nseg] = 1.0
        A = A.tocsr()
        b[nseg] = 0.0
    X = spla.spsolve(A.tocsc(), b) if nseg > 0 else np.zeros(0)
    U, P = X[:nseg], X[nseg:]
    out = assemble_final(prob, dec, leaves, U, P)
    if return_leaf_ops:
        out["leaf_ops"] = [lp.robin_to_flux() for lp in leaves]
        out["leaf_segs"] = [lp.segs for lp in leaves]
    out["dec"] = dec
    return out


def assemble_final(prob, dec, leaves, U, P):
    """Eq. (final): u^i = sum_j X_j Phi^i_j + ubar^i, p^i likewise, then the
    pure-Neumann mean shift."""
    nx, ny = prob.nx, prob.ny
    p = np.zeros((ny, nx))
    Fa_x = np.zeros((ny, nx + 1)); Fb_x = np.zeros((ny, nx + 1))
    Fa_y = np.zeros((ny + 1, nx)); Fb_y = np.zeros((ny + 1, nx))
    nseg = len(dec.segments)
    for lp in leaves:
        i = lp.leaf["id"]
        m = len(lp.segs)
        lam = np.zeros((m, 2 * m + 1))
        coef = np.zeros(2 * m + 1)
        for k, t in enumerate(lp.segs):
            lam[k, k] = -dec.segments[t]["beta"] * dec.side(t, i)
            lam[k, m + k] = 1.0
            coef[k] = U[t]
            coef[m + k] = P[t]
        coef[2 * m] = 1.0
        # columns: 2m MMBFs (homogeneous) and, last, the particular solution
        ph, _, fh = lp.solve(lam[:, :2 * m], with_data=False)
        pp, _, fp = lp.solve(np.zeros(m), with_data=True)
        pl = ph @ coef[:2 * m] + pp
        p[lp.j0:lp.j1, lp.i0:lp.i1] = pl.reshape(lp.h, lp.w)
        for key, fv in fh.items():
            val = fv @ coef[:2 * m] + fp[key]
            d, jj, ii = key
            kind = lp.faces[key][0]
            if d == "x":
                lower_side = ii > lp.i0        # the leaf is the lower cell's side
                tgt_a, tgt_b = Fa_x, Fb_x
            else:
                lower_side = jj > lp.j0
                tgt_a, tgt_b = Fa_y, Fb_y
            if kind == "robin":
                (tgt_a if lower_side else tgt_b)[jj, ii] = val
            else:
                tgt_a[jj, ii] = val
                tgt_b[jj, ii] = val
    if prob.pure_neumann:
        cell_area = prob.hx * prob.hy
        shift = (p * cell_area).sum() / (cell_area * nx * ny)
        p -= shift
        P = P - shift
    Fx = 0.5 * (Fa_x + Fb_x)
    Fy = 0.5 * (Fa_y + Fb_y)
    return dict(p=p, Fx=Fx, Fy=Fy, Fa_x=Fa_x, Fb_x=Fb_x, Fa_y=Fa_y, Fb_y=Fb_y,
                U=U, P=P)
