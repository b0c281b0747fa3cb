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

refine > 0: the discrete MRCM solution is the exact solution of Eqs.
(11.2)-(14.2); a direct FP64 solve reaches it only up to the conditioning of
the problem times the rounding unit, which for high-contrast permeability is
far from FP64 accuracy.  With refine = k the solution is improved k times by
iterative refinement (Wilkinson): the residual of those equations is
evaluated in double-double arithmetic (oracle.refine) and the correction is
computed by the same three steps with the residual as data.  The result is
then the discrete solution to about the rounding unit, whatever the
conditioning (as long as it is below 1/u), and fluxes are formed from the
refined (p, P, U) by the face relations of oracle.refine.

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


def mmbf_data(lp, dec):
    """Robin data of the 2m MMBFs of one leaf: U-type columns first
    (U_H = phi^t: lambda_t = -beta_t n_t.n^i), then P-type (lambda_t = 1)."""
    m = len(lp.segs)
    lam = np.zeros((m, 2 * m))
    for k, t in enumerate(lp.segs):
        lam[k, k] = -dec.segments[t]["beta"] * dec.side(t, lp.leaf["id"])
        lam[k, m + k] = 1.0
    return lam


def mmbf_traces(lp, dec):
    """Step 1 for one leaf: the segment flux traces of the 2m MMBFs and of
    the particular solution."""
    lam = mmbf_data(lp, dec)
    _, traces, _ = lp.solve(lam, with_data=False, want_faces=False)
    _, part, _ = lp.solve(np.zeros(len(lp.segs)), with_data=True, want_faces=False)
    return lam, traces, part


class GlobalMRCM:
    """Steps 1-3 for arbitrary data: source per cell, external boundary data
    on or off, and right-hand sides of the Eq. (13.2) / (14.2) rows."""

    def __init__(self, prob, dec=None, leaf_cls=None):
        # dec / leaf_cls: another decomposition and local problem with the
        # same interface (the 3D ones of oracle.mrcm3d); the assembly below
        # only sees segment lists
        self.prob = prob
        self.dec = dec = dec if dec is not None else Decomposition(prob)
        self.nseg = nseg = len(dec.segments)
        leaf_cls = leaf_cls or LeafProblem
        self.leaves = [leaf_cls(dec, lf["id"]) for lf in dec.leaves]
        self.lams, self.traces = [], []
        rows, cols, vals = [], [], []
        for lp in self.leaves:
            i = lp.leaf["id"]
            m = len(lp.segs)
            lam = mmbf_data(lp, dec)
            _, traces, _ = lp.solve(lam, with_data=False, want_faces=False)
            self.lams.append(lam)
            self.traces.append(traces)
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
        A = sp.csr_matrix((vals, (rows, cols)), shape=(2 * nseg, 2 * nseg))
        if prob.pure_neumann and nseg > 0:
            A = A.tolil()
            A[nseg, :] = 0.0
            A[nseg, nseg] = 1.0
            A = A.tocsr()
        self.A = A
        self.lu = spla.splu(A.tocsc()) if nseg > 0 else None

    def solve_system(self, with_bc=True, source=None, rhs13=None, rhs14=None):
        """Returns (p[ny, nx], U, P) for the given data."""
        dec, nseg, prob = self.dec, self.nseg, self.prob
        b = np.zeros(2 * nseg)
        parts = []
        for lp in self.leaves:
            i = lp.leaf["id"]
            src = lp.block(source)
            _, part, _ = lp.solve(np.zeros(len(lp.segs)), with_data=with_bc, source=src,
                                  want_faces=False)
            parts.append(src)
            for kr, r in enumerate(lp.segs):
                s_ir = dec.side(r, i)
                beta_r = dec.segments[r]["beta"]
                b[r] -= beta_r * part[kr] * s_ir
                b[nseg + r] -= part[kr]
        if rhs14 is not None:
            b[:nseg] += np.array([t["beta"] for t in dec.segments]) * rhs14
        if rhs13 is not None:
            b[nseg:] += rhs13
        if prob.pure_neumann and nseg > 0:
            b[nseg] = 0.0
        X = self.lu.solve(b) if nseg > 0 else np.zeros(0)
        U, P = X[:nseg], X[nseg:]
        # Eq. (final): pressures as the MMBF combination plus the particular part
        p = np.zeros(prob.K.shape)
        for lp, lam, src in zip(self.leaves, self.lams, parts):
            m = len(lp.segs)
            coef = np.array([U[t] for t in lp.segs] + [P[t] for t in lp.segs])
            ph, _, _ = lp.solve(lam, with_data=False, want_faces=False)
            pp, _, _ = lp.solve(np.zeros(m), with_data=with_bc, source=src, want_faces=False)
            lp.place(p, ph @ coef + pp)
        return p, U, P


def solve_mrcm(prob, return_leaf_ops=False, refine=0):
    g = GlobalMRCM(prob)
    if refine > 0:
        from .refine import refine_solution, fluxes_from_state, shift_mean
        p, U, P = g.solve_system()
        state, hist = refine_solution(prob, g.dec, g.solve_system, p, U, P, refine)
        if prob.pure_neumann:
            state = shift_mean(prob, state)
        out = fluxes_from_state(prob, g.dec, state)
        out["refine_history"] = hist
    else:
        out = assemble_final(prob, g.dec, g.leaves, *g.solve_system()[1:])
    if return_leaf_ops:
        out["leaf_ops"] = [lp.robin_to_flux() for lp in g.leaves]
        out["leaf_segs"] = [lp.segs for lp in g.leaves]
    out["dec"] = g.dec
    return out


def assemble_final(prob, dec, leaves, U, P):
    """Eq. (final): u^i = sum_j X_j Phi^i_j + ubar^i, p^i likewise, then the
    pure-Neumann mean shift."""
    nx, ny = prob.nx, prob.ny
    p = np.zeros((ny, nx))
    Fa_x = np.zeros((ny, nx + 1)); Fb_x = np.zeros((ny, nx + 1))
    Fa_y = np.zeros((ny + 1, nx)); Fb_y = np.zeros((ny + 1, nx))
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
