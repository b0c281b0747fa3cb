"""CPU Recursive MRCM (Algorithm 1 of the paper), dense FP64.

The hierarchy of Section 3.1 (Eqs. dd.l, dd.2, interface.1): the root box of
leaves is bisected recursively until single leaves remain.  Reading for the
split (the paper assumes powers of two per direction): cut the axis with more
leaves (ties: x first, or y first when tie="y"), the lower half receiving
ceil(count/2) leaves.

Each node is represented by the traces of its MMBFs on its outer segments,
i.e. its Robin-to-flux map: outward segment fluxes F = R lambda + rbar,
where lambda is the Robin datum P - beta U (n.n^i) of Eq. (11.2).  A P-type
MMBF (Eq. 11Hhatbasisb) is lambda = e_s, and a U-type one (Eq.
11Hhatbasisa) is lambda = -beta_s n_s.n^i e_s, so R carries the traces of
all MMBFs of the node, as in the coefficient-tracking remark of Section 3.2.

Merging two children (Algorithm 1, "compute the coefficients X, Xbar by
solving (linsys) on gamma"): the unknowns on gamma are the paper's (U_t,
P_t); the rows are Eq. (14.2) and Eq. (13.2) for each gamma segment, with
the children's fluxes written through their R, rbar.  Solving gives gamma's
(U, P) as X lambda_outer + Xbar, and the node's map follows by substitution
(Eqs. new_bfs / particular.1-2, read as: basis responses are purely
homogeneous, the particular part combines as in Eq. particular).
"""
import numpy as np

from .geometry import Decomposition
from .local import LeafProblem


class Node:
    def __init__(self, box, depth):
        self.box = box          # (I0, I1, J0, J1) leaf index ranges
        self.depth = depth
        self.children = []
        self.leaf = None


def build_tree(dec, tie="x"):
    def rec(box, depth):
        node = Node(box, depth)
        I0, I1, J0, J1 = box
        nxl, nyl = I1 - I0, J1 - J0
        if nxl == 1 and nyl == 1:
            node.leaf = dec.leaf_id(I0, J0)
            return node
        split_x = nxl > nyl or (nxl == nyl and tie == "x")
        if split_x:
            mid = I0 + (nxl + 1) // 2
            node.axis = 0
            node.children = [rec((I0, mid, J0, J1), depth + 1), rec((mid, I1, J0, J1), depth + 1)]
        else:
            mid = J0 + (nyl + 1) // 2
            node.axis = 1
            node.children = [rec((I0, I1, J0, mid), depth + 1), rec((I0, I1, mid, J1), depth + 1)]
        return node
    return rec((0, dec.Nlx, 0, dec.Nly), 0)


def _in_box(dec, leaf, box):
    lf = dec.leaves[leaf]
    return box[0] <= lf["I"] < box[1] and box[2] <= lf["J"] < box[3]


def outer_segments(dec, box):
    """Segments with exactly one side inside the box, sorted by id."""
    out = []
    for t in dec.segments:
        ia, ib = _in_box(dec, t["a"], box), _in_box(dec, t["b"], box)
        if ia != ib:
            out.append(t["id"])
    return out


class RecursiveMRCM:
    def __init__(self, prob, tie="x"):
        self.prob = prob
        self.dec = Decomposition(prob)
        self.root = build_tree(self.dec, tie)
        self.leaf_problems = {}

    # ---- upward pass: leaves via MFEM, then merges ---------------------
    def _up(self, node):
        dec = self.dec
        node.segs = outer_segments(dec, node.box)
        if node.leaf is not None:
            lp = LeafProblem(dec, node.leaf)
            self.leaf_problems[node.leaf] = lp
            assert lp.segs == node.segs
            node.R, node.rbar = lp.robin_to_flux()
            return
        c1, c2 = node.children
        self._up(c1)
        self._up(c2)
        gamma = [t for t in c1.segs if t in set(c2.segs)]
        node.gamma = gamma
        g = len(gamma)
        p1 = {t: k for k, t in enumerate(c1.segs)}
        p2 = {t: k for k, t in enumerate(c2.segs)}
        o1 = [t for t in c1.segs if t not in set(gamma)]
        o2 = [t for t in c2.segs if t not in set(gamma)]
        assert sorted(o1 + o2) == node.segs
        node.o1, node.o2 = o1, o2
        beta = np.array([dec.segments[t]["beta"] for t in gamma])
        length = np.array([dec.segments[t]["length"] for t in gamma])
        # c1 lies on side a of every gamma segment (lower coordinate)
        for t in gamma:
            assert _in_box(dec, dec.segments[t]["a"], c1.box)
        # lambda^{c1}_t = P_t - beta_t U_t ; lambda^{c2}_t = P_t + beta_t U_t
        # as functions of Y = (U_gamma, P_gamma):
        L1 = np.hstack([-np.diag(beta), np.eye(g)])
        L2 = np.hstack([np.diag(beta), np.eye(g)])
        ig1 = [p1[t] for t in gamma]; ig2 = [p2[t] for t in gamma]
        io1 = [p1[t] for t in o1]; io2 = [p2[t] for t in o2]
        # fluxes of each child through gamma: F^c_gamma = R^c_gg L^c Y + R^c_go lam_o + rbar^c_g
        Fy1 = c1.R[np.ix_(ig1, ig1)] @ L1
        Fy2 = c2.R[np.ix_(ig2, ig2)] @ L2
        no = len(o1) + len(o2)
        Fo1 = np.zeros((g, no)); Fo1[:, :len(o1)] = c1.R[np.ix_(ig1, io1)]
        Fo2 = np.zeros((g, no)); Fo2[:, len(o1):] = c2.R[np.ix_(ig2, io2)]
        # rows of Eq. (14.2): beta (F1 - U|t|) - beta (F2 + U|t|) = 0
        # rows of Eq. (13.2): F1 + F2 = 0
        Ucol = np.hstack([np.diag(length), np.zeros((g, g))])
        E = np.vstack([beta[:, None] * (Fy1 - Fy2 - 2 * Ucol), Fy1 + Fy2])
        G = -np.vstack([beta[:, None] * (Fo1 - Fo2), Fo1 + Fo2])
        h = -np.vstack([(beta * (c1.rbar[ig1] - c2.rbar[ig2]))[:, None],
                        (c1.rbar[ig1] + c2.rbar[ig2])[:, None]])[:, 0]
        node.E, node.G, node.h = E, G, h
        node.L1, node.L2 = L1, L2
        if node is self.root:
            return
        X = np.linalg.solve(E, G)
        Xbar = np.linalg.solve(E, h)
        node.X, node.Xbar = X, Xbar
        # node map on o = o1 + o2
        R = np.zeros((no, no)); rbar = np.zeros(no)
        n1 = len(o1)
        R[:n1, :n1] = c1.R[np.ix_(io1, io1)]
        R[n1:, n1:] = c2.R[np.ix_(io2, io2)]
        R[:n1, :] += c1.R[np.ix_(io1, ig1)] @ L1 @ X
        R[n1:, :] += c2.R[np.ix_(io2, ig2)] @ L2 @ X
        rbar[:n1] = c1.rbar[io1] + c1.R[np.ix_(io1, ig1)] @ L1 @ Xbar
        rbar[n1:] = c2.rbar[io2] + c2.R[np.ix_(io2, ig2)] @ L2 @ Xbar
        # reorder o1 + o2 into sorted segment order
        order = np.argsort(o1 + o2)
        node.perm = order
        node.R = R[np.ix_(order, order)]
        node.rbar = rbar[order]

    # ---- downward pass ----------------------------------------------------
    def _down(self, node, lam):
        """lam: Robin data on node.segs (this node's side)."""
        if node.leaf is not None:
            node.lam = lam
            return
        c1, c2 = node.children
        g = len(node.gamma)
        if node is self.root:
            E, h = node.E.copy(), node.h.copy()
            if self.prob.pure_neumann:
                # replace the Eq. (13.2) row of the first gamma segment by P = 0
                E[g, :] = 0.0
                E[g, g] = 1.0
                h[g] = 0.0
            Y = np.linalg.solve(E, h)
        else:
            lam_o = np.zeros(len(node.o1) + len(node.o2))
            lam_o[node.perm] = lam
            Y = node.X @ lam_o + node.Xbar
        lam1 = dict(zip(node.gamma, node.L1 @ Y))
        lam2 = dict(zip(node.gamma, node.L2 @ Y))
        pos = {t: k for k, t in enumerate(node.segs)}
        for t in node.o1:
            lam1[t] = lam[pos[t]]
        for t in node.o2:
            lam2[t] = lam[pos[t]]
        self._down(c1, np.array([lam1[t] for t in c1.segs]))
        self._down(c2, np.array([lam2[t] for t in c2.segs]))

    def solve(self):
        prob = self.prob
        self._up(self.root)
        self._down(self.root, np.zeros(0))
        nx, ny = prob.nx, prob.ny
        p = np.zeros((ny, nx))
        Fa_x = np.zeros((ny, nx + 1)); Fb_x = np.zeros((ny, nx + 1))
        Fa_y = np.zeros((ny + 1, nx)); Fb_y = np.zeros((ny + 1, nx))
        stack = [self.root]
        while stack:
            node = stack.pop()
            if node.leaf is None:
                stack += node.children
                continue
            lp = self.leaf_problems[node.leaf]
            pl, _, faces = lp.solve(node.lam, with_data=True)
            p[lp.j0:lp.j1, lp.i0:lp.i1] = pl.reshape(lp.h, lp.w)
            for key, val in faces.items():
                d, jj, ii = key
                lower = (ii > lp.i0) if d == "x" else (jj > lp.j0)
                ta, tb = (Fa_x, Fb_x) if d == "x" else (Fa_y, Fb_y)
                if lp.faces[key][0] == "robin":
                    (ta if lower else tb)[jj, ii] = val
                else:
                    ta[jj, ii] = val
                    tb[jj, ii] = val
        if prob.pure_neumann:
            p -= p.mean()
        return dict(p=p, Fx=0.5 * (Fa_x + Fb_x), Fy=0.5 * (Fa_y + Fb_y),
                    Fa_x=Fa_x, Fb_x=Fb_x, Fa_y=Fa_y, Fb_y=Fb_y)


def solve_recursive(prob, tie="x"):
    return RecursiveMRCM(prob, tie).solve()
