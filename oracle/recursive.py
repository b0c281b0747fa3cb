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

The homogeneous part (R, X) is built once; solve_rhs() runs the particular
up-sweep and the top-down pass for any data (source, external boundary data
on or off, right-hand sides of the Eq. 13.2 / 14.2 rows), which also serves
iterative refinement (oracle.refine).

Large problems (leaf_map): the per-leaf work -- each leaf's map R, its
particular fluxes for given data, its final pressures for given Robin data
-- is independent from leaf to leaf (the local problems of Eqs. 11.2-12.2).
With leaf_map (a map function, e.g. a process pool's, whose workers ran
leaf_worker_init(prob)) that work is handed to it leaf by leaf and the leaf
problems are rebuilt for every use instead of being kept: the same
arithmetic per leaf, without the memory of 256 x 256 dense factors for tens
of thousands of leaves.
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


# per-process state of the leaf workers (leaf_map mode)
_WORKER = {}


def leaf_worker_init(prob):
    """Initialiser of a leaf worker: the decomposition of the problem."""
    _WORKER["dec"] = Decomposition(prob)


def leaf_R_task(leaf):
    """Robin-to-flux map of one leaf (as in RecursiveMRCM._build)."""
    R, _ = LeafProblem(_WORKER["dec"], leaf).robin_to_flux()
    return R


def leaf_rbar_task(args):
    """Particular segment fluxes of one leaf for the data (lambda = 0)."""
    leaf, with_bc, src = args
    lp = LeafProblem(_WORKER["dec"], leaf)
    _, rbar, _ = lp.solve(np.zeros(len(lp.segs)), with_data=with_bc, source=src, want_faces=False)
    return rbar


def leaf_p_task(args):
    """Final pressures of one leaf for its Robin data lam and the data."""
    leaf, lam, with_bc, src = args
    lp = LeafProblem(_WORKER["dec"], leaf)
    pl, _, _ = lp.solve(lam, with_data=with_bc, source=src, want_faces=False)
    return pl


class RecursiveMRCM:
    def __init__(self, prob, tie="x", leaf_map=None):
        self.prob = prob
        self.dec = Decomposition(prob)
        self.root = build_tree(self.dec, tie)
        self.leaf_problems = {}
        self.leaf_map = leaf_map
        if leaf_map is not None:
            ids = [lf["id"] for lf in self.dec.leaves]
            self._leaf_R = dict(zip(ids, leaf_map(leaf_R_task, ids)))
        self._build(self.root)
        self._leaf_R = None

    # ---- homogeneous part: leaves via MFEM, merges -------------------------
    def _build(self, node):
        dec = self.dec
        if node.leaf is not None:
            # the segments touching the leaf: those with exactly one side
            # in its box
            node.segs = dec.leaves[node.leaf]["segs"]
            if self.leaf_map is not None:
                node.R = self._leaf_R[node.leaf]
                return
            lp = LeafProblem(dec, node.leaf)
            self.leaf_problems[node.leaf] = lp
            assert lp.segs == node.segs
            node.R, _ = lp.robin_to_flux()
            return
        c1, c2 = node.children
        self._build(c1)
        self._build(c2)
        # gamma: segments with one side in each child; the node's outer
        # segments (exactly one side in its box) are the children's others
        s2 = set(c2.segs)
        gamma = [t for t in c1.segs if t in s2]
        node.gamma = gamma
        gset = set(gamma)
        node.segs = sorted([t for t in c1.segs if t not in gset] + [t for t in c2.segs if t not in gset])
        g = len(gamma)
        p1 = {t: k for k, t in enumerate(c1.segs)}
        p2 = {t: k for k, t in enumerate(c2.segs)}
        o1 = [t for t in c1.segs if t not in gset]
        o2 = [t for t in c2.segs if t not in gset]
        assert sorted(o1 + o2) == node.segs
        node.o1, node.o2 = o1, o2
        beta = np.array([dec.segments[t]["beta"] for t in gamma])
        length = np.array([dec.segments[t]["length"] for t in gamma])
        node.beta = beta
        # c1 lies on side a of every gamma segment (lower coordinate)
        for t in gamma:
            assert _in_box(dec, dec.segments[t]["a"], c1.box)
        # lambda^{c1}_t = P_t - beta_t U_t ; lambda^{c2}_t = P_t + beta_t U_t
        # as functions of Y = (U_gamma, P_gamma):
        L1 = np.hstack([-np.diag(beta), np.eye(g)])
        L2 = np.hstack([np.diag(beta), np.eye(g)])
        ig1 = [p1[t] for t in gamma]; ig2 = [p2[t] for t in gamma]
        io1 = [p1[t] for t in o1]; io2 = [p2[t] for t in o2]
        node.ig1, node.ig2, node.io1, node.io2 = ig1, ig2, io1, io2
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
        node.E, node.G = E, G
        node.L1, node.L2 = L1, L2
        if node is self.root:
            if self.prob.pure_neumann:
                # replace the Eq. (13.2) row of the first gamma segment by P = 0
                E = E.copy()
                E[g, :] = 0.0
                E[g, g] = 1.0
                node.E = E
            return
        X = np.linalg.solve(E, G)
        node.X = X
        # node map on o = o1 + o2
        R = np.zeros((no, no))
        n1 = len(o1)
        R[:n1, :n1] = c1.R[np.ix_(io1, io1)]
        R[n1:, n1:] = c2.R[np.ix_(io2, io2)]
        R[:n1, :] += c1.R[np.ix_(io1, ig1)] @ L1 @ X
        R[n1:, :] += c2.R[np.ix_(io2, ig2)] @ L2 @ X
        # reorder o1 + o2 into sorted segment order
        order = np.argsort(o1 + o2)
        node.perm = order
        node.R = R[np.ix_(order, order)]

    # ---- particular part for given data -----------------------------------
    def _up(self, node, data):
        if node.leaf is not None:
            if self.leaf_map is not None:
                node.rbar = data["leaf_rbar"][node.leaf]
                return
            lp = self.leaf_problems[node.leaf]
            src = data["source"]
            src = None if src is None else src[lp.j0:lp.j1, lp.i0:lp.i1]
            _, node.rbar, _ = lp.solve(np.zeros(len(lp.segs)), with_data=data["with_bc"], source=src,
                                       want_faces=False)
            return
        c1, c2 = node.children
        self._up(c1, data)
        self._up(c2, data)
        g = len(node.gamma)
        r1 = c1.rbar[node.ig1]
        r2 = c2.rbar[node.ig2]
        h = -np.concatenate([node.beta * (r1 - r2), r1 + r2])
        if data["rhs14"] is not None:
            h[:g] += node.beta * data["rhs14"][node.gamma]
        if data["rhs13"] is not None:
            h[g:] += data["rhs13"][node.gamma]
        if node is self.root:
            if self.prob.pure_neumann:
                h[g] = 0.0
            node.h = h
            return
        node.Xbar = np.linalg.solve(node.E, h)
        n1 = len(node.o1)
        rbar = np.zeros(len(node.o1) + len(node.o2))
        rbar[:n1] = c1.rbar[node.io1] + c1.R[np.ix_(node.io1, node.ig1)] @ node.L1 @ node.Xbar
        rbar[n1:] = c2.rbar[node.io2] + c2.R[np.ix_(node.io2, node.ig2)] @ node.L2 @ node.Xbar
        node.rbar = rbar[node.perm]

    def _down(self, node, lam, UP):
        """lam: Robin data on node.segs (this node's side)."""
        if node.leaf is not None:
            node.lam = lam
            return
        c1, c2 = node.children
        g = len(node.gamma)
        if node is self.root:
            Y = np.linalg.solve(node.E, node.h)
        else:
            lam_o = np.zeros(len(node.o1) + len(node.o2))
            lam_o[node.perm] = lam
            Y = node.X @ lam_o + node.Xbar
        UP[0][node.gamma] = Y[:g]
        UP[1][node.gamma] = Y[g:]
        lam1 = dict(zip(node.gamma, node.L1 @ Y))
        lam2 = dict(zip(node.gamma, node.L2 @ Y))
        pos = {t: k for k, t in enumerate(node.segs)}
        for t in node.o1:
            lam1[t] = lam[pos[t]]
        for t in node.o2:
            lam2[t] = lam[pos[t]]
        self._down(c1, np.array([lam1[t] for t in c1.segs]), UP)
        self._down(c2, np.array([lam2[t] for t in c2.segs]), UP)

    def _leaves(self):
        stack = [self.root]
        while stack:
            node = stack.pop()
            if node.leaf is None:
                stack += node.children
            else:
                yield node

    def solve_rhs(self, with_bc=True, source=None, rhs13=None, rhs14=None):
        """(p[ny, nx], U, P) for the given data."""
        prob = self.prob
        data = dict(with_bc=with_bc, source=source, rhs13=rhs13, rhs14=rhs14)
        nseg = len(self.dec.segments)
        UP = (np.zeros(nseg), np.zeros(nseg))
        leaves = self.dec.leaves

        def block(lf):
            return None if source is None else source[lf["j0"]:lf["j1"], lf["i0"]:lf["i1"]]

        if self.leaf_map is not None:
            ids = [lf["id"] for lf in leaves]
            data["leaf_rbar"] = dict(zip(ids, self.leaf_map(
                leaf_rbar_task, [(i, with_bc, block(leaves[i])) for i in ids])))
        self._up(self.root, data)
        self._down(self.root, np.zeros(0), UP)
        p = np.zeros((prob.ny, prob.nx))
        nodes = list(self._leaves())
        if self.leaf_map is not None:
            pls = self.leaf_map(leaf_p_task, [(nd.leaf, nd.lam, with_bc, block(leaves[nd.leaf])) for nd in nodes])
        else:
            pls = []
            for node in nodes:
                lp = self.leaf_problems[node.leaf]
                pl, _, _ = lp.solve(node.lam, with_data=with_bc, source=block(leaves[node.leaf]),
                                    want_faces=False)
                pls.append(pl)
        for node, pl in zip(nodes, pls):
            lf = leaves[node.leaf]
            p[lf["j0"]:lf["j1"], lf["i0"]:lf["i1"]] = np.asarray(pl).reshape(lf["j1"] - lf["j0"],
                                                                               lf["i1"] - lf["i0"])
        return p, UP[0], UP[1]

    def solve(self, refine=0):
        prob = self.prob
        if refine > 0:
            from .refine import refine_solution, fluxes_from_state, shift_mean
            p, U, P = self.solve_rhs()
            state, hist = refine_solution(prob, self.dec, self.solve_rhs, p, U, P, refine)
            if prob.pure_neumann:
                state = shift_mean(prob, state)
            out = fluxes_from_state(prob, self.dec, state)
            out["refine_history"] = hist
            return out
        self._up(self.root, dict(with_bc=True, source=None, rhs13=None, rhs14=None))
        nseg = len(self.dec.segments)
        self._down(self.root, np.zeros(0), (np.zeros(nseg), np.zeros(nseg)))
        nx, ny = prob.nx, prob.ny
        p = np.zeros((ny, nx))
        Fa_x = np.zeros((ny, nx + 1)); Fb_x = np.zeros((ny, nx + 1))
        Fa_y = np.zeros((ny + 1, nx)); Fb_y = np.zeros((ny + 1, nx))
        for node in self._leaves():
            lp = self.leaf_problems.get(node.leaf) or LeafProblem(self.dec, node.leaf)
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


def solve_recursive(prob, tie="x", refine=0, leaf_map=None):
    return RecursiveMRCM(prob, tie, leaf_map=leaf_map).solve(refine=refine)
