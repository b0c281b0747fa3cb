"""Leaves, interface segments and Robin coefficients (oracle side).

Follows Section 2 (Eqs. decomp.1-2: non-overlapping subdomains, skeleton
Gamma, interfaces Gamma^{ik}) and Section 4 (the intermediate scale H-bar:
each interface is cut into segments of H-bar that carry one piecewise-
constant interface unknown each).  The Robin coefficient per segment is
Eq. (robin.beta) with K_eff from Eq. (permeff).

Conventions of this oracle (readings where the paper is silent):
  * leaves are sub[0] x sub[1] cell boxes; the last leaf of a row/column is
    truncated when the grid is not a multiple of the leaf size;
  * a segment spans seg[1] cells along y on an x-normal interface and
    seg[0] cells along x on a y-normal interface; the last segment of a
    truncated interface is shorter;
  * the reference normal of every segment is the +axis direction; side "a"
    is the leaf below it (lower coordinate), side "b" the one above.  The
    paper points it towards the larger subdomain index instead; that only
    flips the sign of U, never p or u.
  * H-bar of a segment is its length |t| (2D, per unit depth).
"""
import numpy as np


class Decomposition:
    def __init__(self, prob):
        self.prob = prob
        nx, ny = prob.nx, prob.ny
        sx, sy = prob.sub
        self.Nlx = -(-nx // sx)
        self.Nly = -(-ny // sy)
        self.leaves = []
        for J in range(self.Nly):
            for I in range(self.Nlx):
                self.leaves.append(dict(
                    id=len(self.leaves), I=I, J=J,
                    i0=I * sx, i1=min((I + 1) * sx, nx),
                    j0=J * sy, j1=min((J + 1) * sy, ny)))
        self.segments = []
        # x-normal interfaces between leaf columns I-1 and I
        for J in range(self.Nly):
            for I in range(1, self.Nlx):
                a = self.leaf_id(I - 1, J)
                b = self.leaf_id(I, J)
                line = self.leaves[b]["i0"]
                lo, hi = self.leaves[b]["j0"], self.leaves[b]["j1"]
                for s0 in range(lo, hi, prob.seg[1]):
                    self._add_segment(0, line, s0, min(s0 + prob.seg[1], hi), a, b)
        # y-normal interfaces between leaf rows J-1 and J
        for J in range(1, self.Nly):
            for I in range(self.Nlx):
                a = self.leaf_id(I, J - 1)
                b = self.leaf_id(I, J)
                line = self.leaves[b]["j0"]
                lo, hi = self.leaves[b]["i0"], self.leaves[b]["i1"]
                for s0 in range(lo, hi, prob.seg[0]):
                    self._add_segment(1, line, s0, min(s0 + prob.seg[0], hi), a, b)
        # face -> segment lookup
        self.xface_seg = -np.ones((ny, nx + 1), dtype=np.int64)
        self.yface_seg = -np.ones((ny + 1, nx), dtype=np.int64)
        for t in self.segments:
            if t["axis"] == 0:
                self.xface_seg[t["lo"]:t["hi"], t["line"]] = t["id"]
            else:
                self.yface_seg[t["line"], t["lo"]:t["hi"]] = t["id"]
        # segments of each leaf (those with the leaf on side a or b), by id
        for lf in self.leaves:
            lf["segs"] = []
        for t in self.segments:
            self.leaves[t["a"]]["segs"].append(t["id"])
            self.leaves[t["b"]]["segs"].append(t["id"])
        for lf in self.leaves:
            lf["segs"].sort()
        self._robin_coefficients()

    def leaf_id(self, I, J):
        return I + self.Nlx * J

    def _add_segment(self, axis, line, lo, hi, a, b):
        self.segments.append(dict(id=len(self.segments), axis=axis, line=line,
                                  lo=lo, hi=hi, a=a, b=b))

    def face_cells(self, t):
        """(cell_a, cell_b) index pairs (j, i) of the faces of segment t."""
        if t["axis"] == 0:
            return [((j, t["line"] - 1), (j, t["line"])) for j in range(t["lo"], t["hi"])]
        return [((t["line"] - 1, i), (t["line"], i)) for i in range(t["lo"], t["hi"])]

    def _robin_coefficients(self):
        """Eqs. (robin.beta) and (permeff): beta_t = alpha * Hbar / Keff_t,
        Keff_t = mean over the segment's fine faces of the harmonic mean of
        the two adjacent cell permeabilities."""
        K = self.prob.K
        for t in self.segments:
            hm = [2.0 * K[ca] * K[cb] / (K[ca] + K[cb]) for ca, cb in self.face_cells(t)]
            keff = sum(hm) / len(hm)
            h_tan = self.prob.hy if t["axis"] == 0 else self.prob.hx
            length = (t["hi"] - t["lo"]) * h_tan
            t["keff"] = keff
            t["length"] = length
            t["beta"] = self.prob.alpha * length / keff

    def side(self, t, leaf):
        """n_t . n^i: +1 when the leaf is side a (below), -1 when side b."""
        return 1.0 if self.segments[t]["a"] == leaf else -1.0
