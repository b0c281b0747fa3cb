"""Local Robin problems on one leaf and its MMBFs (oracle side).

Eqs. (11.2)-(12.2) restricted to one subdomain Omega^i with lumped RT0
(two-point fluxes, see oracle.fine).  On a skeleton face e inside segment t
the Robin term of Eq. (11.2), with the half-cell Darcy law
u.n^i = 2K_c (p_c - p_e)/h_d, gives the outward integrated flux

    F_e = rho_e (p_c - lambda^i_t),   rho_e = |e| / (h_d/(2K_c) + beta_t),
    lambda^i_t = P_t - beta_t U_t (n_t . n^i),

so the interface data (U_H, P_H) enter only through lambda.  Domain
boundary faces carry the Dirichlet / Neumann data of Eqs. (ellip.2-3).

MMBFs (Section 3.1, Eqs. 11Hhatbasisa and 11Hhatbasisb): for each segment j
of the leaf, one solve with U_H = phi^j, P_H = 0 (lambda_j = -beta_j
n_j.n^i) and one with P_H = psi^j, U_H = 0 (lambda_j = 1), both with zero
source and zero external data; the particular solution has lambda = 0 and
the source / external data (Eqs. addu, addp).
"""
import numpy as np
import scipy.linalg as sla

from inputs.problems import DIRICHLET


class LeafProblem:
    def __init__(self, dec, leaf_id):
        prob = dec.prob
        lf = dec.leaves[leaf_id]
        self.dec, self.leaf = dec, lf
        self.i0, self.i1, self.j0, self.j1 = lf["i0"], lf["i1"], lf["j0"], lf["j1"]
        w, h = self.i1 - self.i0, self.j1 - self.j0
        self.w, self.h, self.n = w, h, w * h
        self.segs = lf["segs"]
        self.seg_pos = {t: k for k, t in enumerate(self.segs)}
        K, hx, hy = prob.K, prob.hx, prob.hy
        A = np.zeros((self.n, self.n))
        bbar = np.zeros(self.n)
        loc = lambda i, j: (i - self.i0) + w * (j - self.j0)
        # faces of the leaf: ("x", j, i) is the x-face i of row j, ("y", j, i)
        # the y-face j of column i.  Each entry records how its flux follows
        # from the cell pressures.
        self.faces = {}
        bcs = prob.bc_slices()
        for j in range(self.j0, self.j1):
            for i in range(self.i0, self.i1):
                c = loc(i, j)
                bbar[c] += prob.q[j, i]
                for d, (fkey, ni, nj, outsign) in enumerate([
                        (("x", j, i), i - 1, j, -1.0), (("x", j, i + 1), i + 1, j, +1.0),
                        (("y", j, i), i, j - 1, -1.0), (("y", j + 1, i), i, j + 1, +1.0)]):
                    axis = 0 if d < 2 else 1
                    hn, area = (hx, hy) if axis == 0 else (hy, hx)
                    inside = self.i0 <= ni < self.i1 and self.j0 <= nj < self.j1
                    in_domain = 0 <= ni < prob.nx and 0 <= nj < prob.ny
                    if inside:
                        T = area / (hn / (2 * K[j, i]) + hn / (2 * K[nj, ni]))
                        A[c, c] += T
                        A[c, loc(ni, nj)] -= T
                        if outsign > 0:
                            self.faces[fkey] = ("int", c, loc(ni, nj), T)
                    elif in_domain:
                        t = (dec.xface_seg[fkey[1], fkey[2]] if axis == 0
                             else dec.yface_seg[fkey[1], fkey[2]])
                        beta = dec.segments[t]["beta"]
                        rho = area / (hn / (2 * K[j, i]) + beta)
                        A[c, c] += rho
                        self.faces[fkey] = ("robin", c, int(t), rho, outsign)
                    else:
                        side = (0 if outsign < 0 else 1) if axis == 0 else (2 if outsign < 0 else 3)
                        k = j if axis == 0 else i
                        gval = prob.bc_val[bcs[side]][k]
                        if prob.bc_type[side] == DIRICHLET:
                            tau = 2.0 * K[j, i] * area / hn
                            A[c, c] += tau
                            bbar[c] += tau * gval
                            self.faces[fkey] = ("dir", c, tau, gval, outsign)
                        else:
                            bbar[c] -= area * gval
                            self.faces[fkey] = ("neu", c, area * gval, outsign)
        self.A = A
        self.bbar = bbar
        # Robin load matrix: column k is the right-hand side of a unit lambda
        # on segment segs[k]
        self.B = np.zeros((self.n, len(self.segs)))
        for f in self.faces.values():
            if f[0] == "robin":
                _, c, t, rho, _ = f
                self.B[c, self.seg_pos[t]] += rho
        # face tables by kind, for vectorised flux evaluation
        keys = {k: [] for k in ("int", "robin", "dir", "neu")}
        for key, f in self.faces.items():
            keys[f[0]].append((key, f))
        self.kind_keys = {k: [kf[0] for kf in v] for k, v in keys.items()}
        fi = [kf[1] for kf in keys["int"]]
        self.int_c = np.array([f[1] for f in fi], dtype=np.int64)
        self.int_c2 = np.array([f[2] for f in fi], dtype=np.int64)
        self.int_T = np.array([f[3] for f in fi])
        fr = [kf[1] for kf in keys["robin"]]
        self.rob_c = np.array([f[1] for f in fr], dtype=np.int64)
        self.rob_k = np.array([self.seg_pos[f[2]] for f in fr], dtype=np.int64)
        self.rob_rho = np.array([f[3] for f in fr])
        self.rob_sign = np.array([f[4] for f in fr])
        fd = [kf[1] for kf in keys["dir"]]
        self.dir_c = np.array([f[1] for f in fd], dtype=np.int64)
        self.dir_tau = np.array([f[2] for f in fd])
        self.dir_g = np.array([f[3] for f in fd])
        self.dir_sign = np.array([f[4] for f in fd])
        fn = [kf[1] for kf in keys["neu"]]
        self.neu_flux = np.array([f[2] for f in fn])
        self.neu_sign = np.array([f[3] for f in fn])
        self._lu = None

    def block(self, arr):
        """The leaf's block of a cell array (None passes through)."""
        return None if arr is None else arr[self.j0:self.j1, self.i0:self.i1]

    def place(self, out, vals):
        """Writes the leaf's cell values into a cell array."""
        out[self.j0:self.j1, self.i0:self.i1] = np.asarray(vals).reshape(self.h, self.w)

    def solve(self, lam, with_data, source=None, want_faces=True):
        """Solve the local problem for Robin data lam (one value per segment
        of the leaf, in self.segs order) with or without the source and
        external boundary data.  Several data sets may be passed as the
        columns of lam (shape (m, k)).  `source` (h x w) adds a cell source
        without external data (used for residual corrections).  Returns
        (p[n, k], outward segment fluxes [m, k], face flux dict in +axis
        direction, or None when want_faces is false)."""
        lam = np.asarray(lam, dtype=np.float64)
        single = lam.ndim == 1
        if single:
            lam = lam[:, None]
        rhs = self.B @ lam
        if with_data:
            rhs = rhs + self.bbar[:, None]
        if source is not None:
            rhs = rhs + np.asarray(source, dtype=np.float64).reshape(-1)[:, None]
        if self._lu is None:
            self._lu = sla.lu_factor(self.A)
        p = sla.lu_solve(self._lu, rhs)
        # Robin faces: outward flux rho (p_c - lambda_t)
        rob = self.rob_rho[:, None] * (p[self.rob_c] - lam[self.rob_k])
        seg_flux = np.zeros_like(lam)
        np.add.at(seg_flux, self.rob_k, rob)
        faces = None
        if want_faces:
            k = p.shape[1]
            vals = {}
            fint = self.int_T[:, None] * (p[self.int_c] - p[self.int_c2])
            vals.update(zip(self.kind_keys["int"], fint))
            vals.update(zip(self.kind_keys["robin"], self.rob_sign[:, None] * rob))
            g = self.dir_g[:, None] if with_data else 0.0
            fdir = self.dir_sign[:, None] * (self.dir_tau[:, None] * (p[self.dir_c] - g))
            vals.update(zip(self.kind_keys["dir"], fdir))
            fneu = self.neu_sign[:, None] * (self.neu_flux[:, None] if with_data else np.zeros((len(self.neu_flux), 1)))
            vals.update(zip(self.kind_keys["neu"], fneu * np.ones((1, k))))
            faces = {key: (v[0] if single else v) for key, v in vals.items()}
        if single:
            p, seg_flux = p[:, 0], seg_flux[:, 0]
        return p, seg_flux, faces

    def robin_to_flux(self):
        """R[t, s] = outward flux through segment t for lambda = e_s, no data
        (the P_H = psi^s MMBF traces), and rbar = particular flux traces."""
        _, R, _ = self.solve(np.eye(len(self.segs)), with_data=False, want_faces=False)
        _, rbar, _ = self.solve(np.zeros(len(self.segs)), with_data=True, want_faces=False)
        return R, rbar
