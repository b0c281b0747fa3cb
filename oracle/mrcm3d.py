"""The 3D oracle: fine solve, leaves, interface patches and O2 in three
dimensions (TEST INFRASTRUCTURE ONLY, like the rest of this package).

Section 5.1 runs every experiment in 3D: subdomains are boxes, interfaces
are rectangles and the intermediate scale H-bar cuts each interface into
patches (Section 4) that carry one piecewise-constant (U_t, P_t) pair each.
Everything below restates the 2D oracle's equations with one axis more:

  * the fine scheme is the lumped RT0 / two-point-flux scheme of oracle.fine
    (Eqs. ellip.1-3): T_e = |e| / (h_d/(2K_c) + h_d/(2K_c')), Dirichlet
    tau_e = 2 K_c |e| / h_d, Neumann outward flux |e| g_N;
  * the local Robin problems are those of oracle.local (Eqs. 11.2-12.2):
    F_e = rho_e (p_c - lambda_t), rho_e = |e| / (h_d/(2K_c) + beta_t);
  * beta_t = alpha Hbar_t / Keff_t (Eqs. robin.beta, permeff) with Keff_t the
    mean over the patch's faces of the harmonic means of the two adjacent
    cells, |t| the patch area and Hbar_t = sqrt(|t|), i.e. the patch side
    (4h for 4 x 4 patches of cubic cells; a reading for non-square patches);
  * the global interface system and the final fields are O2's (Eqs. linsys,
    brhs, final), taken from oracle.mrcm, which is written over segment lists
    and works unchanged on patches.

Conventions: arrays are (nz, ny, nx), x fastest.  Face arrays: Fx (nz, ny,
nx+1), Fy (nz, ny+1, nx), Fz (nz+1, ny, nx), integrated fluxes positive in
the +axis direction.  A face key (d, k, j, i) indexes the face array of axis
d.  Leaves are sub-cell boxes, truncated at the high edges; a patch on a
d-normal interface spans seg[t1] x seg[t2] faces along the two tangential
axes t1 < t2 (truncated likewise).  Side a of a patch is the leaf below it.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from inputs.problems import DIRICHLET


def _tangential(d):
    return [a for a in range(3) if a != d]


def _face_area(h, d):
    t1, t2 = _tangential(d)
    return h[t1] * h[t2]


def _cells_of_face(d, k, j, i):
    """(lower cell, upper cell) of the d-normal face (k, j, i), as (k, j, i)."""
    if d == 0:
        return (k, j, i - 1), (k, j, i)
    if d == 1:
        return (k, j - 1, i), (k, j, i)
    return (k - 1, j, i), (k, j, i)


def _side_index(prob, side, cell):
    """Position of a boundary cell's face inside its side's bc_val block."""
    k, j, i = cell
    nx, ny, nz = prob.n
    if side < 2:
        return k * ny + j
    if side < 4:
        return k * nx + i
    return j * nx + i


class Decomposition3D:
    def __init__(self, prob):
        self.prob = prob
        n, sub, seg = prob.n, prob.sub, prob.seg
        self.Nl = [-(-n[d] // sub[d]) for d in range(3)]
        self.leaves = []
        for L in range(self.Nl[2]):
            for J in range(self.Nl[1]):
                for I in range(self.Nl[0]):
                    idx = (I, J, L)
                    lo = tuple(idx[d] * sub[d] for d in range(3))
                    hi = tuple(min((idx[d] + 1) * sub[d], n[d]) for d in range(3))
                    self.leaves.append(dict(id=len(self.leaves), idx=idx, lo=lo, hi=hi))
        self.segments = []
        shapes = [(n[2], n[1], n[0] + 1), (n[2], n[1] + 1, n[0]), (n[2] + 1, n[1], n[0])]
        self.face_seg = [-np.ones(s, dtype=np.int64) for s in shapes]
        for d in range(3):
            t1, t2 = _tangential(d)
            for lb in self.leaves:
                if lb["idx"][d] == 0:
                    continue
                ia = list(lb["idx"]); ia[d] -= 1
                a = self.leaf_id(*ia)
                line = lb["lo"][d]
                for u0 in range(lb["lo"][t1], lb["hi"][t1], seg[t1]):
                    u1 = min(u0 + seg[t1], lb["hi"][t1])
                    for v0 in range(lb["lo"][t2], lb["hi"][t2], seg[t2]):
                        v1 = min(v0 + seg[t2], lb["hi"][t2])
                        t = dict(id=len(self.segments), axis=d, line=line,
                                 lo=(u0, v0), hi=(u1, v1), a=a, b=lb["id"])
                        self.segments.append(t)
                        for key in self.face_keys(t):
                            self.face_seg[d][key[1:]] = t["id"]
        for lf in self.leaves:
            lf["segs"] = []
        for t in self.segments:
            self.leaves[t["a"]]["segs"].append(t["id"])
            self.leaves[t["b"]]["segs"].append(t["id"])
        for lf in self.leaves:
            lf["segs"].sort()
        self._robin_coefficients()

    def leaf_id(self, I, J, L):
        return I + self.Nl[0] * (J + self.Nl[1] * L)

    @staticmethod
    def face_keys(t):
        """Face keys (d, k, j, i) of patch t."""
        d = t["axis"]
        t1, t2 = _tangential(d)
        keys = []
        for v in range(t["lo"][1], t["hi"][1]):
            for u in range(t["lo"][0], t["hi"][0]):
                pos = [0, 0, 0]
                pos[d], pos[t1], pos[t2] = t["line"], u, v
                keys.append((d, pos[2], pos[1], pos[0]))
        return keys

    def _robin_coefficients(self):
        """Eqs. (robin.beta) and (permeff) on patches: Keff_t = mean over the
        patch's faces of 2 K_a K_b / (K_a + K_b); beta_t = alpha Hbar_t /
        Keff_t with Hbar_t = sqrt(|t|)."""
        K, h = self.prob.K, self.prob.h
        for t in self.segments:
            hm = []
            for key in self.face_keys(t):
                ca, cb = _cells_of_face(*key)
                hm.append(2.0 * K[ca] * K[cb] / (K[ca] + K[cb]))
            keff = sum(hm) / len(hm)
            area = len(hm) * _face_area(h, t["axis"])
            t["keff"] = keff
            t["length"] = area            # |t|, the name O2's assembly uses
            t["hbar"] = np.sqrt(area)
            t["beta"] = self.prob.alpha * t["hbar"] / keff

    def side(self, t, leaf):
        """n_t . n^i: +1 when the leaf is side a (below), -1 when side b."""
        return 1.0 if self.segments[t]["a"] == leaf else -1.0


class LeafProblem3D:
    """The local Robin problem of one 3D leaf (Eqs. 11.2-12.2), sparse LU.
    Same interface as oracle.local.LeafProblem."""

    def __init__(self, dec, leaf_id):
        prob = dec.prob
        lf = dec.leaves[leaf_id]
        self.dec, self.leaf = dec, lf
        self.lo, self.hi = lf["lo"], lf["hi"]
        w = [self.hi[d] - self.lo[d] for d in range(3)]
        self.w = w
        self.n = n = w[0] * w[1] * w[2]
        self.segs = lf["segs"]
        self.seg_pos = {t: k for k, t in enumerate(self.segs)}
        K, h, N = prob.K, prob.h, prob.n
        lo, hi = self.lo, self.hi
        loc = lambda c: ((c[0] - lo[2]) * w[1] + (c[1] - lo[1])) * w[0] + (c[2] - lo[0])
        rows, cols, vals = [], [], []
        diag = np.zeros(n)
        bbar = np.zeros(n)
        self.faces = {}
        bcs = prob.bc_slices()
        for k in range(lo[2], hi[2]):
            for j in range(lo[1], hi[1]):
                for i in range(lo[0], hi[0]):
                    cell = (k, j, i)
                    c = loc(cell)
                    bbar[c] += prob.q[cell]
                    for d in range(3):
                        hn, area = h[d], _face_area(h, d)
                        for outsign in (-1, 1):
                            nb = list(cell)
                            nb[2 - d] += outsign
                            nb = tuple(nb)
                            fpos = [k, j, i]
                            if outsign > 0:
                                fpos[2 - d] += 1
                            key = (d, fpos[0], fpos[1], fpos[2])
                            coord = nb[2 - d]
                            inside = lo[d] <= coord < hi[d]
                            in_domain = 0 <= coord < N[d]
                            if inside:
                                T = area / (hn / (2 * K[cell]) + hn / (2 * K[nb]))
                                diag[c] += T
                                rows.append(c); cols.append(loc(nb)); vals.append(-T)
                                if outsign > 0:
                                    self.faces[key] = ("int", c, loc(nb), T)
                            elif in_domain:
                                t = int(dec.face_seg[d][key[1:]])
                                beta = dec.segments[t]["beta"]
                                rho = area / (hn / (2 * K[cell]) + beta)
                                diag[c] += rho
                                self.faces[key] = ("robin", c, t, rho, float(outsign))
                            else:
                                side = 2 * d + (0 if outsign < 0 else 1)
                                gval = prob.bc_val[bcs[side]][_side_index(prob, side, cell)]
                                if prob.bc_type[side] == DIRICHLET:
                                    tau = 2.0 * K[cell] * area / hn
                                    diag[c] += tau
                                    bbar[c] += tau * gval
                                    self.faces[key] = ("dir", c, tau, gval, float(outsign))
                                else:
                                    bbar[c] -= area * gval
                                    self.faces[key] = ("neu", c, area * gval, float(outsign))
        rows += list(range(n)); cols += list(range(n)); vals += list(diag)
        self.A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
        self.bbar = bbar
        self.B = np.zeros((n, len(self.segs)))
        for f in self.faces.values():
            if f[0] == "robin":
                self.B[f[1], self.seg_pos[f[2]]] += f[3]
        keys = {kind: [] for kind in ("int", "robin", "dir", "neu")}
        for key, f in self.faces.items():
            keys[f[0]].append((key, f))
        self.kind_keys = {kind: [kf[0] for kf in v] for kind, v in keys.items()}
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
        if arr is None:
            return None
        lo, hi = self.lo, self.hi
        return arr[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]

    def place(self, out, vals):
        lo, hi = self.lo, self.hi
        out[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = np.asarray(vals).reshape(self.w[2], self.w[1], self.w[0])

    def solve(self, lam, with_data, source=None, want_faces=True):
        """As oracle.local.LeafProblem.solve: p[n, k], outward patch fluxes
        [m, k] and, optionally, every face flux of the leaf (+axis sign)."""
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
            self._lu = spla.splu(self.A)
        p = self._lu.solve(np.ascontiguousarray(rhs))
        rob = self.rob_rho[:, None] * (p[self.rob_c] - lam[self.rob_k])
        seg_flux = np.zeros_like(lam)
        np.add.at(seg_flux, self.rob_k, rob)
        faces = None
        if want_faces:
            k = p.shape[1]
            vals = {}
            vals.update(zip(self.kind_keys["int"], self.int_T[:, None] * (p[self.int_c] - p[self.int_c2])))
            vals.update(zip(self.kind_keys["robin"], self.rob_sign[:, None] * rob))
            g = self.dir_g[:, None] if with_data else 0.0
            vals.update(zip(self.kind_keys["dir"],
                            self.dir_sign[:, None] * (self.dir_tau[:, None] * (p[self.dir_c] - g))))
            fneu = self.neu_sign[:, None] * (self.neu_flux[:, None] if with_data
                                             else np.zeros((len(self.neu_flux), 1)))
            vals.update(zip(self.kind_keys["neu"], fneu * np.ones((1, k))))
            faces = {key: (v[0] if single else v) for key, v in vals.items()}
        if single:
            p, seg_flux = p[:, 0], seg_flux[:, 0]
        return p, seg_flux, faces

    def robin_to_flux(self):
        """R[t, s]: outward flux through patch t for lambda = e_s, no data;
        rbar: the particular solution's patch fluxes."""
        _, R, _ = self.solve(np.eye(len(self.segs)), with_data=False, want_faces=False)
        _, rbar, _ = self.solve(np.zeros(len(self.segs)), with_data=True, want_faces=False)
        return R, rbar


def solve_fine3d(prob):
    """O1 in 3D (Eqs. ellip.1-3, lumped RT0 = two-point fluxes), sparse
    direct; assembled with array operations, independently of the cell
    loops of LeafProblem3D.  Pure Neumann: p_0 = 0, then zero mean."""
    nx, ny, nz = prob.n
    h = prob.h
    K = prob.K
    ncell = nx * ny * nz
    idx = np.arange(ncell).reshape(nz, ny, nx)
    r = [h[d] / (2.0 * K) for d in range(3)]
    diag = np.zeros((nz, ny, nx))
    rhs = prob.q.astype(np.float64).copy()
    rows, cols, vals = [], [], []
    T = []
    for d in range(3):
        ax = 2 - d
        area = _face_area(h, d)
        lo = [slice(None)] * 3; hi = [slice(None)] * 3
        lo[ax] = slice(0, -1); hi[ax] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        Td = area / (r[d][lo] + r[d][hi])
        T.append(Td)
        diag[lo] += Td
        diag[hi] += Td
        a, b = idx[lo].ravel(), idx[hi].ravel()
        rows += [a, b]; cols += [b, a]; vals += [-Td.ravel(), -Td.ravel()]
    bcs = prob.bc_slices()
    tau = {}
    for side in range(6):
        d, up = side // 2, side % 2
        ax = 2 - d
        area = _face_area(h, d)
        sl = [slice(None)] * 3
        sl[ax] = -1 if up else 0
        sl = tuple(sl)
        g = prob.bc_val[bcs[side]].reshape(prob.side_shape(side))
        if prob.bc_type[side] == DIRICHLET:
            t = area / r[d][sl]
            diag[sl] += t
            rhs[sl] += t * g
            tau[side] = t
        else:
            rhs[sl] -= area * g
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ncell, ncell))
    b = rhs.ravel().copy()
    if prob.pure_neumann:
        A = A.tolil()
        A[0, :] = 0.0
        A[0, 0] = 1.0
        A = A.tocsr()
        b[0] = 0.0
    p = spla.spsolve(A.tocsc(), b).reshape(nz, ny, nx)
    if prob.pure_neumann:
        p = p - p.mean()
    F = [np.zeros((nz, ny, nx + 1)), np.zeros((nz, ny + 1, nx)), np.zeros((nz + 1, ny, nx))]
    for d in range(3):
        ax = 2 - d
        lo = [slice(None)] * 3; hi = [slice(None)] * 3; mid = [slice(None)] * 3
        lo[ax] = slice(0, -1); hi[ax] = slice(1, None); mid[ax] = slice(1, -1)
        F[d][tuple(mid)] = T[d] * (p[tuple(lo)] - p[tuple(hi)])
    for side in range(6):
        d, up = side // 2, side % 2
        ax = 2 - d
        area = _face_area(h, d)
        sl = [slice(None)] * 3
        sl[ax] = -1 if up else 0
        sl = tuple(sl)
        g = prob.bc_val[bcs[side]].reshape(prob.side_shape(side))
        out = tau[side] * (p[sl] - g) if prob.bc_type[side] == DIRICHLET else area * g
        F[d][sl] = out if up else -out
    return dict(p=p, Fx=F[0], Fy=F[1], Fz=F[2], A=A, rhs=b)


def assemble_final3d(prob, dec, leaves, U, P):
    """Eq. (final) in 3D: every leaf's final local solve with the interface
    unknowns (U, P), its face fluxes, and on the skeleton both one-sided
    values (a: the lower leaf's, b: the upper leaf's; +axis sign)."""
    nx, ny, nz = prob.n
    shapes = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
    Fa = [np.zeros(s) for s in shapes]
    Fb = [np.zeros(s) for s in shapes]
    p = np.zeros((nz, ny, nx))
    for lp in leaves:
        i = lp.leaf["id"]
        lam = np.array([P[t] - dec.segments[t]["beta"] * U[t] * dec.side(t, i) for t in lp.segs])
        pl, _, faces = lp.solve(lam, with_data=True)
        lp.place(p, pl)
        for key, val in faces.items():
            d = key[0]
            pos = key[3 - d]                       # the face's coordinate along d
            lower = pos > lp.lo[d]                 # the leaf lies below the face
            if lp.faces[key][0] == "robin":
                (Fa if lower else Fb)[d][key[1:]] = val
            else:
                Fa[d][key[1:]] = val
                Fb[d][key[1:]] = val
    if prob.pure_neumann:
        shift = p.mean()
        p -= shift
        P = P - shift
    F = [0.5 * (Fa[d] + Fb[d]) for d in range(3)]
    return dict(p=p, Fx=F[0], Fy=F[1], Fz=F[2], Fa_x=Fa[0], Fb_x=Fb[0], Fa_y=Fa[1], Fb_y=Fb[1],
                Fa_z=Fa[2], Fb_z=Fb[2], U=U, P=P)


def solve_mrcm3d(prob, return_leaf_ops=False):
    """O2 in 3D: MMBFs per leaf, the global interface system over patches,
    the final local solves (the steps of oracle.mrcm.GlobalMRCM)."""
    from .mrcm import GlobalMRCM
    g = GlobalMRCM(prob, dec=Decomposition3D(prob), leaf_cls=LeafProblem3D)
    _, U, P = g.solve_system()
    out = assemble_final3d(prob, g.dec, g.leaves, U, P)
    if return_leaf_ops:
        out["leaf_ops"] = [lp.robin_to_flux() for lp in g.leaves]
        out["leaf_segs"] = [lp.segs for lp in g.leaves]
    out["dec"] = g.dec
    return out
