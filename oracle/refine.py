"""Residual of the discrete MRCM equations and iterative refinement (oracle).

The discrete MRCM solution is defined by Eqs. (11.2)-(14.2) with lumped RT0
(see oracle.local).  Eliminating the skeleton face fluxes with the lumped
Robin relation of Eq. (11.2),
    F^i_e = rho_e (p_c - lambda^i_t),  lambda^a_t = P_t - beta_t U_t,
                                       lambda^b_t = P_t + beta_t U_t
(side a = lower leaf, n_t . n^a = +1), leaves the unknowns (p, P, U) and
    E_c    = sum of the outward fluxes of cell c - q_c            (Eq. 12.2)
    E13_t  = F^a_t + F^b_t                                          (Eq. 13.2)
    E14_t  = F^a_t - F^b_t - 2 |t| U_t                              (Eq. 14.2)
with F^i_t = sum_{e in t} F^i_e.  The coefficients are evaluated in float64
in this fixed order, which defines the discrete system exactly:
    r_c    = h_d / (2 K_c)                       (half-cell resistance)
    T_e    = |e| / (r_c + r_c')                  (interior face)
    rho_e  = |e| / (r_c + beta_t)                (skeleton face, its cell c)
    tau_e  = 2 K_c |e| / h_d                     (Dirichlet face)
    beta_t = alpha |t| / Keff_t,  Keff_t = (sum_e 2 K_a K_b / (K_a + K_b)) / N.
The refined state is kept as double-double pairs (x_hi + x_lo): E is
evaluated in double-double arithmetic (oracle.dd) from that state, every
correction is added in double-double, and the output pressures and fluxes
are formed in double-double and rounded once, so they are the discrete
solution rounded to float64 (to within about one ulp) even where a flux is
the small difference of two large pressures.
"""
import numpy as np

from inputs.problems import DIRICHLET
from .dd import dd_add, dd_mul_d, two_prod, two_sum


def coefficients(prob, dec):
    K, hx, hy = prob.K, prob.hx, prob.hy
    c = {}
    c["rx"] = hx / (2 * K)
    c["ry"] = hy / (2 * K)
    c["Tx"] = hy / (c["rx"][:, :-1] + c["rx"][:, 1:])        # x-faces 1..nx-1
    c["Ty"] = hx / (c["ry"][:-1, :] + c["ry"][1:, :])        # y-faces 1..ny-1
    c["beta"] = np.array([t["beta"] for t in dec.segments])
    c["length"] = np.array([t["length"] for t in dec.segments])
    return c


def _segment_faces(prob, dec, c):
    """Arrays over all skeleton faces: cell a (j, i), cell b, segment, rho^a, rho^b."""
    ja, ia, jb, ib, seg, ra, rb = [], [], [], [], [], [], []
    for t in dec.segments:
        beta = t["beta"]
        for (ca, cb) in dec.face_cells(t):
            ja.append(ca[0]); ia.append(ca[1]); jb.append(cb[0]); ib.append(cb[1])
            seg.append(t["id"])
    ja, ia, jb, ib, seg = map(np.array, (ja, ia, jb, ib, seg))
    if len(seg) == 0:
        return None
    axis = np.array([dec.segments[t]["axis"] for t in seg])
    area = np.where(axis == 0, prob.hy, prob.hx)
    r_a = np.where(axis == 0, c["rx"][ja, ia], c["ry"][ja, ia])
    r_b = np.where(axis == 0, c["rx"][jb, ib], c["ry"][jb, ib])
    beta = c["beta"][seg]
    return dict(ja=ja, ia=ia, jb=jb, ib=ib, seg=seg, axis=axis,
                rho_a=area / (r_a + beta), rho_b=area / (r_b + beta))


def _boundary_terms(prob, c):
    """(j, i, outward flux as function of p) descriptors of boundary faces."""
    out = []
    bcs = prob.bc_slices()
    nx, ny, K = prob.nx, prob.ny, prob.K
    for side in range(4):
        g = prob.bc_val[bcs[side]]
        if side < 2:
            i = 0 if side == 0 else nx - 1
            js, is_ = np.arange(ny), np.full(ny, i)
            area, hn = prob.hy, prob.hx
        else:
            j = 0 if side == 2 else ny - 1
            js, is_ = np.full(nx, j), np.arange(nx)
            area, hn = prob.hx, prob.hy
        if prob.bc_type[side] == DIRICHLET:
            tau = 2.0 * K[js, is_] * area / hn
            out.append(("dir", side, js, is_, tau, g))
        else:
            out.append(("neu", side, js, is_, area, g))
    return out


def _dd_sub(ah, al, bh, bl):
    return dd_add(ah, al, -bh, -bl)


def residual(prob, dec, state):
    """(E_cell[ny, nx], E13[nseg], E14[nseg]) rounded to float64, for the
    double-double state (ph, pl, Uh, Ul, Ph, Pl)."""
    ph, pl, Uh, Ul, Ph, Pl = state
    c = coefficients(prob, dec)
    nx, ny = prob.nx, prob.ny
    eh = np.zeros((ny, nx)); el = np.zeros((ny, nx))
    # interior faces (not on the skeleton): flux out of the lower cell
    skx = dec.xface_seg[:, 1:nx] >= 0
    dh, dl = _dd_sub(ph[:, :-1], pl[:, :-1], ph[:, 1:], pl[:, 1:])
    fh, fl = dd_mul_d(dh, dl, c["Tx"])
    fh = np.where(skx, 0.0, fh); fl = np.where(skx, 0.0, fl)
    eh[:, :-1], el[:, :-1] = dd_add(eh[:, :-1], el[:, :-1], fh, fl)
    eh[:, 1:], el[:, 1:] = dd_add(eh[:, 1:], el[:, 1:], -fh, -fl)
    sky = dec.yface_seg[1:ny, :] >= 0
    dh, dl = _dd_sub(ph[:-1, :], pl[:-1, :], ph[1:, :], pl[1:, :])
    fh, fl = dd_mul_d(dh, dl, c["Ty"])
    fh = np.where(sky, 0.0, fh); fl = np.where(sky, 0.0, fl)
    eh[:-1, :], el[:-1, :] = dd_add(eh[:-1, :], el[:-1, :], fh, fl)
    eh[1:, :], el[1:, :] = dd_add(eh[1:, :], el[1:, :], -fh, -fl)
    # boundary faces
    for kind, side, js, is_, coef, g in _boundary_terms(prob, c):
        if kind == "dir":
            dh, dl = dd_add(ph[js, is_], pl[js, is_], -g, np.zeros(len(g)))
            fh, fl = dd_mul_d(dh, dl, coef)
        else:
            fh, fl = two_prod(np.full(len(g), coef), g)
        eh[js, is_], el[js, is_] = dd_add(eh[js, is_], el[js, is_], fh, fl)
    # skeleton faces
    nseg = len(dec.segments)
    fah = np.zeros(nseg); fal = np.zeros(nseg); fbh = np.zeros(nseg); fbl = np.zeros(nseg)
    sf = _segment_faces(prob, dec, c)
    if sf is not None:
        s = sf["seg"]
        bh, bl = dd_mul_d(Uh[s], Ul[s], c["beta"][s])         # beta U
        # p_a - lambda^a = p_a - P + beta U ;  p_b - lambda^b = p_b - P - beta U
        xh, xl = _dd_sub(ph[sf["ja"], sf["ia"]], pl[sf["ja"], sf["ia"]], Ph[s], Pl[s])
        xh, xl = dd_add(xh, xl, bh, bl)
        fah_e, fal_e = dd_mul_d(xh, xl, sf["rho_a"])
        yh, yl = _dd_sub(ph[sf["jb"], sf["ib"]], pl[sf["jb"], sf["ib"]], Ph[s], Pl[s])
        yh, yl = dd_add(yh, yl, -bh, -bl)
        fbh_e, fbl_e = dd_mul_d(yh, yl, sf["rho_b"])
        # cell sums (a cell may touch two skeleton faces: accumulate in order)
        for k in range(len(s)):
            ja, ia, jb, ib = sf["ja"][k], sf["ia"][k], sf["jb"][k], sf["ib"][k]
            eh[ja, ia], el[ja, ia] = dd_add(eh[ja, ia], el[ja, ia], fah_e[k], fal_e[k])
            eh[jb, ib], el[jb, ib] = dd_add(eh[jb, ib], el[jb, ib], fbh_e[k], fbl_e[k])
            fah[s[k]], fal[s[k]] = dd_add(fah[s[k]], fal[s[k]], fah_e[k], fal_e[k])
            fbh[s[k]], fbl[s[k]] = dd_add(fbh[s[k]], fbl[s[k]], fbh_e[k], fbl_e[k])
    eh, el = dd_add(eh, el, -prob.q, np.zeros_like(prob.q))
    e13h, e13l = dd_add(fah, fal, fbh, fbl)
    uh, ul = dd_mul_d(Uh, Ul, 2.0 * c["length"])
    e14h, e14l = dd_add(fah, fal, -fbh, -fbl)
    e14h, e14l = dd_add(e14h, e14l, -uh, -ul)
    return eh + el, e13h + e13l, e14h + e14l


def refine_solution(prob, dec, solve_system, p, U, P, iters):
    """Wilkinson iterative refinement with the state kept in double-double:
    x += solve(-E(x)), `iters` times.  Returns the double-double state
    (ph, pl, Uh, Ul, Ph, Pl) and the history of max |E| per evaluation."""
    state = [p, np.zeros_like(p), U, np.zeros_like(U), P, np.zeros_like(P)]
    hist = []

    def evaluate():
        Ec, E13, E14 = residual(prob, dec, state)
        hist.append(float(max(np.abs(Ec).max(), np.abs(E13).max() if len(E13) else 0.0,
                              np.abs(E14).max() if len(E14) else 0.0)))
        return Ec, E13, E14

    for _ in range(iters):
        Ec, E13, E14 = evaluate()
        dp, dU, dP = solve_system(with_bc=False, source=-Ec, rhs13=-E13, rhs14=-E14)
        state[0], state[1] = dd_add(state[0], state[1], dp, np.zeros_like(dp))
        state[2], state[3] = dd_add(state[2], state[3], dU, np.zeros_like(dU))
        state[4], state[5] = dd_add(state[4], state[5], dP, np.zeros_like(dP))
    evaluate()
    return tuple(state), hist


def shift_mean(prob, state):
    """Zero-mean pressure (all-Neumann problems): subtract the mean of the
    rounded cell pressures from p and P, in double-double."""
    ph, pl, Uh, Ul, Ph, Pl = state
    pr = ph + pl
    shift = (pr * (prob.hx * prob.hy)).sum() / (prob.hx * prob.hy * prob.nx * prob.ny)
    ph, pl = dd_add(ph, pl, np.full_like(ph, -shift), np.zeros_like(ph))
    Ph, Pl = dd_add(Ph, Pl, np.full_like(Ph, -shift), np.zeros_like(Ph))
    return ph, pl, Uh, Ul, Ph, Pl


def fluxes_from_state(prob, dec, state):
    """Cell pressures and face fluxes (+axis direction) from the
    double-double state by the face relations, each formed in double-double
    and rounded once."""
    ph, pl, Uh, Ul, Ph, Pl = state
    c = coefficients(prob, dec)
    nx, ny = prob.nx, prob.ny
    Fx = np.zeros((ny, nx + 1)); Fy = np.zeros((ny + 1, nx))
    dh, dl = _dd_sub(ph[:, :-1], pl[:, :-1], ph[:, 1:], pl[:, 1:])
    fh, fl = dd_mul_d(dh, dl, c["Tx"])
    Fx[:, 1:nx] = fh + fl
    dh, dl = _dd_sub(ph[:-1, :], pl[:-1, :], ph[1:, :], pl[1:, :])
    fh, fl = dd_mul_d(dh, dl, c["Ty"])
    Fy[1:ny, :] = fh + fl
    for kind, side, js, is_, coef, g in _boundary_terms(prob, c):
        if kind == "dir":
            dh, dl = dd_add(ph[js, is_], pl[js, is_], -g, np.zeros(len(g)))
            fh, fl = dd_mul_d(dh, dl, coef)
            out = fh + fl
        else:
            out = coef * g
        if side == 0:
            Fx[js, 0] = -out
        elif side == 1:
            Fx[js, nx] = out
        elif side == 2:
            Fy[0, is_] = -out
        else:
            Fy[ny, is_] = out
    Fa_x, Fb_x, Fa_y, Fb_y = Fx.copy(), Fx.copy(), Fy.copy(), Fy.copy()
    sf = _segment_faces(prob, dec, c)
    if sf is not None:
        s = sf["seg"]
        bh, bl = dd_mul_d(Uh[s], Ul[s], c["beta"][s])
        xh, xl = _dd_sub(ph[sf["ja"], sf["ia"]], pl[sf["ja"], sf["ia"]], Ph[s], Pl[s])
        xh, xl = dd_add(xh, xl, bh, bl)
        fah, fal = dd_mul_d(xh, xl, sf["rho_a"])               # outward of a = +axis
        yh, yl = _dd_sub(ph[sf["jb"], sf["ib"]], pl[sf["jb"], sf["ib"]], Ph[s], Pl[s])
        yh, yl = dd_add(yh, yl, -bh, -bl)
        fbh, fbl = dd_mul_d(yh, yl, sf["rho_b"])               # outward of b = -axis
        fa, fb = fah + fal, -(fbh + fbl)
        mh, ml = dd_add(fah, fal, -fbh, -fbl)
        fm = 0.5 * (mh + ml)
        x = sf["axis"] == 0
        Fa_x[sf["jb"][x], sf["ib"][x]] = fa[x]
        Fb_x[sf["jb"][x], sf["ib"][x]] = fb[x]
        Fa_y[sf["jb"][~x], sf["ib"][~x]] = fa[~x]
        Fb_y[sf["jb"][~x], sf["ib"][~x]] = fb[~x]
        Fx[sf["jb"][x], sf["ib"][x]] = fm[x]
        Fy[sf["jb"][~x], sf["ib"][~x]] = fm[~x]
    return dict(p=ph + pl, Fx=Fx, Fy=Fy, Fa_x=Fa_x, Fb_x=Fb_x, Fa_y=Fa_y, Fb_y=Fb_y,
                U=Uh + Ul, P=Ph + Pl)
