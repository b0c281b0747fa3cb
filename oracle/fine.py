"""O1: fine-scale mixed solve (lumped RT0 = two-point flux), sparse direct.

Eqs. (ellip.1)-(ellip.3): div u = f, u = -K grad p, p = g_D on the
Dirichlet boundary, u.n = g_N on the Neumann boundary.  The paper
discretises with lowest-order Raviart-Thomas elements, stated equivalent to
conservative finite volumes, and reduces the system to one for the pressure
(Section 2.2 and the implementation paragraph of Section 4).  On a Cartesian
grid with the trapezoidal (lumped) velocity mass matrix that is the
two-point flux scheme:

  interior face e between cells c, c' (normal axis d):
      F_e = T_e (p_c - p_c'),   T_e = |e| / (h_d/(2K_c) + h_d/(2K_c'))
  Dirichlet face:  outward F = tau_e (p_c - g_D),  tau_e = 2 K_c |e| / h_d
  Neumann face:    outward F = |e| g_N
  cell balance:    sum of outward face fluxes = q_c   (q = integrated f)

Fluxes are integrated over the face (per unit depth) and signed positive
in the +axis direction.  For a pure-Neumann problem the equation of cell 0
is replaced by p_0 = 0 and the pressure is then shifted to zero mean.
This is the accuracy reference of Section 5.4, not the parity target.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from inputs.problems import DIRICHLET


def solve_fine(prob):
    nx, ny, hx, hy = prob.nx, prob.ny, prob.hx, prob.hy
    K = prob.K
    n = nx * ny
    idx = lambda i, j: i + nx * j
    rows, cols, vals = [], [], []
    rhs = prob.q.reshape(-1).astype(np.float64).copy()
    diag = np.zeros(n)
    bcs = prob.bc_slices()
    g = prob.bc_val
    # interior x faces
    Tx = np.zeros((ny, nx + 1))
    for j in range(ny):
        for i in range(1, nx):
            Tx[j, i] = hy / (hx / (2 * K[j, i - 1]) + hx / (2 * K[j, i]))
    Ty = np.zeros((ny + 1, nx))
    for j in range(1, ny):
        for i in range(nx):
            Ty[j, i] = hx / (hy / (2 * K[j - 1, i]) + hy / (2 * K[j, i]))
    for j in range(ny):
        for i in range(1, nx):
            c, c2, T = idx(i - 1, j), idx(i, j), Tx[j, i]
            diag[c] += T; diag[c2] += T
            rows += [c, c2]; cols += [c2, c]; vals += [-T, -T]
    for j in range(1, ny):
        for i in range(nx):
            c, c2, T = idx(i, j - 1), idx(i, j), Ty[j, i]
            diag[c] += T; diag[c2] += T
            rows += [c, c2]; cols += [c2, c]; vals += [-T, -T]
    # boundary faces: side -> list of (cell, |e|, h_normal, value)
    tau = {}
    for side in range(4):
        vals_side = g[bcs[side]]
        if side < 2:
            i = 0 if side == 0 else nx - 1
            cells = [(i, j) for j in range(ny)]
            area, hn = hy, hx
        else:
            j = 0 if side == 2 else ny - 1
            cells = [(i, j) for i in range(nx)]
            area, hn = hx, hy
        for k, (i, j) in enumerate(cells):
            c = idx(i, j)
            if prob.bc_type[side] == DIRICHLET:
                t = 2.0 * K[j, i] * area / hn
                diag[c] += t
                rhs[c] += t * vals_side[k]
                tau[(side, k)] = t
            else:
                rhs[c] -= area * vals_side[k]
    rows += list(range(n)); cols += list(range(n)); vals += list(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    if prob.pure_neumann:
        A = A.tolil()
        A[0, :] = 0.0
        A[0, 0] = 1.0
        A = A.tocsr()
        rhs[0] = 0.0
    p = spla.spsolve(A.tocsc(), rhs)
    if prob.pure_neumann:
        p = p - p.mean()
    P = p.reshape(ny, nx)
    Fx = np.zeros((ny, nx + 1))
    Fy = np.zeros((ny + 1, nx))
    Fx[:, 1:nx] = Tx[:, 1:nx] * (P[:, :-1] - P[:, 1:])
    Fy[1:ny, :] = Ty[1:ny, :] * (P[:-1, :] - P[1:, :])
    for side in range(4):
        vals_side = g[bcs[side]]
        for k in range(ny if side < 2 else nx):
            if side == 0:
                j, i, area = k, 0, hy
            elif side == 1:
                j, i, area = k, nx - 1, hy
            elif side == 2:
                j, i, area = 0, k, hx
            else:
                j, i, area = ny - 1, k, hx
            if prob.bc_type[side] == DIRICHLET:
                out = tau[(side, k)] * (P[j, i] - vals_side[k])
            else:
                out = area * vals_side[k]
            if side == 0:
                Fx[j, 0] = -out
            elif side == 1:
                Fx[j, nx] = out
            elif side == 2:
                Fy[0, i] = -out
            else:
                Fy[ny, i] = out
    return dict(p=P, Fx=Fx, Fy=Fy, A=A, rhs=rhs)
