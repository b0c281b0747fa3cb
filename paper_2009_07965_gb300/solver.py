"""Convenience wrapper: owns a context and the output tensors (torch, cuda)."""
import torch

from . import binding as B


class Solver:
    """Recursive MRCM solver for one grid / decomposition / alpha / BC types.

    K: (ny, nx) float64 CUDA tensor.  bc_type: (x-, x+, y-, y+).
    precision: binding.MRCM_FP64 or binding.MRCM_MIXED.
    """

    def __init__(self, K, Lx=1.0, Ly=1.0, sub=(16, 16), seg=(4, 4), alpha=1.0,
                 bc_type=(1, 1, 0, 0), stream=None, precision=B.MRCM_FP64):
        if not (K.is_cuda and K.dtype == torch.float64):
            raise TypeError("K must be a float64 CUDA tensor")
        self.ny, self.nx = K.shape
        self.stream = stream if stream is not None else torch.cuda.current_stream(K.device)
        self.device = K.device
        self.ctx = B.mrcm_setup((self.nx, self.ny), (Lx, Ly), K.contiguous(), sub, seg, alpha,
                                bc_type, precision, self.stream.cuda_stream)
        dev = self.device
        self.p = torch.empty(self.ny, self.nx, dtype=torch.float64, device=dev)
        self.Fx = torch.empty(self.ny, self.nx + 1, dtype=torch.float64, device=dev)
        self.Fy = torch.empty(self.ny + 1, self.nx, dtype=torch.float64, device=dev)
        self.iface = None

    def set_permeability(self, K):
        B.mrcm_set_permeability(self.ctx, K.contiguous())

    def build_basis(self):
        B.mrcm_build_basis(self.ctx)

    def solve(self, q, bc_val, want_iface=False):
        if want_iface and self.iface is None:
            n = (self.nx + 1) * self.ny + self.nx * (self.ny + 1)
            self.iface = torch.empty(2 * n, dtype=torch.float64, device=self.device)
        B.mrcm_solve(self.ctx, q.contiguous(), bc_val.contiguous(), self.p, self.Fx, self.Fy, None,
                     self.iface if want_iface else None)
        return self.p, self.Fx, self.Fy

    def iface_parts(self):
        """Split the one-sided flux output into Fa_x, Fb_x, Fa_y, Fb_y."""
        nx, ny = self.nx, self.ny
        nxf, nyf = (nx + 1) * ny, nx * (ny + 1)
        f = self.iface
        return (f[:nxf].view(ny, nx + 1), f[nxf:2 * nxf].view(ny, nx + 1),
                f[2 * nxf:2 * nxf + nyf].view(ny + 1, nx), f[2 * nxf + nyf:].view(ny + 1, nx))

    def query(self, what):
        return B.mrcm_query(self.ctx, what)

    def close(self):
        if self.ctx:
            B.mrcm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver3D:
    """Recursive MRCM solver for one 3D grid: blocks of the patch shape seg,
    subdomains sub, one patch per seg-sized side between subdomains.
    precision: MRCM_FP64, or MRCM_MIXED (FP32 merges, FP64 blocks and
    refinement).

    K: (nz, ny, nx) float64 CUDA tensor.  bc_type: (x-, x+, y-, y+, z-, z+)
    (all Neumann: zero-mean pressure).  solve() returns p (nz, ny, nx), Fx
    (nz, ny, nx+1), Fy (nz, ny+1, nx), Fz (nz+1, ny, nx).
    """

    def __init__(self, K, L=(1.0, 1.0, 1.0), sub=(16, 16, 16), seg=(4, 4, 4), alpha=1.0,
                 bc_type=(1, 1, 0, 0, 0, 0), stream=None, precision=B.MRCM_FP64):
        if not (K.is_cuda and K.dtype == torch.float64 and K.dim() == 3):
            raise TypeError("K must be a 3D float64 CUDA tensor")
        self.nz, self.ny, self.nx = K.shape
        self.stream = stream if stream is not None else torch.cuda.current_stream(K.device)
        self.device = K.device
        self.ctx = B.mrcm_setup((self.nx, self.ny, self.nz), L, K.contiguous(), sub, seg, alpha,
                                bc_type, precision, self.stream.cuda_stream)
        dev, nx, ny, nz = self.device, self.nx, self.ny, self.nz
        self.p = torch.empty(nz, ny, nx, dtype=torch.float64, device=dev)
        self.Fx = torch.empty(nz, ny, nx + 1, dtype=torch.float64, device=dev)
        self.Fy = torch.empty(nz, ny + 1, nx, dtype=torch.float64, device=dev)
        self.Fz = torch.empty(nz + 1, ny, nx, dtype=torch.float64, device=dev)

    def set_permeability(self, K):
        B.mrcm_set_permeability(self.ctx, K.contiguous())

    def build_basis(self):
        B.mrcm_build_basis(self.ctx)

    def solve(self, q, bc_val, want_iface=False):
        if want_iface and getattr(self, "iface", None) is None:
            n = self.Fx.numel() + self.Fy.numel() + self.Fz.numel()
            self.iface = torch.empty(2 * n, dtype=torch.float64, device=self.device)
        B.mrcm_solve(self.ctx, q.contiguous(), bc_val.contiguous(), self.p, self.Fx, self.Fy, self.Fz,
                     self.iface if want_iface else None)
        return self.p, self.Fx, self.Fy, self.Fz

    def iface_parts(self):
        """The one-sided flux output as Fa_x, Fb_x, Fa_y, Fb_y, Fa_z, Fb_z."""
        out, off = [], 0
        for F in (self.Fx, self.Fy, self.Fz):
            n = F.numel()
            out += [self.iface[off:off + n].view(F.shape), self.iface[off + n:off + 2 * n].view(F.shape)]
            off += 2 * n
        return tuple(out)

    def query(self, what):
        return B.mrcm_query(self.ctx, what)

    def close(self):
        if self.ctx:
            B.mrcm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """One context for several independent problems (mrcm_setup_batch): the
    build and every solve run all of them together, one launch per tree
    height over all their trees.

    Ks: list of (ny_k, nx_k) float64 CUDA tensors; Ls: list of (Lx, Ly);
    bc_types: list of (x-, x+, y-, y+).  solve() takes lists of q and bc_val
    tensors and returns lists of (p, Fx, Fy) views into the packed outputs.
    """

    def __init__(self, Ks, Ls, bc_types, sub=(16, 16), seg=(4, 4), alpha=1.0, stream=None,
                 precision=B.MRCM_FP64):
        if not all(K.is_cuda and K.dtype == torch.float64 for K in Ks):
            raise TypeError("every K must be a float64 CUDA tensor")
        self.shapes = [tuple(K.shape) for K in Ks]
        dev = Ks[0].device
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.K = torch.cat([K.reshape(-1) for K in Ks])
        ns = [(nx, ny) for (ny, nx) in self.shapes]
        self.ctx = B.mrcm_setup_batch(ns, Ls, bc_types, self.K, sub, seg, alpha, precision,
                                      self.stream.cuda_stream)
        self.ncell = sum(nx * ny for nx, ny in ns)
        self.nxf = sum((nx + 1) * ny for nx, ny in ns)
        self.nyf = sum(nx * (ny + 1) for nx, ny in ns)
        self.p = torch.empty(self.ncell, dtype=torch.float64, device=dev)
        self.Fx = torch.empty(self.nxf, dtype=torch.float64, device=dev)
        self.Fy = torch.empty(self.nyf, dtype=torch.float64, device=dev)
        self.iface = None

    def pack(self, arrays):
        """Concatenate per-problem tensors in problem order."""
        return torch.cat([a.reshape(-1) for a in arrays])

    def set_permeability(self, Ks):
        self.K.copy_(self.pack(Ks))
        B.mrcm_set_permeability(self.ctx, self.K)

    def build_basis(self):
        B.mrcm_build_basis(self.ctx)

    def solve_packed(self, q, bc_val, want_iface=False):
        """q, bc_val already packed (problem after problem)."""
        if want_iface and self.iface is None:
            self.iface = torch.empty(2 * (self.nxf + self.nyf), dtype=torch.float64, device=self.device)
        B.mrcm_solve(self.ctx, q, bc_val, self.p, self.Fx, self.Fy, None, self.iface if want_iface else None)
        return self.p, self.Fx, self.Fy

    def solve(self, qs, bc_vals, want_iface=False):
        self.solve_packed(self.pack(qs), self.pack(bc_vals), want_iface)
        return self.split()

    def split(self):
        """Per-problem (p, Fx, Fy) views of the packed outputs."""
        out = []
        c = fx = fy = 0
        for ny, nx in self.shapes:
            out.append((self.p[c:c + nx * ny].view(ny, nx), self.Fx[fx:fx + (nx + 1) * ny].view(ny, nx + 1),
                        self.Fy[fy:fy + nx * (ny + 1)].view(ny + 1, nx)))
            c += nx * ny
            fx += (nx + 1) * ny
            fy += nx * (ny + 1)
        return out

    def iface_split(self):
        """Per-problem (Fa_x, Fb_x, Fa_y, Fb_y) views of the one-sided fluxes."""
        f = self.iface
        parts = [f[:self.nxf], f[self.nxf:2 * self.nxf], f[2 * self.nxf:2 * self.nxf + self.nyf],
                 f[2 * self.nxf + self.nyf:]]
        out = []
        fx = fy = 0
        for ny, nx in self.shapes:
            out.append((parts[0][fx:fx + (nx + 1) * ny].view(ny, nx + 1),
                        parts[1][fx:fx + (nx + 1) * ny].view(ny, nx + 1),
                        parts[2][fy:fy + nx * (ny + 1)].view(ny + 1, nx),
                        parts[3][fy:fy + nx * (ny + 1)].view(ny + 1, nx)))
            fx += (nx + 1) * ny
            fy += nx * (ny + 1)
        return out

    def query(self, what):
        return B.mrcm_query(self.ctx, what)

    def close(self):
        if self.ctx:
            B.mrcm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
