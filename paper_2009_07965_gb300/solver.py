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
