"""Seeded Gaussian random fields by FFT circulant embedding.

The paper's permeability is a log-normal field (Section 5.2, Eq. for the
log-normal K: K = K0 exp(omega_K xi)); its realisation is not published, so
every heterogeneous workload here uses a seeded stand-in: log K = sigma * xi,
xi a zero-mean unit-variance Gaussian field with exponential covariance
exp(-|r|/lambda) (anisotropic lengths allowed), sampled exactly on the grid by
circulant embedding (Dietrich & Newsam, SIAM J. Sci. Comput. 18, 1997).
"""
import numpy as np


def _fft_size(n):
    """Smallest 2^a 3^b 5^c >= n (fast FFT sizes)."""
    best = None
    p2 = 1
    while p2 < 2 * n:
        p3 = p2
        while p3 < 2 * n:
            p5 = p3
            while p5 < 2 * n:
                if p5 >= n and (best is None or p5 < best):
                    best = p5
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return best


def gaussian_random_field(nx, ny, hx, hy, corr, seed):
    """Zero-mean unit-variance field on an ny x nx cell-centred grid.

    corr is a scalar or (lx, ly) correlation-length pair for the covariance
    C(dx, dy) = exp(-sqrt((dx/lx)^2 + (dy/ly)^2)).  The periodic embedding has
    at least 2n points per axis plus the correlation length; negative
    eigenvalues of the embedding are clipped to zero (the clipped fraction is
    returned so callers can report it).  Returns (xi[ny, nx], clipped_frac).
    """
    lx, ly = (corr, corr) if np.isscalar(corr) else corr
    px = _fft_size(2 * nx + int(np.ceil(lx / hx)))
    py = _fft_size(2 * ny + int(np.ceil(ly / hy)))
    ix = np.arange(px)
    iy = np.arange(py)
    dx = np.minimum(ix, px - ix) * hx
    dy = np.minimum(iy, py - iy) * hy
    r = np.sqrt((dx[None, :] / lx) ** 2 + (dy[:, None] / ly) ** 2)
    c = np.exp(-r)
    lam = np.real(np.fft.fft2(c))
    neg = lam < 0
    clipped = float(-lam[neg].sum() / np.abs(lam).sum()) if neg.any() else 0.0
    lam = np.where(neg, 0.0, lam)
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((py, px)) + 1j * rng.standard_normal((py, px))
    w = np.sqrt(lam / (px * py)) * z
    xi = np.real(np.fft.fft2(w))[:ny, :nx]
    return np.ascontiguousarray(xi, dtype=np.float64), clipped


def lognormal_permeability(nx, ny, hx, hy, sigma2, corr, seed):
    """K = exp(sigma * xi) on an ny x nx grid (x fastest when flattened)."""
    xi, _ = gaussian_random_field(nx, ny, hx, hy, corr, seed)
    return np.exp(np.sqrt(sigma2) * xi)


def gaussian_random_field_3d(n, h, corr, seed):
    """Zero-mean unit-variance field on an nz x ny x nx cell-centred grid.

    n = (nx, ny, nz), h = (hx, hy, hz), corr = (lx, ly, lz) correlation
    lengths of C(d) = exp(-sqrt(sum_d (d_d / l_d)^2)); the same circulant
    embedding as the 2D generator, one axis more.  Returns (xi, clipped)."""
    sizes = [_fft_size(2 * n[d] + int(np.ceil(corr[d] / h[d]))) for d in range(3)]
    r2 = 0.0
    for d in range(3):
        i = np.arange(sizes[d])
        dist = np.minimum(i, sizes[d] - i) * h[d] / corr[d]
        shape = [1, 1, 1]
        shape[2 - d] = sizes[d]            # array axes are (z, y, x)
        r2 = r2 + (dist ** 2).reshape(shape)
    c = np.exp(-np.sqrt(r2))
    lam = np.real(np.fft.fftn(c))
    neg = lam < 0
    clipped = float(-lam[neg].sum() / np.abs(lam).sum()) if neg.any() else 0.0
    lam = np.where(neg, 0.0, lam)
    rng = np.random.default_rng(seed)
    shape = lam.shape
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    w = np.sqrt(lam / lam.size) * z
    xi = np.real(np.fft.fftn(w))[:n[2], :n[1], :n[0]]
    return np.ascontiguousarray(xi, dtype=np.float64), clipped


def lognormal_permeability_3d(n, h, sigma2, corr, seed):
    """K = exp(sigma * xi) on an nz x ny x nx grid (x fastest when flattened)."""
    xi, _ = gaussian_random_field_3d(n, h, corr, seed)
    return np.exp(np.sqrt(sigma2) * xi)
