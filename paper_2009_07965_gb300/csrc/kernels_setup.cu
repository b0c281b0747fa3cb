// Permeability check, Robin coefficients and face coefficients (build step 1).
//
// Robin coefficient per segment t, Eqs. (robin.beta) and (permeff) of
// arXiv 2009.07965 (Section 5.1):
//     Keff_t = (1/N) sum_{e in t} 2 K_a K_b / (K_a + K_b),
//     beta_t = alpha * Hbar_t / Keff_t,   Hbar_t = |t| (segment length),
// and the coupling of the two Robin sides D_t = |t| / (2 beta_t).
//
// Face coefficients of the lumped RT0 (two-point flux) local operators,
// seen from each of the two cells of a face, with r_c = h/(2K_c):
//     interior face:   T   = |e| / (r_a + r_b)                 (both sides)
//     skeleton face:   rho = |e| / (r_c + beta_t)              (Eq. 11.2, lumped)
//     Dirichlet face:  tau = 2 K_c |e| / h,   Neumann face: 0.
// Each coefficient is evaluated in this order (no fused operations); the
// quotients of the cell and interior / skeleton face terms are products with
// a reciprocal within an ulp (rcp_nr: an FP64 division costs about ten FP64
// instructions on this part, and these kernels are bound by them), so the
// discrete system agrees with the plain quotients to a few ulps.
#include "mrcm_internal.h"

namespace mrcm {
namespace {

__global__ void check_K_kernel(const double* __restrict__ K, long long n, int* status) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < n; i += stride) {
        double k = K[i];
        // k > 0 is false for NaN; the upper bound rejects +inf
        bad |= !(k > 0.0 && k < 1.0e300);
    }
    if (bad) atomicOr(status, kStatusBadK);
}

// Half-cell resistances r = h_d / (2 K_c), the building block of every face
// coefficient below (evaluated once per cell, in this order).
__global__ void cell_resist_kernel(DevView v) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= v.ncell) return;
    const GridDesc& G = v.grids[grid_of<0>(v, c)];
    const double rk = rcp_nr(2.0 * v.K[c]);
    v.rx[c] = G.hx * rk;
    v.ry[c] = G.hy * rk;
}

__global__ void seg_beta_kernel(DevView v) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.nseg) return;
    const int axis = v.seg_axis[t], line = v.seg_line[t], lo = v.seg_lo[t], len = v.seg_len[t];
    const GridDesc& G = v.grids[v.seg_grid[t]];
    const double* K = v.K + G.c0;
    double sum = 0.0;
    for (int e = 0; e < len; ++e) {
        double ka, kb;
        if (axis == 0) {
            const long long row = (long long)(lo + e) * G.nx;
            ka = K[row + line - 1];
            kb = K[row + line];
        } else {
            ka = K[(long long)(line - 1) * G.nx + lo + e];
            kb = K[(long long)line * G.nx + lo + e];
        }
        sum += 2.0 * ka * kb / (ka + kb);
    }
    const double keff = sum / len;
    const double length = len * (axis == 0 ? G.hy : G.hx);
    v.seg_beta[t] = v.alpha * length / keff;
    // D = |t| / (2 beta) = Keff / (2 alpha)
    v.seg_D[t] = keff / (2.0 * v.alpha);
}

__global__ void face_coef_kernel(DevView v) {
    long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (f < v.nxface) {
        const GridDesc& G = v.grids[grid_of<1>(v, f)];
        int i, j;
        udivmod(f - G.fx0, G.nx + 1, j, i);
        const double area = G.hy, hn = G.hx;
        const long long row = G.c0 + (long long)j * G.nx;
        double cl = 0.0, cu = 0.0;
        if (i == 0) {
            if (G.bc[0]) cu = 2.0 * v.K[row] * area / hn;
        } else if (i == G.nx) {
            if (G.bc[1]) cl = 2.0 * v.K[row + G.nx - 1] * area / hn;
        } else {
            const double ra = v.rx[row + i - 1], rb = v.rx[row + i];
            const int t = v.xface_seg[f];
            if (t >= 0) {
                const double beta = v.seg_beta[t];
                cl = area * rcp_nr(ra + beta);
                cu = area * rcp_nr(rb + beta);
            } else {
                cl = cu = area * rcp_nr(ra + rb);
            }
        }
        v.cxL[f] = cl;
        v.cxU[f] = cu;
        return;
    }
    f -= v.nxface;
    if (f < v.nyface) {
        const GridDesc& G = v.grids[grid_of<2>(v, f)];
        int i, j;
        udivmod(f - G.fy0, G.nx, j, i);
        const double area = G.hx, hn = G.hy;
        const double* K = v.K + G.c0;
        double cl = 0.0, cu = 0.0;
        if (j == 0) {
            if (G.bc[2]) cu = 2.0 * K[i] * area / hn;
        } else if (j == G.ny) {
            if (G.bc[3]) cl = 2.0 * K[(long long)(G.ny - 1) * G.nx + i] * area / hn;
        } else {
            const double ra = v.ry[G.c0 + (long long)(j - 1) * G.nx + i], rb = v.ry[G.c0 + (long long)j * G.nx + i];
            const int t = v.yface_seg[f];
            if (t >= 0) {
                const double beta = v.seg_beta[t];
                cl = area * rcp_nr(ra + beta);
                cu = area * rcp_nr(rb + beta);
            } else {
                cl = cu = area * rcp_nr(ra + rb);
            }
        }
        v.cyL[f] = cl;
        v.cyU[f] = cu;
    }
}

__global__ void reciprocal_kernel(const double* __restrict__ x, double* __restrict__ r, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = rcp_nr(x[i]);
}

}  // namespace

cudaError_t launch_reciprocal(const double* x, double* r, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    reciprocal_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, r, n);
    return cudaGetLastError();
}

cudaError_t launch_check_K(const DevView& v, cudaStream_t s) {
    const long long n = v.ncell;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    check_K_kernel<<<blocks, 256, 0, s>>>(v.K, n, v.status);
    return cudaGetLastError();
}

cudaError_t launch_cell_resist(const DevView& v, cudaStream_t s) {
    const long long n = v.ncell;
    cell_resist_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_seg_beta(const DevView& v, cudaStream_t s) {
    if (v.nseg == 0) return cudaSuccess;
    seg_beta_kernel<<<(v.nseg + 127) / 128, 128, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_face_coef(const DevView& v, cudaStream_t s) {
    const long long nf = v.nxface + v.nyface;
    face_coef_kernel<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(v);
    return cudaGetLastError();
}

}  // namespace mrcm
