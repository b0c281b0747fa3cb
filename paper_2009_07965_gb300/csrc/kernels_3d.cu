// The 3D path: Robin and face coefficients, the leaf blocks' local Robin
// problems and their solve-phase passes, and the face fluxes.
//
// arXiv 2009.07965 runs its experiments in 3D (Section 5.1): box subdomains,
// rectangular interfaces cut into patches of H-bar (Section 4).  The Robin
// coefficient of a segment t is Eq. (robin.beta) with K_eff from Eq.
// (permeff): Keff_t = mean over the faces of t of 2 K_a K_b / (K_a + K_b),
// beta_t = alpha Hbar_t / Keff_t with Hbar_t = sqrt(|t|) (the patch side of
// a square patch), and the Robin coupling D_t = |t| / (2 beta_t).
//
// Leaves.  The grid is tiled by blocks of the patch shape (at most 64
// cells), so a patch between two subdomains is exactly the shared side of
// two blocks.  Inside a subdomain every face between two blocks is its own
// segment: with one unknown pair per fine face the Robin coupling reproduces
// the two-point flux exactly, whatever beta (the one-face-segment property of
// Eqs. 11.2-14.2), so merging the blocks of a subdomain solves its local
// Robin problems exactly -- a nested dissection of the subdomain by the same
// merges that couple subdomains.  A block's local problem (Eqs. 11.2-12.2,
// lumped RT0) is p = A^-1 (bbar + B lambda), its Robin-to-flux map
// R = B^T A^-1 B - W, W_s = sum of rho over the faces of s; with the
// Cholesky factor A = L L^T and Z = L^-1 B: R = Z^T Z - W, rbar = Z^T L^-1
// bbar and p = L^-T (L^-1 bbar + Z lambda).
//
// Mapping: one CTA per block for the factorisation (A and Z in shared
// memory; the banded Cholesky step and the forward solve of every column of Z
// advance together), one warp per block for the solve-phase passes.
#include "mrcm_internal.h"

#include <algorithm>

namespace mrcm {
namespace {

constexpr int kBuild3Threads = 128;
constexpr int kSolve3Warps = 4;          // blocks (one warp each) per CTA in the solve passes

__device__ __forceinline__ long long cell3(const Grid3& G, int i, int j, int k) {
    return ((long long)k * G.ny + j) * G.nx + i;
}
__device__ __forceinline__ long long xface3(const Grid3& G, int i, int j, int k) {
    return ((long long)k * G.ny + j) * (G.nx + 1) + i;
}
__device__ __forceinline__ long long yface3(const Grid3& G, int i, int j, int k) {
    return ((long long)k * (G.ny + 1) + j) * G.nx + i;
}
__device__ __forceinline__ long long zface3(const Grid3& G, int i, int j, int k) {
    return ((long long)k * G.ny + j) * G.nx + i;
}
__device__ __forceinline__ double area3(const Grid3& G, int d) {
    return d == 0 ? G.hy * G.hz : (d == 1 ? G.hx * G.hz : G.hx * G.hy);
}
__device__ __forceinline__ double hnorm3(const Grid3& G, int d) {
    return d == 0 ? G.hx : (d == 1 ? G.hy : G.hz);
}

// beta_t and D_t of every segment (faces: v outer along the second
// tangential axis, u inner along the first).
__global__ void seg_beta3_kernel(DevView v) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.nseg) return;
    const Grid3& G = v.g3;
    const int d = v.seg_axis[t], line = v.seg_line[t];
    const int lo1 = v.seg_lo[t], len1 = v.seg_len[t], lo2 = v.seg_lo2[t], len2 = v.seg_len2[t];
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    double sum = 0.0;
    for (int w = lo2; w < lo2 + len2; ++w)
        for (int u = lo1; u < lo1 + len1; ++u) {
            int pos[3];
            pos[d] = line; pos[t1] = u; pos[t2] = w;
            const double kb = v.K[cell3(G, pos[0], pos[1], pos[2])];
            pos[d] = line - 1;
            const double ka = v.K[cell3(G, pos[0], pos[1], pos[2])];
            sum += 2.0 * ka * kb / (ka + kb);
        }
    const int nf = len1 * len2;
    const double keff = sum / nf;
    const double area = nf * area3(G, d);
    const double beta = v.alpha * sqrt(area) / keff;
    v.seg_beta[t] = beta;
    v.seg_D[t] = area / (2.0 * beta);
}

// Face coefficients seen from the lower (cL) and the upper (cU) cell:
// interior T = |e| / (r_a + r_b), skeleton rho = |e| / (r_c + beta_t),
// Dirichlet tau = 2 K_c |e| / h, Neumann 0 (r_c = h / (2 K_c)).
__global__ void face_coef3_kernel(DevView v) {
    const Grid3& G = v.g3;
    const long long total = v.nxface + v.nyface + v.nzface;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < total;
         f += (long long)gridDim.x * blockDim.x) {
        int d, i, j, k;
        long long fl;
        double *cL, *cU;
        const int* fseg;
        if (f < v.nxface) {
            d = 0; fl = f; cL = v.cxL; cU = v.cxU; fseg = v.xface_seg;
            i = (int)(fl % (G.nx + 1)); const long long r = fl / (G.nx + 1); j = (int)(r % G.ny); k = (int)(r / G.ny);
        } else if (f < v.nxface + v.nyface) {
            d = 1; fl = f - v.nxface; cL = v.cyL; cU = v.cyU; fseg = v.yface_seg;
            i = (int)(fl % G.nx); const long long r = fl / G.nx; j = (int)(r % (G.ny + 1)); k = (int)(r / (G.ny + 1));
        } else {
            d = 2; fl = f - v.nxface - v.nyface; cL = v.czL; cU = v.czU; fseg = v.zface_seg;
            i = (int)(fl % G.nx); const long long r = fl / G.nx; j = (int)(r % G.ny); k = (int)(r / G.ny);
        }
        const int n_d = d == 0 ? G.nx : (d == 1 ? G.ny : G.nz);
        const int pos = d == 0 ? i : (d == 1 ? j : k);
        const double area = area3(G, d), hn = hnorm3(G, d);
        const long long cu = pos < n_d ? cell3(G, i, j, k) : -1;
        const long long cl = pos > 0 ? cell3(G, i - (d == 0), j - (d == 1), k - (d == 2)) : -1;
        double vl = 0.0, vu = 0.0;
        if (cl < 0) {
            if (G.bc[2 * d]) vu = 2.0 * v.K[cu] * area / hn;
        } else if (cu < 0) {
            if (G.bc[2 * d + 1]) vl = 2.0 * v.K[cl] * area / hn;
        } else {
            // quotients as products with a reciprocal within an ulp (rcp_nr)
            const double ra = hn * rcp_nr(2.0 * v.K[cl]), rb = hn * rcp_nr(2.0 * v.K[cu]);
            const int t = fseg[fl];
            if (t >= 0) {
                const double beta = v.seg_beta[t];
                vl = area * rcp_nr(ra + beta);
                vu = area * rcp_nr(rb + beta);
            } else {
                vl = vu = area * rcp_nr(ra + rb);
            }
        }
        cL[fl] = vl;
        cU[fl] = vu;
    }
}

// The six faces of local cell (ii, jj, kk) of block B: the coefficient seen
// from the cell, whether the face couples to a cell of the block, and the
// local segment of a skeleton face (-1 otherwise).
struct Face3Info {
    double c;
    int nb;       // local neighbour cell, -1 when the face is not inside the block
    int seg;      // local segment, -1 when not a skeleton face
    int bside;    // domain boundary side (0..5), -1 otherwise
};

__device__ __forceinline__ Face3Info block_face(const DevView& v, const LeafDesc3& B, int ii, int jj, int kk,
                                                int side) {
    const Grid3& G = v.g3;
    const int d = side >> 1, up = side & 1;
    const int loc[3] = {ii, jj, kk};
    const int w0 = B.w[0], w1 = B.w[1];
    const int gi = B.i0 + ii, gj = B.j0 + jj, gk = B.k0 + kk;
    long long f;
    const double* cf;
    if (d == 0) {
        f = xface3(G, gi + up, gj, gk);
        cf = up ? v.cxL : v.cxU;
    } else if (d == 1) {
        f = yface3(G, gi, gj + up, gk);
        cf = up ? v.cyL : v.cyU;
    } else {
        f = zface3(G, gi, gj, gk + up);
        cf = up ? v.czL : v.czU;
    }
    Face3Info r;
    r.c = cf[f];
    r.nb = -1;
    r.seg = -1;
    r.bside = -1;
    const int p = loc[d] + (up ? 1 : -1);
    if (p >= 0 && p < B.w[d]) {
        int q[3] = {ii, jj, kk};
        q[d] = p;
        r.nb = (q[2] * w1 + q[1]) * w0 + q[0];
        return r;
    }
    if (B.side_off[side] < 0) {
        r.bside = side;
        return r;
    }
    // face index on the side: v outer along the second tangential axis
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    r.seg = B.side_off[side] + (B.side_fine[side] ? loc[t2] * B.w[t1] + loc[t1] : 0);
    return r;
}

struct Leaf3Smem {
    double A[kLeaf3Cells][kLeaf3Cells + 1];   // A, then its Cholesky factor (lower)
    double Z[kLeaf3Segs][kLeaf3Cells + 1];    // B, then Z = L^-1 B, columns ordered by first row
    double W[kLeaf3Segs];                     // sum of rho per ordered column
    int first[kLeaf3Segs];                    // first nonzero row of B per local segment
    int start[kLeaf3Segs];                    // ... per ordered column (ascending)
    int order[kLeaf3Segs];                    // ordered column -> local segment
    int rank[kLeaf3Segs];                     // local segment -> ordered column
    int act[kLeaf3Cells];                     // columns started at or above row k
    double rl[kLeaf3Cells];                   // 1 / L_kk, formed once per pivot
    int bad;                                  // a pivot that is not positive
};

// The factorisation of each block, one CTA per block.  Columns of Z are
// ordered by their first nonzero row, so the columns a step updates are a
// prefix, and every step's work (the band triangle of the Cholesky update,
// then one item per started column and band row) is spread evenly over the
// threads: an FP64 instruction costs a whole warp's issue whatever its mask,
// so the kernel avoids lanes that idle inside a busy warp.  R = Z^T Z - W
// gives each warp one ordered row r (its pairs run from the row's first
// nonzero, the later of the two), its lanes the columns q <= r.
__global__ void __launch_bounds__(kBuild3Threads) leaf3_build_kernel(DevView v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Leaf3Smem& S = *reinterpret_cast<Leaf3Smem*>(smem_raw);
    const int leaf = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const LeafDesc3 B = v.leaves3[leaf];
    const int n = B.w[0] * B.w[1] * B.w[2], m = B.m;
    for (int e = tid; e < kLeaf3Cells * (kLeaf3Cells + 1); e += kBuild3Threads) (&S.A[0][0])[e] = 0.0;
    for (int e = tid; e < kLeaf3Segs * (kLeaf3Cells + 1); e += kBuild3Threads) (&S.Z[0][0])[e] = 0.0;
    for (int q = tid; q < m; q += kBuild3Threads) S.first[q] = n;
    __syncthreads();
    // assembly of A (one cell per thread: diagonal in the order x-, x+, y-,
    // y+, z-, z+) and the first row of every column of B
    for (int c = tid; c < n; c += kBuild3Threads) {
        const int ii = c % B.w[0], jj = (c / B.w[0]) % B.w[1], kk = c / (B.w[0] * B.w[1]);
        double diag = 0.0;
        for (int side = 0; side < 6; ++side) {
            const Face3Info F = block_face(v, B, ii, jj, kk, side);
            diag += F.c;
            if (F.nb >= 0) S.A[c][F.nb] = -F.c;
            else if (F.seg >= 0) atomicMin(&S.first[F.seg], c);
        }
        S.A[c][c] = diag;
    }
    __syncthreads();
    for (int q = tid; q < m; q += kBuild3Threads) {
        int r = 0;
        for (int t = 0; t < m; ++t)
            r += S.first[t] < S.first[q] || (S.first[t] == S.first[q] && t < q);
        S.rank[q] = r;
        S.order[r] = q;
    }
    __syncthreads();
    for (int c = tid; c < n; c += kBuild3Threads) {
        const int ii = c % B.w[0], jj = (c / B.w[0]) % B.w[1], kk = c / (B.w[0] * B.w[1]);
        for (int side = 0; side < 6; ++side) {
            const Face3Info F = block_face(v, B, ii, jj, kk, side);
            if (F.nb < 0 && F.seg >= 0) S.Z[S.rank[F.seg]][c] = F.c;
        }
    }
    for (int q = tid; q < m; q += kBuild3Threads) S.start[q] = S.first[S.order[q]];
    __syncthreads();
    for (int q = tid; q < m; q += kBuild3Threads) {
        double w = 0.0;
        for (int c = S.start[q]; c < n; ++c) w += S.Z[q][c];
        S.W[q] = w;
    }
    for (int k = tid; k < n; k += kBuild3Threads) {
        int a = 0;
        while (a < m && S.start[a] <= k) ++a;
        S.act[k] = a;
    }
    // Cholesky A = L L^T, right-looking; cells are x fastest, so the factor
    // keeps A's half-bandwidth bw = w_x w_y.  Step k scales column k of L and
    // row k of the started columns of Z (both final then), then updates the
    // band triangle below it and rows k+1..k+bw of those columns.  1 / L_kk
    // is kept on the diagonal.
    // The reciprocal 1 / L_kk is formed once per pivot (an FP64 square root
    // and division cost about twenty FP64 instructions, per warp that runs
    // them): pivot k + 1 receives its last update at step k, as entry 0 of
    // that step's band triangle, and the thread that makes it forms the next
    // reciprocal there; the barrier that opens the next step publishes it.
    const int bw = B.w[0] * B.w[1];
    int lb = 0;
    while ((1 << lb) < bw) ++lb;                       // items per column: 2^lb >= bw band rows
    if (tid == 0) {
        const double a00 = S.A[0][0];
        S.bad = !(a00 > 0.0);
        S.rl[0] = 1.0 / sqrt(a00);
    }
    for (int k = 0; k < n; ++k) {
        __syncthreads();
        const double rl = S.rl[k];
        const int len = min(bw, n - 1 - k);
        const int a = S.act[k];
        for (int i = k + 1 + tid; i <= k + len; i += kBuild3Threads) S.A[i][k] *= rl;
        for (int q = tid; q < a; q += kBuild3Threads) S.Z[q][k] *= rl;
        __syncthreads();
        if (tid == 0) S.A[k][k] = rl;
        const int ntri = len * (len + 1) / 2;
        const int nitem = ntri + (a << lb);
        for (int e = tid; e < nitem; e += kBuild3Threads) {
            if (e < ntri) {
                int r = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                while ((r + 1) * (r + 2) / 2 <= e) ++r;
                while (r * (r + 1) / 2 > e) --r;
                const int i = k + 1 + r, j = k + 1 + (e - r * (r + 1) / 2);
                const double a = fma(-S.A[i][k], S.A[j][k], S.A[i][j]);
                S.A[i][j] = a;
                if (e == 0) {                      // pivot k + 1, final now
                    if (!(a > 0.0)) S.bad = 1;
                    S.rl[k + 1] = 1.0 / sqrt(a);
                }
            } else {
                const int e2 = e - ntri, q = e2 >> lb, r = (e2 & ((1 << lb) - 1)) + 1;
                if (r <= len) S.Z[q][k + r] = fma(-S.A[k + r][k], S.Z[q][k], S.Z[q][k + r]);
            }
        }
    }
    __syncthreads();
    if (S.bad && tid == 0) atomicOr(v.status, kStatusSingular);
    // R = Z^T Z - W (symmetric, both halves written, at the local segments)
    double* Rg = v.R + B.R_off;
    for (int r = warp; r < m; r += kBuild3Threads / 32) {
        const int k0 = S.start[r], sr = S.order[r];
        for (int qb = 0; qb <= r; qb += 32) {
            const int q = min(qb + lane, r);
            double acc = 0.0;
            for (int k = k0; k < n; ++k) acc = fma(S.Z[r][k], S.Z[q][k], acc);
            if (qb + lane <= r) {
                const int sq = S.order[q];
                if (q == r) acc -= S.W[r];
                Rg[(long long)sr * m + sq] = acc;
                Rg[(long long)sq * m + sr] = acc;
            }
        }
    }
    // the factor (column-major, 1 / L_kk on the diagonal) and Z for the solve
    double* Lg = v.leafL + B.L_off;
    for (int e = tid; e < n * n; e += kBuild3Threads) {
        const int k = e / n, i = e % n;      // column k, row i
        Lg[e] = (i > k && i <= k + bw) || i == k ? S.A[i][k] : 0.0;
    }
    double* Zg = v.leafZ + B.Z_off;
    for (int e = tid; e < m * n; e += kBuild3Threads) {
        const int q = e / n, k = e % n;
        Zg[(long long)S.order[q] * n + k] = S.Z[q][k];
    }
}

// Boundary value of the face of global cell (gi, gj, gk) on domain side s.
__device__ __forceinline__ double bc_value3(const Grid3& G, const double* bc_val, int s, int gi, int gj, int gk) {
    const long long sx = (long long)G.ny * G.nz, sy = (long long)G.nx * G.nz, sz = (long long)G.nx * G.ny;
    long long o;
    if (s < 2) o = (s ? sx : 0) + (long long)gk * G.ny + gj;
    else if (s < 4) o = 2 * sx + (s == 3 ? sy : 0) + (long long)gk * G.nx + gi;
    else o = 2 * sx + 2 * sy + (s == 5 ? sz : 0) + (long long)gj * G.nx + gi;
    return bc_val[o];
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Particular solve of each block: zbar = L^-1 bbar (bbar: the source and
// the external boundary data, Eqs. addu / addp) and rbar = Z^T zbar.
__global__ void __launch_bounds__(32 * kSolve3Warps)
leaf3_particular_kernel(DevView v, const double* __restrict__ q, const double* __restrict__ bc_val,
                        bool with_sadj) {
    __shared__ double ys[kSolve3Warps][kLeaf3Cells];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int leaf = blockIdx.x * kSolve3Warps + wi;
    if (leaf >= v.nleaf) return;            // uniform over the warp
    const LeafDesc3 B = v.leaves3[leaf];
    const Grid3& G = v.g3;
    const int n = B.w[0] * B.w[1] * B.w[2], m = B.m;
    const double* Lg = v.leafL + B.L_off;
    const double* Zg = v.leafZ + B.Z_off;
    const int bw = B.w[0] * B.w[1];
    double* y = ys[wi];
    for (int c = lane; c < n; c += 32) {
        const int ii = c % B.w[0], jj = (c / B.w[0]) % B.w[1], kk = c / (B.w[0] * B.w[1]);
        const int gi = B.i0 + ii, gj = B.j0 + jj, gk = B.k0 + kk;
        double b = q[cell3(G, gi, gj, gk)];
        for (int side = 0; side < 6 && bc_val; ++side) {
            const Face3Info F = block_face(v, B, ii, jj, kk, side);
            if (F.bside < 0) continue;
            const double g = bc_value3(G, bc_val, side, gi, gj, gk);
            if (G.bc[side]) b += F.c * g;
            else b -= area3(G, side >> 1) * g;
        }
        y[c] = b;
    }
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const double yk = y[k] * Lg[(long long)k * n + k];
        __syncwarp();
        if (lane == 0) y[k] = yk;
        const int iend = min(n - 1, k + bw);
        for (int i = k + 1 + lane; i <= iend; i += 32) y[i] = fma(-Lg[(long long)k * n + i], yk, y[i]);
        __syncwarp();
    }
    double* zb = v.leafzb + B.zb_off;
    for (int c = lane; c < n; c += 32) zb[c] = y[c];
    double* rb = v.rbar + B.r_off;
    for (int s = 0; s < m; ++s) {
        double acc = 0.0;
        for (int k = lane; k < n; k += 32) acc = fma(Zg[(long long)s * n + k], y[k], acc);
        acc = warp_sum(acc);
        // a right-hand side sigma of the segment's interface row (refinement)
        // acts as rbar - sigma
        if (lane == 0) rb[s] = with_sadj ? acc - v.sadj[B.r_off + s] : acc;
    }
}

// Final pressures of each block: p = L^-T (zbar + Z lambda), written into the
// cell state (p_hi, p_lo = 0).
__global__ void __launch_bounds__(32 * kSolve3Warps) leaf3_pressure_kernel(DevView v, bool accumulate) {
    __shared__ double ys[kSolve3Warps][kLeaf3Cells];
    __shared__ double ls[kSolve3Warps][kLeaf3Segs];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int leaf = blockIdx.x * kSolve3Warps + wi;
    if (leaf >= v.nleaf) return;
    const LeafDesc3 B = v.leaves3[leaf];
    const Grid3& G = v.g3;
    const int n = B.w[0] * B.w[1] * B.w[2], m = B.m;
    const double* Lg = v.leafL + B.L_off;
    const double* Zg = v.leafZ + B.Z_off;
    const double* zb = v.leafzb + B.zb_off;
    const int bw = B.w[0] * B.w[1];
    double* y = ys[wi];
    double* lam = ls[wi];
    for (int s = lane; s < m; s += 32) lam[s] = v.lam[B.r_off + s];
    __syncwarp();
    for (int c = lane; c < n; c += 32) {
        double acc = zb[c];
        for (int s = 0; s < m; ++s) acc = fma(Zg[(long long)s * n + c], lam[s], acc);
        y[c] = acc;
    }
    __syncwarp();
    // L^T p = y, left-looking from the last row: p_k = (y_k - sum_{i>k} L_ik p_i) / L_kk
    for (int k = n - 1; k >= 0; --k) {
        double part = 0.0;
        const int iend = min(n - 1, k + bw);
        for (int i = k + 1 + lane; i <= iend; i += 32) part = fma(Lg[(long long)k * n + i], y[i], part);
        part = warp_sum(part);
        const double pk = (y[k] - part) * Lg[(long long)k * n + k];
        __syncwarp();
        if (lane == 0) y[k] = pk;
        __syncwarp();
    }
    for (int c = lane; c < n; c += 32) {
        const int ii = c % B.w[0], jj = (c / B.w[0]) % B.w[1], kk = c / (B.w[0] * B.w[1]);
        const long long gc = cell3(G, B.i0 + ii, B.j0 + jj, B.k0 + kk);
        if (accumulate) {
            const DD x = dd_add(DD{v.p_hi[gc], v.p_lo[gc]}, DD{y[c], 0.0});
            v.p_hi[gc] = x.h;
            v.p_lo[gc] = x.l;
        } else {
            v.p_hi[gc] = y[c];
            v.p_lo[gc] = 0.0;
        }
    }
}

__device__ __forceinline__ void block_max3(unsigned long long* slot, double x) {
    __shared__ double wmax[32];
    double a = fabs(x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        double b = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        // non-negative doubles order like their bit patterns
        if (threadIdx.x == 0 && b > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(b));
    }
}

// Refinement residuals in FP64 of the discrete equations (Eqs. 11.2-14.2
// with lumped RT0) at the current state (p_hi + p_lo, the segments' Robin
// data lambda^a = P - beta U, lambda^b = P + beta U): cell balances
// E_c = sum of outward fluxes - q_c, rcell = -E_c.
__global__ void __launch_bounds__(256) residual3_cells_kernel(DevView v, const double* __restrict__ q,
                                                              const double* __restrict__ bc_val, int step) {
    const Grid3& G = v.g3;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (c < v.ncell) {
        const int i = (int)(c % G.nx);
        const long long r = c / G.nx;
        const int j = (int)(r % G.ny), k = (int)(r / G.ny);
        const double pc = v.p_hi[c] + v.p_lo[c];
        double E = -q[c];
        for (int side = 0; side < 6; ++side) {
            const int d = side >> 1, up = side & 1;
            const int pos = d == 0 ? i : (d == 1 ? j : k);
            const int nd = d == 0 ? G.nx : (d == 1 ? G.ny : G.nz);
            long long f;
            const double* cf;
            const int* fs;
            if (d == 0) { f = xface3(G, i + up, j, k); cf = up ? v.cxL : v.cxU; fs = v.xface_seg; }
            else if (d == 1) { f = yface3(G, i, j + up, k); cf = up ? v.cyL : v.cyU; fs = v.yface_seg; }
            else { f = zface3(G, i, j, k + up); cf = up ? v.czL : v.czU; fs = v.zface_seg; }
            const double coef = cf[f];
            if (up ? pos == nd - 1 : pos == 0) {
                const double g = bc_value3(G, bc_val, side, i, j, k);
                E += G.bc[side] ? coef * (pc - g) : area3(G, d) * g;
                continue;
            }
            const int t = fs[f];
            if (t >= 0) {
                const double2 l = v.seg_lam_dd[2 * t + (up ? 0 : 1)];
                E += coef * (pc - (l.x + l.y));
            } else {
                const long long nb = c + (up ? 1 : -1) * (d == 0 ? 1LL : (d == 1 ? (long long)G.nx : (long long)G.nx * G.ny));
                E += coef * (pc - (v.p_hi[nb] + v.p_lo[nb]));
            }
        }
        e = E;
        v.rcell[c] = -E;
    }
    block_max3(v.res_max + step, e);
}

// Segment residuals: E13 = F^a + F^b (Eq. 13.2), E14 = F^a - F^b - 2 |t| U
// (Eq. 14.2, divided by beta), outward integrated fluxes of the two sides;
// they enter the correction solve as right-hand sides of the two interface
// rows of the segment.
__global__ void __launch_bounds__(128) residual3_segments_kernel(DevView v, int step) {
    const Grid3& G = v.g3;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double E13 = 0.0, E14 = 0.0;
    if (t < v.nseg) {
        const int d = v.seg_axis[t], line = v.seg_line[t];
        const int lo1 = v.seg_lo[t], len1 = v.seg_len[t], lo2 = v.seg_lo2[t], len2 = v.seg_len2[t];
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        const double2 l2a = v.seg_lam_dd[2 * t], l2b = v.seg_lam_dd[2 * t + 1];
        const double la = l2a.x + l2a.y, lb = l2b.x + l2b.y;
        const double* cL = d == 0 ? v.cxL : (d == 1 ? v.cyL : v.czL);
        const double* cU = d == 0 ? v.cxU : (d == 1 ? v.cyU : v.czU);
        double Fa = 0.0, Fb = 0.0;
        for (int w = lo2; w < lo2 + len2; ++w)
            for (int u = lo1; u < lo1 + len1; ++u) {
                int pos[3];
                pos[d] = line; pos[t1] = u; pos[t2] = w;
                const long long cb = cell3(G, pos[0], pos[1], pos[2]);
                const long long f = d == 0 ? xface3(G, pos[0], pos[1], pos[2])
                                           : (d == 1 ? yface3(G, pos[0], pos[1], pos[2]) : zface3(G, pos[0], pos[1], pos[2]));
                pos[d] = line - 1;
                const long long ca = cell3(G, pos[0], pos[1], pos[2]);
                Fa += cL[f] * ((v.p_hi[ca] + v.p_lo[ca]) - la);
                Fb += cU[f] * ((v.p_hi[cb] + v.p_lo[cb]) - lb);
            }
        const double area = len1 * len2 * area3(G, d);
        const double two_u = 2.0 * area * (v.segU[t] + v.segU_lo[t]);
        E13 = Fa + Fb;
        E14 = (Fa - Fb) - two_u;
        v.sadj[v.seg_lam_a[t]] = -0.5 * (E13 + E14);
        v.sadj[v.seg_lam_b[t]] = -0.5 * (E13 - E14);
    }
    block_max3(v.res_max + step, fmax(fabs(E13), fabs(E14)));
}

// Cell pressures and face fluxes (+axis sign) from the state (p_hi + p_lo,
// the segments' Robin data of the interface unknowns); on the skeleton the
// mean of the two one-sided values rho (p_c - lambda) of the blocks on either
// side.  iface (optional): the one-sided values [Fa_x, Fb_x, Fa_y, Fb_y,
// Fa_z, Fb_z], side a the lower block, both equal to F off the skeleton.
__global__ void face_flux3_kernel(DevView v, const double* __restrict__ bc_val, double* __restrict__ p,
                                  double* __restrict__ Fx, double* __restrict__ Fy, double* __restrict__ Fz,
                                  double* __restrict__ iface) {
    const Grid3& G = v.g3;
    const long long nf = v.nxface + v.nyface + v.nzface;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf + v.ncell;
         f += (long long)gridDim.x * blockDim.x) {
        if (f >= nf) {
            const long long c = f - nf;
            p[c] = v.p_hi[c] + v.p_lo[c];
            continue;
        }
        int d, i, j, k;
        long long fl;
        const double *cL, *cU;
        const int* fseg;
        double* out;
        if (f < v.nxface) {
            d = 0; fl = f; cL = v.cxL; cU = v.cxU; fseg = v.xface_seg; out = Fx;
            i = (int)(fl % (G.nx + 1)); const long long r = fl / (G.nx + 1); j = (int)(r % G.ny); k = (int)(r / G.ny);
        } else if (f < v.nxface + v.nyface) {
            d = 1; fl = f - v.nxface; cL = v.cyL; cU = v.cyU; fseg = v.yface_seg; out = Fy;
            i = (int)(fl % G.nx); const long long r = fl / G.nx; j = (int)(r % (G.ny + 1)); k = (int)(r / (G.ny + 1));
        } else {
            d = 2; fl = f - v.nxface - v.nyface; cL = v.czL; cU = v.czU; fseg = v.zface_seg; out = Fz;
            i = (int)(fl % G.nx); const long long r = fl / G.nx; j = (int)(r % G.ny); k = (int)(r / G.ny);
        }
        const int n_d = d == 0 ? G.nx : (d == 1 ? G.ny : G.nz);
        const int pos = d == 0 ? i : (d == 1 ? j : k);
        const double area = area3(G, d);
        double F, fa1 = 0.0, fb1 = 0.0;
        bool skel = false;
        if (pos == 0) {
            const double pb = v.p_hi[cell3(G, i, j, k)] + v.p_lo[cell3(G, i, j, k)];
            const double g = bc_value3(G, bc_val, 2 * d, i, j, k);
            F = G.bc[2 * d] ? -(cU[fl] * (pb - g)) : -(area * g);
        } else {
            const int ai = i - (d == 0), aj = j - (d == 1), ak = k - (d == 2);
            const long long ca = cell3(G, ai, aj, ak);
            const double pa = v.p_hi[ca] + v.p_lo[ca];
            if (pos == n_d) {
                const double g = bc_value3(G, bc_val, 2 * d + 1, ai, aj, ak);
                F = G.bc[2 * d + 1] ? cL[fl] * (pa - g) : area * g;
            } else {
                const long long cb = cell3(G, i, j, k);
                const double pb = v.p_hi[cb] + v.p_lo[cb];
                const int t = fseg[fl];
                if (t >= 0) {
                    const double2 la = v.seg_lam_dd[2 * t], lb = v.seg_lam_dd[2 * t + 1];
                    const double fa = cL[fl] * (pa - (la.x + la.y));
                    const double fb = -(cU[fl] * (pb - (lb.x + lb.y)));
                    F = 0.5 * (fa + fb);
                    fa1 = fa;
                    fb1 = fb;
                    skel = true;
                } else {
                    F = cL[fl] * (pa - pb);
                }
            }
        }
        out[fl] = F;
        if (iface) {
            // block of this axis: Fa at 2 (faces of the earlier axes), Fb after it
            const long long nd = d == 0 ? v.nxface : (d == 1 ? v.nyface : v.nzface);
            const long long base = 2 * (d == 0 ? 0 : (d == 1 ? v.nxface : v.nxface + v.nyface));
            iface[base + fl] = skel ? fa1 : F;
            iface[base + nd + fl] = skel ? fb1 : F;
        }
    }
}

inline unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 16) b = 152LL * 16;
    return (unsigned)std::max(b, 1LL);
}

}  // namespace

cudaError_t launch_coef3(const DevView& v, cudaStream_t s) {
    if (v.nseg > 0) seg_beta3_kernel<<<(v.nseg + 127) / 128, 128, 0, s>>>(v);
    face_coef3_kernel<<<grid_for(v.nxface + v.nyface + v.nzface, 256), 256, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_leaf3_build(const DevView& v, cudaStream_t s) {
    // set on every launch (a host call; the attribute belongs to the current device)
    const int bytes = (int)sizeof(Leaf3Smem);
    cudaError_t e = cudaFuncSetAttribute(leaf3_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    leaf3_build_kernel<<<v.nleaf, kBuild3Threads, bytes, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_leaf3_particular(const DevView& v, const double* q, const double* bc_val, bool with_sadj,
                                    cudaStream_t s) {
    leaf3_particular_kernel<<<(v.nleaf + kSolve3Warps - 1) / kSolve3Warps, 32 * kSolve3Warps, 0, s>>>(
        v, q, bc_val, with_sadj);
    return cudaGetLastError();
}

cudaError_t launch_leaf3_pressure(const DevView& v, bool accumulate, cudaStream_t s) {
    leaf3_pressure_kernel<<<(v.nleaf + kSolve3Warps - 1) / kSolve3Warps, 32 * kSolve3Warps, 0, s>>>(v, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_residual3(const DevView& v, const double* q, const double* bc_val, int step, cudaStream_t s) {
    residual3_cells_kernel<<<(unsigned)((v.ncell + 255) / 256), 256, 0, s>>>(v, q, bc_val, step);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || v.nseg == 0) return e;
    residual3_segments_kernel<<<(v.nseg + 127) / 128, 128, 0, s>>>(v, step);
    return cudaGetLastError();
}

cudaError_t launch_face_fluxes3(const DevView& v, const double* bc_val, double* p, double* Fx, double* Fy,
                                double* Fz, double* iface, cudaStream_t s) {
    const long long n = v.nxface + v.nyface + v.nzface + v.ncell;
    face_flux3_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, bc_val, p, Fx, Fy, Fz, iface);
    return cudaGetLastError();
}

}  // namespace mrcm
