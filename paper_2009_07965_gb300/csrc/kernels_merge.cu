// Merge kernels: the recursive interface systems of Algorithm 1.
//
// arXiv 2009.07965, Section 3: a node Omega^{i,l} is the union of two
// children, gamma^{i,l} their common interface.  Each child c is known by
// its Robin-to-flux map on its outer segments, F^c = R^c lambda^c + rbar^c
// (outward segment fluxes, lambda^c the Robin datum P - beta U (n.n^c) of
// Eq. 11.2).  On a gamma segment t, with c1 on side a (lower coordinate) and
// c2 on side b, Eqs. (13.2) and (14.2) read
//     F^a_t + F^b_t = 0,   F^a_t - F^b_t = 2 U_t |t|,
// and with lambda^a = P - beta U, lambda^b = P + beta U they become
//     F^a_t = D_t (lambda^b_t - lambda^a_t),  F^b_t = D_t (lambda^a_t - lambda^b_t),
// D_t = |t| / (2 beta_t).  Unknowns on gamma: y = [lambda^a_gamma; lambda^b_gamma]
// (2g values; the paper's (U, P) pair, Eq. linsys restricted to gamma):
//     M y = -C lambda_o - [rbar^a_gamma; rbar^b_gamma],
//     M = [[R^a_gg + D, -D], [-D, R^b_gg + D]],  C = blockdiag(R^a_go, R^b_go).
// The coefficients X = -M^-1 C and xbar = -M^-1 rbar_gamma are the X^{i,l},
// Xbar^{i,l} of Algorithm 1; substituting them into the children's outer
// fluxes gives the node's own map (Eqs. new_bfs.1-2 / particular.1-2):
//     R = blockdiag(R^a_oo, R^b_oo) + blockdiag(R^a_og, R^b_og) X,
//     rbar = rbar_o + blockdiag(R^a_og, R^b_og) xbar.
// The root has no outer segments; for an all-Neumann problem its system has
// the constant null vector and the continuity row of gamma[0] is replaced by
// P_{gamma[0]} = 0 (lambda^a + lambda^b = 0), keeping the difference row.
//
// Storage: M is factored in place, column-major (entry (r, c) at c*2g + r),
// with partial pivoting organised in panels of kNB columns: at step k rows k
// and piv[k] are exchanged in the columns of k's panel and to its right, so
// the multipliers of earlier panels stay where they were computed.  A forward
// solve therefore takes the panels in order: apply the panel's exchanges,
// then eliminate its columns.  X is column-major too (2g x m).
//
// Two launch shapes.  Levels with many nodes: one CTA per node, M in shared
// memory (merge_small_kernel).  Levels with few, large nodes: a blocked
// right-looking LU across many CTAs -- a panel kernel (NB columns, one CTA
// per node), a TRSM kernel for the block row of U and a tiled FP64 GEMM for
// the trailing update -- then X by column blocks and R by output tiles.
#include "mrcm_internal.h"

namespace mrcm {
namespace {

constexpr int kNB = 32;         // panel width of the blocked LU
constexpr int kGemmTile = 64;   // trailing-update tile (kGemmTile^2 outputs per CTA)
constexpr int kXCols = 8;       // X columns per CTA in the blocked X solve
constexpr int kRTile = 32;      // R update tile

struct NodeRefs {
    int g, g2, m, o1, m1, m2;
    const int *gpos1, *gpos2, *opos1, *opos2;
    const double *R1, *R2;
};

__device__ __forceinline__ NodeRefs node_refs(const DevView& v, const MergeDesc& D) {
    NodeRefs r;
    r.g = D.g; r.g2 = 2 * D.g; r.m = D.m; r.o1 = D.o1; r.m1 = D.m1; r.m2 = D.m2;
    r.gpos1 = v.node_map + D.map_off;
    r.gpos2 = r.gpos1 + D.g;
    r.opos1 = r.gpos2 + D.g;
    r.opos2 = r.opos1 + D.o1;
    r.R1 = v.R + D.R1_off;
    r.R2 = v.R + D.R2_off;
    return r;
}

// Entry (r, c) of the interface matrix M (before the pinning rows).
__device__ __forceinline__ double m_entry(const DevView& v, const MergeDesc& D, const NodeRefs& N, int r, int c) {
    const int g = N.g;
    if (r < g && c < g) {
        double val = N.R1[N.gpos1[r] * N.m1 + N.gpos1[c]];
        if (r == c) val += v.seg_D[v.gamma_segs[D.gamma_off + r]];
        return val;
    }
    if (r >= g && c >= g) {
        double val = N.R2[N.gpos2[r - g] * N.m2 + N.gpos2[c - g]];
        if (r == c) val += v.seg_D[v.gamma_segs[D.gamma_off + r - g]];
        return val;
    }
    if (r < g && c - g == r) return -v.seg_D[v.gamma_segs[D.gamma_off + r]];
    if (r >= g && r - g == c) return -v.seg_D[v.gamma_segs[D.gamma_off + c]];
    return 0.0;
}

// Entry (r, c) of M with the all-Neumann pinning of the root applied:
// row 0 <- (lambda^a + lambda^b of gamma[0]), row g <- row 0 - row g.
__device__ __forceinline__ double m_entry_pinned(const DevView& v, const MergeDesc& D, const NodeRefs& N, int r,
                                                 int c) {
    if (D.pinned) {
        if (r == 0) return (c == 0 || c == N.g) ? 1.0 : 0.0;
        if (r == N.g) return m_entry(v, D, N, 0, c) - m_entry(v, D, N, N.g, c);
    }
    return m_entry(v, D, N, r, c);
}

// Entry (r, j) of C = blockdiag(R^a_go, R^b_go).
__device__ __forceinline__ double c_entry(const NodeRefs& N, int r, int j) {
    if (r < N.g && j < N.o1) return N.R1[N.gpos1[r] * N.m1 + N.opos1[j]];
    if (r >= N.g && j >= N.o1) return N.R2[N.gpos2[r - N.g] * N.m2 + N.opos2[j - N.o1]];
    return 0.0;
}

// R(i, j) = blockdiag(R_oo) + blockdiag(R_og) X, X column-major (2g x m).
__device__ __forceinline__ double r_entry(const NodeRefs& N, const double* X, int i, int j) {
    double acc = 0.0;
    const double* xc = X + (long long)j * N.g2;
    if (i < N.o1) {
        const double* row = N.R1 + N.opos1[i] * N.m1;
        if (j < N.o1) acc = row[N.opos1[j]];
        for (int k = 0; k < N.g; ++k) acc += row[N.gpos1[k]] * xc[k];
    } else {
        const double* row = N.R2 + N.opos2[i - N.o1] * N.m2;
        if (j >= N.o1) acc = row[N.opos2[j - N.o1]];
        for (int k = 0; k < N.g; ++k) acc += row[N.gpos2[k]] * xc[N.g + k];
    }
    return acc;
}

template <int NT>
__device__ __forceinline__ double block_max(double val, double* sv) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val = fmax(val, __shfl_xor_sync(0xffffffffu, val, o));
    if ((threadIdx.x & 31) == 0) sv[threadIdx.x >> 5] = val;
    __syncthreads();
    double mx = 0.0;
    for (int w = 0; w < NT / 32; ++w) mx = fmax(mx, sv[w]);
    __syncthreads();
    return mx;
}

// One elimination step k on a column-major matrix M (ld = n): pivot search
// in column k, exchange of rows k and p in columns [cstart, cend) (cstart =
// first column of k's panel), scaling of the multipliers, rank-1 update of
// columns (k, cend).  The pivot's reciprocal is formed once (thread 0) and
// shared through *s_rcp.
template <int NT>
__device__ __forceinline__ void lu_step(double* M, int n, int k, int cstart, int cend, double thresh, int* piv,
                                        double* sv, int* si, double* s_rcp, bool& singular) {
    const int tid = threadIdx.x;
    double best = -1.0;
    int bi = k;
    const double* col = M + (long long)k * n;
    for (int i = k + tid; i < n; i += NT) {
        const double a = fabs(col[i]);
        if (a > best) { best = a; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { sv[tid >> 5] = best; si[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
        double bv = sv[0];
        int b = si[0];
        for (int w = 1; w < NT / 32; ++w)
            if (sv[w] > bv || (sv[w] == bv && si[w] < b)) { bv = sv[w]; b = si[w]; }
        piv[k] = b;
        si[0] = b;
        const double pivot = col[b];
        if (!(fabs(pivot) > thresh)) singular = true;
        *s_rcp = 1.0 / pivot;
    }
    __syncthreads();
    const int p = si[0];
    if (p != k) {
        for (int c = cstart + tid; c < cend; c += NT) {
            double* cc = M + (long long)c * n;
            const double a = cc[k];
            cc[k] = cc[p];
            cc[p] = a;
        }
        __syncthreads();
    }
    const double rcp = *s_rcp;
    double* ck = M + (long long)k * n;
    for (int i = k + 1 + tid; i < n; i += NT) ck[i] *= rcp;
    __syncthreads();
    const int rows = n - k - 1, cols = cend - k - 1;
    for (int idx = tid; idx < rows * cols; idx += NT) {
        const int i = k + 1 + idx % rows, c = k + 1 + idx / rows;
        double* cc = M + (long long)c * n;
        cc[i] -= ck[i] * cc[k];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Fused path: one CTA per node, M in shared memory.
template <int NT>
__global__ void __launch_bounds__(NT) merge_small_kernel(DevView v, int first) {
    extern __shared__ __align__(16) double M[];
    __shared__ double sv[NT / 32];
    __shared__ int si[NT / 32];
    __shared__ double s_rcp;
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int g2 = N.g2, m = N.m;
    const int tid = threadIdx.x;
    int* piv = v.piv + D.piv_off;
    double* X = v.X + D.X_off;
    double amax = 0.0;
    for (int idx = tid; idx < g2 * g2; idx += NT) {
        const int r = idx % g2, c = idx / g2;
        const double val = m_entry_pinned(v, D, N, r, c);
        M[idx] = val;
        amax = fmax(amax, fabs(val));
    }
    for (int idx = tid; idx < g2 * m; idx += NT) X[idx] = -c_entry(N, idx % g2, idx / g2);
    const double thresh = 1e-14 * block_max<NT>(amax, sv);
    bool singular = false;
    for (int k = 0; k < g2; ++k)
        lu_step<NT>(M, g2, k, (k / kNB) * kNB, g2, thresh, piv, sv, si, &s_rcp, singular);
    if (singular && tid == 0) atomicOr(v.status, kStatusSingular);
    // X = -M^-1 C, one column per thread (forward with the exchanges, backward)
    for (int j = tid; j < m; j += NT) {
        double* x = X + (long long)j * g2;
        for (int k0 = 0; k0 < g2; k0 += kNB) {
            const int kend = min(k0 + kNB, g2);
            for (int k = k0; k < kend; ++k) {
                const int p = piv[k];
                if (p != k) { const double a = x[p]; x[p] = x[k]; x[k] = a; }
            }
            for (int k = k0; k < kend; ++k) {
                const double xk = x[k];
                const double* ck = M + k * g2;
                for (int i = k + 1; i < g2; ++i) x[i] -= ck[i] * xk;
            }
        }
        for (int k = g2 - 1; k >= 0; --k) {
            const double* ck = M + k * g2;
            const double xk = x[k] / ck[k];
            x[k] = xk;
            for (int i = 0; i < k; ++i) x[i] -= ck[i] * xk;
        }
    }
    __syncthreads();
    double* Rp = v.R + D.R_off;
    for (int idx = tid; idx < m * m; idx += NT) Rp[idx] = r_entry(N, X, idx / m, idx % m);
    double* Mg = v.LU + D.LU_off;
    for (int idx = tid; idx < g2 * g2; idx += NT) Mg[idx] = M[idx];
}

// ---------------------------------------------------------------------------
// Blocked path.
// Assembly of M (column-major, pinned rows applied) and of -C into X.
__global__ void __launch_bounds__(256) merge_assemble_kernel(DevView v, int first, unsigned long long* amax_bits) {
    const int node = first + blockIdx.x;
    const MergeDesc D = v.merges[node];
    const NodeRefs N = node_refs(v, D);
    const int g2 = N.g2, m = N.m;
    double* M = v.LU + D.LU_off;
    double* X = v.X + D.X_off;
    const long long nM = (long long)g2 * g2, nX = (long long)g2 * m;
    double amax = 0.0;
    for (long long idx = blockIdx.y * 256LL + threadIdx.x; idx < nM + nX; idx += (long long)gridDim.y * 256) {
        if (idx < nM) {
            const int r = (int)(idx % g2), c = (int)(idx / g2);
            const double val = m_entry_pinned(v, D, N, r, c);
            M[idx] = val;
            amax = fmax(amax, fabs(val));
        } else {
            const long long x = idx - nM;
            X[x] = -c_entry(N, (int)(x % g2), (int)(x / g2));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.0)
        atomicMax(amax_bits + (node - first), (unsigned long long)__double_as_longlong(amax));
}

// Panel factorisation of columns [k0, k0+NB) (rows k0..2g-1), one CTA per node.
template <int NT>
__global__ void __launch_bounds__(NT) lu_panel_kernel(DevView v, int first, int k0,
                                                      const unsigned long long* amax_bits) {
    __shared__ double sv[NT / 32];
    __shared__ int si[NT / 32];
    __shared__ double s_rcp;
    const MergeDesc D = v.merges[first + blockIdx.x];
    const int g2 = 2 * D.g;
    if (k0 >= g2) return;
    const int kend = min(k0 + kNB, g2);
    double* M = v.LU + D.LU_off;
    int* piv = v.piv + D.piv_off;
    const double thresh = 1e-14 * __longlong_as_double((long long)amax_bits[blockIdx.x]);
    bool singular = false;
    for (int k = k0; k < kend; ++k) lu_step<NT>(M, g2, k, k0, kend, thresh, piv, sv, si, &s_rcp, singular);
    if (singular && threadIdx.x == 0) atomicOr(v.status, kStatusSingular);
}

// Block row of U: apply the panel's exchanges to columns [kend, 2g) and
// solve U12 = L11^-1 A12; one thread per column.
__global__ void __launch_bounds__(64) lu_trsm_kernel(DevView v, int first, int k0) {
    __shared__ double L11[kNB][kNB + 1];
    __shared__ int pv[kNB];
    const MergeDesc D = v.merges[first + blockIdx.x];
    const int g2 = 2 * D.g;
    const int kend = min(k0 + kNB, g2);
    const int j = kend + blockIdx.y * 64 + threadIdx.x;
    if (kend >= g2 || kend + blockIdx.y * 64 >= g2) return;   // uniform per CTA
    double* M = v.LU + D.LU_off;
    const int nb = kend - k0;
    for (int idx = threadIdx.x; idx < kNB * kNB; idx += 64) {
        const int r = idx % kNB, c = idx / kNB;
        L11[r][c] = (r < nb && c < nb) ? M[(long long)(k0 + c) * g2 + k0 + r] : 0.0;
    }
    for (int idx = threadIdx.x; idx < nb; idx += 64) pv[idx] = v.piv[D.piv_off + k0 + idx];
    __syncthreads();
    if (j >= g2) return;
    double* col = M + (long long)j * g2;
    for (int c = 0; c < nb; ++c) {
        const int p = pv[c];
        if (p != k0 + c) {
            const double a = col[k0 + c];
            col[k0 + c] = col[p];
            col[p] = a;
        }
    }
    double u[kNB];
#pragma unroll
    for (int r = 0; r < kNB; ++r) u[r] = r < nb ? col[k0 + r] : 0.0;
#pragma unroll
    for (int c = 0; c < kNB; ++c)
#pragma unroll
        for (int r = c + 1; r < kNB; ++r) u[r] -= L11[r][c] * u[c];
#pragma unroll
    for (int r = 0; r < kNB; ++r)
        if (r < nb) col[k0 + r] = u[r];
}

// Trailing update A22 -= L21 U12 on kGemmTile^2 tiles; 256 threads, 4x4 each.
__global__ void __launch_bounds__(256) lu_gemm_kernel(DevView v, int first, int k0) {
    __shared__ double Ls[kNB][kGemmTile + 1];   // Ls[c][r]
    __shared__ double Us[kNB][kGemmTile + 1];   // Us[c][j]
    const MergeDesc D = v.merges[first + blockIdx.x];
    const int g2 = 2 * D.g;
    const int kend = min(k0 + kNB, g2);
    const int nb = kend - k0;
    const int rest = g2 - kend;
    const int tiles = (rest + kGemmTile - 1) / kGemmTile;
    if (rest <= 0 || (int)blockIdx.y >= tiles * tiles) return;   // uniform per CTA
    const int r0 = kend + (blockIdx.y % tiles) * kGemmTile;
    const int j0 = kend + (blockIdx.y / tiles) * kGemmTile;
    double* M = v.LU + D.LU_off;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kNB * kGemmTile; idx += 256) {
        const int r = idx % kGemmTile, c = idx / kGemmTile;
        Ls[c][r] = (c < nb && r0 + r < g2) ? M[(long long)(k0 + c) * g2 + r0 + r] : 0.0;
    }
    for (int idx = tid; idx < kNB * kGemmTile; idx += 256) {
        const int c = idx % kNB, jj = idx / kNB;
        Us[c][jj] = (c < nb && j0 + jj < g2) ? M[(long long)(j0 + jj) * g2 + k0 + c] : 0.0;
    }
    __syncthreads();
    const int tr = (tid % 16) * 4, tc = (tid / 16) * 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll 4
    for (int c = 0; c < kNB; ++c) {
        double lv[4], uv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) { lv[a] = Ls[c][tr + a]; uv[a] = Us[c][tc + a]; }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += lv[a] * uv[b];
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = j0 + tc + b;
        if (j >= g2) continue;
        double* col = M + (long long)j * g2;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int r = r0 + tr + a;
            if (r < g2) col[r] -= acc[a][b];
        }
    }
}

// X = -M^-1 C for kXCols columns per CTA, columns staged in shared memory.
__global__ void __launch_bounds__(256) merge_xsolve_kernel(DevView v, int first) {
    extern __shared__ __align__(16) double xs[];   // kXCols x 2g
    const MergeDesc D = v.merges[first + blockIdx.x];
    const int g2 = 2 * D.g, m = D.m;
    const int j0 = blockIdx.y * kXCols;
    if (j0 >= m) return;                              // uniform per CTA
    const int nc = min(kXCols, m - j0);
    const double* M = v.LU + D.LU_off;
    const int* piv = v.piv + D.piv_off;
    double* X = v.X + D.X_off;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < nc * g2; idx += 256) xs[idx] = X[(long long)j0 * g2 + idx];
    __syncthreads();
    // forward: per panel, its exchanges, then its columns of the unit lower L
    for (int k0 = 0; k0 < g2; k0 += kNB) {
        const int kend = min(k0 + kNB, g2);
        if (tid < nc) {
            for (int k = k0; k < kend; ++k) {
                const int p = piv[k];
                if (p != k) {
                    const double a = xs[tid * g2 + k];
                    xs[tid * g2 + k] = xs[tid * g2 + p];
                    xs[tid * g2 + p] = a;
                }
            }
        }
        __syncthreads();
        for (int k = k0; k < kend; ++k) {
            const double* ck = M + (long long)k * g2;
            const int rows = g2 - k - 1;
            for (int idx = tid; idx < rows * nc; idx += 256) {
                const int i = k + 1 + idx % rows, c = idx / rows;
                xs[c * g2 + i] -= ck[i] * xs[c * g2 + k];
            }
            __syncthreads();
        }
    }
    // backward: U
    for (int k = g2 - 1; k >= 0; --k) {
        const double* ck = M + (long long)k * g2;
        if (tid < nc) xs[tid * g2 + k] /= ck[k];
        __syncthreads();
        for (int idx = tid; idx < k * nc; idx += 256) {
            const int i = idx % k, c = idx / k;
            xs[c * g2 + i] -= ck[i] * xs[c * g2 + k];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < nc * g2; idx += 256) X[(long long)j0 * g2 + idx] = xs[idx];
}

// R = blockdiag(R_oo) + blockdiag(R_og) X on kRTile^2 output tiles.
__global__ void __launch_bounds__(256) merge_rupdate_kernel(DevView v, int first) {
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int m = N.m;
    const int tiles = (m + kRTile - 1) / kRTile;
    if ((int)blockIdx.y >= tiles * tiles) return;
    const int i0 = (blockIdx.y % tiles) * kRTile, jt = (blockIdx.y / tiles) * kRTile;
    const double* X = v.X + D.X_off;
    double* Rp = v.R + D.R_off;
    for (int idx = threadIdx.x; idx < kRTile * kRTile; idx += 256) {
        const int i = i0 + idx / kRTile, j = jt + idx % kRTile;
        if (i < m && j < m) Rp[(long long)i * m + j] = r_entry(N, X, i, j);
    }
}

// ---------------------------------------------------------------------------
// Solve phase, bottom-up: xbar = -M^-1 [rbar^a_gamma; rbar^b_gamma] and the
// node's particular fluxes (Eqs. particular.1-2).
template <int NT>
__global__ void __launch_bounds__(NT) merge_up_kernel(DevView v, int first) {
    extern __shared__ __align__(16) double rhs[];
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int g = N.g, g2 = N.g2, m = N.m, o1 = N.o1;
    const int tid = threadIdx.x;
    const double* M = v.LU + D.LU_off;
    const int* piv = v.piv + D.piv_off;
    const double* rb1 = v.rbar + D.r1_off;
    const double* rb2 = v.rbar + D.r2_off;
    for (int r = tid; r < g2; r += NT) rhs[r] = -(r < g ? rb1[N.gpos1[r]] : rb2[N.gpos2[r - g]]);
    __syncthreads();
    if (D.pinned && tid == 0) {
        const double a = rhs[0], b = rhs[g];
        rhs[g] = a - b;
        rhs[0] = 0.0;
    }
    __syncthreads();
    for (int k0 = 0; k0 < g2; k0 += kNB) {
        const int kend = min(k0 + kNB, g2);
        if (tid == 0) {
            for (int k = k0; k < kend; ++k) {
                const int p = piv[k];
                if (p != k) { const double a = rhs[p]; rhs[p] = rhs[k]; rhs[k] = a; }
            }
        }
        __syncthreads();
        for (int k = k0; k < kend; ++k) {
            const double xk = rhs[k];
            const double* ck = M + (long long)k * g2;
            for (int i = k + 1 + tid; i < g2; i += NT) rhs[i] -= ck[i] * xk;
            __syncthreads();
        }
    }
    for (int k = g2 - 1; k >= 0; --k) {
        const double* ck = M + (long long)k * g2;
        if (tid == 0) rhs[k] /= ck[k];
        __syncthreads();
        const double xk = rhs[k];
        for (int i = tid; i < k; i += NT) rhs[i] -= ck[i] * xk;
        __syncthreads();
    }
    double* xb = v.xbar + D.xb_off;
    for (int r = tid; r < g2; r += NT) xb[r] = rhs[r];
    double* rbp = v.rbar + D.r_off;
    for (int i = tid; i < m; i += NT) {
        double acc;
        if (i < o1) {
            const double* row = N.R1 + N.opos1[i] * N.m1;
            acc = rb1[N.opos1[i]];
            for (int k = 0; k < g; ++k) acc += row[N.gpos1[k]] * rhs[k];
        } else {
            const double* row = N.R2 + N.opos2[i - o1] * N.m2;
            acc = rb2[N.opos2[i - o1]];
            for (int k = 0; k < g; ++k) acc += row[N.gpos2[k]] * rhs[g + k];
        }
        rbp[i] = acc;
    }
}

// Solve phase, top-down: lambda_gamma = X lambda_o + xbar, scattered into the
// children's Robin data together with the node's own outer data.
template <int NT>
__global__ void __launch_bounds__(NT) merge_down_kernel(DevView v, int first) {
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int g = N.g, g2 = N.g2, m = N.m, o1 = N.o1;
    const int tid = threadIdx.x;
    const double* lam_o = v.lam + D.r_off;
    const double* X = v.X + D.X_off;
    const double* xb = v.xbar + D.xb_off;
    double* l1 = v.lam + D.r1_off;
    double* l2 = v.lam + D.r2_off;
    for (int r = tid; r < g2; r += NT) {
        double acc = xb[r];
        for (int j = 0; j < m; ++j) acc += X[(long long)j * g2 + r] * lam_o[j];
        if (r < g) l1[N.gpos1[r]] = acc;
        else l2[N.gpos2[r - g]] = acc;
    }
    for (int j = tid; j < m; j += NT) {
        if (j < o1) l1[N.opos1[j]] = lam_o[j];
        else l2[N.opos2[j - o1]] = lam_o[j];
    }
}

constexpr int kMergeThreads = 256;
constexpr int kSmemG2 = 128;          // fused path: M in shared memory up to 128 x 128
constexpr int kBlockedBelow = 304;    // levels with fewer nodes take the blocked path

}  // namespace

bool merge_level_blocked(int count, int max_g2) { return max_g2 > kSmemG2 || count < kBlockedBelow; }

cudaError_t launch_merge_build(const DevView& v, int first, int count, int max_g2, int max_m,
                               unsigned long long* amax_bits, cudaStream_t s, int* launches) {
    if (count == 0) return cudaSuccess;
    cudaError_t e;
    if (!merge_level_blocked(count, max_g2)) {
        const size_t sm = (size_t)max_g2 * max_g2 * sizeof(double);
        e = cudaFuncSetAttribute(merge_small_kernel<kMergeThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kSmemG2 * kSmemG2 * sizeof(double)));
        if (e != cudaSuccess) return e;
        merge_small_kernel<kMergeThreads><<<count, kMergeThreads, sm, s>>>(v, first);
        ++*launches;
        return cudaGetLastError();
    }
    e = cudaMemsetAsync(amax_bits, 0, sizeof(unsigned long long) * count, s);
    if (e != cudaSuccess) return e;
    {
        const long long work = (long long)max_g2 * (max_g2 + max_m);
        int gy = (int)((work + 255) / 256);
        gy = gy < 1 ? 1 : (gy > 64 ? 64 : gy);
        merge_assemble_kernel<<<dim3(count, gy), 256, 0, s>>>(v, first, amax_bits);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int k0 = 0; k0 < max_g2; k0 += kNB) {
        lu_panel_kernel<kMergeThreads><<<count, kMergeThreads, 0, s>>>(v, first, k0, amax_bits);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int rest = max_g2 - min(k0 + kNB, max_g2);
        if (rest <= 0) break;
        lu_trsm_kernel<<<dim3(count, (rest + 63) / 64), 64, 0, s>>>(v, first, k0);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int tiles = (rest + kGemmTile - 1) / kGemmTile;
        lu_gemm_kernel<<<dim3(count, tiles * tiles), 256, 0, s>>>(v, first, k0);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (max_m > 0) {
        const size_t sm = (size_t)kXCols * max_g2 * sizeof(double);
        e = cudaFuncSetAttribute(merge_xsolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        merge_xsolve_kernel<<<dim3(count, (max_m + kXCols - 1) / kXCols), 256, sm, s>>>(v, first);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int tiles = (max_m + kRTile - 1) / kRTile;
        merge_rupdate_kernel<<<dim3(count, tiles * tiles), 256, 0, s>>>(v, first);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_merge_up(const DevView& v, int first, int count, int max_g2, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    merge_up_kernel<kMergeThreads><<<count, kMergeThreads, (size_t)max_g2 * sizeof(double), s>>>(v, first);
    return cudaGetLastError();
}

cudaError_t launch_merge_down(const DevView& v, int first, int count, int, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    merge_down_kernel<kMergeThreads><<<count, kMergeThreads, 0, s>>>(v, first);
    return cudaGetLastError();
}

}  // namespace mrcm
