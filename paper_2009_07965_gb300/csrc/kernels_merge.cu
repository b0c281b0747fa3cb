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
// The build also forms W = M^-1 explicitly; X = -W C then exploits the block
// structure of C, and every solve pass is a pair of matrix-vector products
// per node instead of two triangular solves: M is symmetric (R^a, R^b
// symmetric, D diagonal), so blockdiag(R_og) xbar = -C^T M^-1 rbar_gamma
// = X^T rbar_gamma, giving the up-sweep rbar = rbar_o + X^T rbar_gamma, and
// the down-sweep lambda_gamma = X lambda_o + W (-rbar_gamma).  Iterative
// refinement (kernels_refine.cu) absorbs the different rounding of an
// inverse-based solve.
//
// Two launch shapes.  Levels with many nodes: one CTA per node, M in shared
// memory (merge_small_kernel).  Levels with few, large nodes: a blocked
// right-looking LU across many CTAs -- a panel kernel (NB columns, one CTA
// per node), a TRSM kernel for the block row of U and a tiled FP64 GEMM for
// the trailing update -- then W by column blocks, X and R by output tiles.
#include "mrcm_internal.h"

namespace mrcm {
namespace {

constexpr int kNB = 32;         // panel width of the blocked LU
constexpr int kGemmTile = 32;   // trailing-update tile (kGemmTile^2 outputs per CTA)
constexpr int kXCols = 4;       // inverse columns per CTA
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
                                        double* dinv, double* sv, int* si, double* s_rcp, bool& singular) {
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
        dinv[k] = *s_rcp;
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
    const double thresh = 1e-14 * block_max<NT>(amax, sv);
    bool singular = false;
    for (int k = 0; k < g2; ++k)
        lu_step<NT>(M, g2, k, (k / kNB) * kNB, g2, thresh, piv, v.udinv + D.xb_off, sv, si, &s_rcp, singular);
    if (singular && tid == 0) atomicOr(v.status, kStatusSingular);
    // W = M^-1, one column per thread (per panel: exchanges, unit lower
    // columns; then the upper triangle)
    double* Wg = v.W + D.LU_off;
    for (int j = tid; j < g2; j += NT) {
        double* x = Wg + (long long)j * g2;
        for (int i = 0; i < g2; ++i) x[i] = (i == j) ? 1.0 : 0.0;
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
    // X = -W C: C is block diagonal, so column j uses one half of W
    for (int idx = tid; idx < g2 * m; idx += NT) {
        const int r = idx % g2, j = idx / g2;
        double acc = 0.0;
        if (j < N.o1) {
            const double* crow = N.R1 + N.opos1[j];
            for (int k = 0; k < N.g; ++k) acc += Wg[(long long)k * g2 + r] * crow[N.gpos1[k] * N.m1];
        } else {
            const double* crow = N.R2 + N.opos2[j - N.o1];
            for (int k = 0; k < N.g; ++k)
                acc += Wg[(long long)(N.g + k) * g2 + r] * crow[N.gpos2[k] * N.m2];
        }
        X[idx] = -acc;
    }
    __syncthreads();
    double* Rp = v.R + D.R_off;
    for (int idx = tid; idx < m * m; idx += NT) Rp[idx] = r_entry(N, X, idx / m, idx % m);
}

// ---------------------------------------------------------------------------
// Blocked path.
// Assembly of M (column-major, pinned rows applied).
__global__ void __launch_bounds__(256) merge_assemble_kernel(DevView v, int first, unsigned long long* amax_bits) {
    const int node = first + blockIdx.x;
    const MergeDesc D = v.merges[node];
    const NodeRefs N = node_refs(v, D);
    const int g2 = N.g2, m = N.m;
    double* M = v.LU + D.LU_off;
    const long long nM = (long long)g2 * g2;
    double amax = 0.0;
    for (long long idx = blockIdx.y * 256LL + threadIdx.x; idx < nM; idx += (long long)gridDim.y * 256) {
        const int r = (int)(idx % g2), c = (int)(idx / g2);
        const double val = m_entry_pinned(v, D, N, r, c);
        M[idx] = val;
        amax = fmax(amax, fabs(val));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.0)
        atomicMax(amax_bits + (node - first), (unsigned long long)__double_as_longlong(amax));
}

// Panel factorisation of columns [k0, k0+NB) (rows k0..2g-1), one CTA per
// node; the panel is staged in shared memory when it fits (smem_rows).
template <int NT>
__global__ void __launch_bounds__(NT) lu_panel_kernel(DevView v, int first, int k0,
                                                      const unsigned long long* amax_bits, int smem_rows) {
    extern __shared__ __align__(16) double Ps[];
    __shared__ unsigned long long skey[NT / 32];
    __shared__ int si[NT / 32];
    __shared__ int s_p;
    __shared__ double s_rcp;
    __shared__ double prow[kNB], krow[kNB];
    const MergeDesc D = v.merges[first + blockIdx.x];
    const int g2 = 2 * D.g;
    if (k0 >= g2) return;
    const int nb = min(kNB, g2 - k0), rows = g2 - k0;
    double* Mg = v.LU + D.LU_off;
    int* piv = v.piv + D.piv_off;
    double* dinv = v.udinv + D.xb_off;
    const int tid = threadIdx.x;
    const bool staged = rows <= smem_rows;
    // shared memory: the multipliers of one step (rows), then the staged panel
    double* lmul = Ps;
    double* P = staged ? Ps + rows : Mg + (long long)k0 * g2 + k0;   // entry (i, c) at P[c * ld + i]
    const int ld = staged ? rows : g2;
    if (staged) {
        for (int idx = tid; idx < rows * nb; idx += NT) {
            const int i = idx % rows, c = idx / rows;
            P[idx] = Mg[(long long)(k0 + c) * g2 + k0 + i];
        }
        __syncthreads();
    }
    const double thresh = 1e-14 * __longlong_as_double((long long)amax_bits[blockIdx.x]);
    bool singular = false;
    for (int kk = 0; kk < nb; ++kk) {
        // pivot search on the bit patterns of |a| (ordered like the values)
        unsigned long long best = 0ull;
        int bi = kk;
        const double* col = P + (long long)kk * ld;
        for (int i = kk + tid; i < rows; i += NT) {
            const unsigned long long a = (unsigned long long)__double_as_longlong(col[i]) & 0x7fffffffffffffffull;
            if (a > best || (a == best && i < bi)) { best = a; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { skey[tid >> 5] = best; si[tid >> 5] = bi; }
        __syncthreads();
        if (tid < 32) {
            unsigned long long kv = tid < NT / 32 ? skey[tid] : 0ull;
            int ki = tid < NT / 32 ? si[tid] : 0x7fffffff;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ov = __shfl_down_sync(0xffffffffu, kv, o);
                const int oi = __shfl_down_sync(0xffffffffu, ki, o);
                if (ov > kv || (ov == kv && oi < ki)) { kv = ov; ki = oi; }
            }
            ki = __shfl_sync(0xffffffffu, ki, 0);
            // the pivot row (old row p) and the old row kk, all panel columns
            if (tid < nb) {
                prow[tid] = P[(long long)tid * ld + ki];
                krow[tid] = P[(long long)tid * ld + kk];
            }
            if (tid == 0) {
                const double pivot = P[(long long)kk * ld + ki];
                const double rcp = 1.0 / pivot;          // one warp: FP64 issue slots are scarce
                if (!(fabs(pivot) > thresh)) singular = true;
                s_rcp = rcp;
                s_p = ki;
                piv[k0 + kk] = k0 + ki;
                dinv[k0 + kk] = rcp;
            }
        }
        __syncthreads();
        const int p = s_p;
        const double rcp = s_rcp;
        const int nr = rows - kk - 1;
        // multipliers, one lane per row (dense warps)
        for (int r = tid; r < nr; r += NT) {
            const int i = kk + 1 + r;
            lmul[r] = (i == p ? krow[kk] : col[i]) * rcp;
        }
        if (tid < nb) P[(long long)tid * ld + kk] = prow[tid];       // row kk <- pivot row
        __syncthreads();
        // rank-1 update of columns kk+1.., (row, column) pairs over all lanes;
        // row p takes the old row kk's values, its multipliers included
        const int ncu = nb - kk - 1;
        for (int idx = tid; idx < nr * ncu; idx += NT) {
            const int r = idx % nr, i = kk + 1 + r, c = kk + 1 + idx / nr;
            const double a = (i == p) ? krow[c] : P[(long long)c * ld + i];
            P[(long long)c * ld + i] = a - lmul[r] * prow[c];
        }
        for (int r = tid; r < nr; r += NT) P[(long long)kk * ld + kk + 1 + r] = lmul[r];
        if (p > kk)
            for (int c = tid; c < kk; c += NT) P[(long long)c * ld + p] = krow[c];
        __syncthreads();
    }
    if (singular && tid == 0) atomicOr(v.status, kStatusSingular);
    if (staged) {
        for (int idx = tid; idx < rows * nb; idx += NT) {
            const int i = idx % rows, c = idx / rows;
            Mg[(long long)(k0 + c) * g2 + k0 + i] = P[idx];
        }
    }
}

// Block row of U: the panel's exchanges applied to columns [kend, 2g) (as one
// composed permutation of the touched rows), then U12 = L11^-1 A12 with one
// warp per column (lane r holds row k0 + r).
constexpr int kTrsmWarps = 8;
__global__ void __launch_bounds__(32 * kTrsmWarps) lu_trsm_kernel(DevView v, int first, int k0) {
    __shared__ double L11[kNB][kNB + 1];
    __shared__ int rows_touched[2 * kNB];
    __shared__ int src_row[2 * kNB];
    __shared__ int n_touched;
    const MergeDesc D = v.merges[first + blockIdx.x];
    const int g2 = 2 * D.g;
    const int kend = min(k0 + kNB, g2);
    if (kend >= g2 || kend + (int)blockIdx.y * kTrsmWarps >= g2) return;   // uniform per CTA
    double* M = v.LU + D.LU_off;
    const int* piv = v.piv + D.piv_off;
    const int nb = kend - k0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int idx = tid; idx < kNB * kNB; idx += 32 * kTrsmWarps) {
        const int r = idx % kNB, c = idx / kNB;
        L11[r][c] = (r < nb && c < nb) ? M[(long long)(k0 + c) * g2 + k0 + r] : 0.0;
    }
    if (tid == 0) {
        // rows touched by the exchanges and, after all of them, the original
        // row whose value each touched row holds
        int n = 0;
        for (int c = 0; c < nb; ++c) { rows_touched[n] = k0 + c; src_row[n] = k0 + c; ++n; }
        for (int c = 0; c < nb; ++c) {
            const int p = piv[k0 + c];
            int ip = -1;
            for (int q = 0; q < n; ++q) if (rows_touched[q] == p) ip = q;
            if (ip < 0) { rows_touched[n] = p; src_row[n] = p; ip = n; ++n; }
            const int t = src_row[c];
            src_row[c] = src_row[ip];
            src_row[ip] = t;
        }
        n_touched = n;
    }
    __syncthreads();
    const int j = kend + blockIdx.y * kTrsmWarps + warp;
    if (j >= g2) return;
    double* col = M + (long long)j * g2;
    const int nt = n_touched;
    double g0 = lane < nt ? col[src_row[lane]] : 0.0;
    double g1 = lane + 32 < nt ? col[src_row[lane + 32]] : 0.0;
    __syncwarp();
    if (lane < nt) col[rows_touched[lane]] = g0;
    if (lane + 32 < nt) col[rows_touched[lane + 32]] = g1;
    __syncwarp();
    double u = lane < nb ? col[k0 + lane] : 0.0;
    for (int c = 0; c < nb; ++c) {
        const double xc = __shfl_sync(0xffffffffu, u, c);
        if (lane > c && lane < nb) u -= L11[lane][c] * xc;
    }
    if (lane < nb) col[k0 + lane] = u;
}

// Trailing update A22 -= L21 U12 on kGemmTile^2 tiles; 256 threads, 2x2 each.
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
    constexpr int TS = kGemmTile / 16;                // outputs per thread per dimension
    const int tr = (tid % 16) * TS, tc = (tid / 16) * TS;
    double acc[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) acc[a][b] = 0.0;
#pragma unroll 8
    for (int c = 0; c < kNB; ++c) {
        double lv[TS], uv[TS];
#pragma unroll
        for (int a = 0; a < TS; ++a) { lv[a] = Ls[c][tr + a]; uv[a] = Us[c][tc + a]; }
#pragma unroll
        for (int a = 0; a < TS; ++a)
#pragma unroll
            for (int b = 0; b < TS; ++b) acc[a][b] += lv[a] * uv[b];
    }
#pragma unroll
    for (int b = 0; b < TS; ++b) {
        const int j = j0 + tc + b;
        if (j >= g2) continue;
        double* col = M + (long long)j * g2;
#pragma unroll
        for (int a = 0; a < TS; ++a) {
            const int r = r0 + tr + a;
            if (r < g2) col[r] -= acc[a][b];
        }
    }
}

// W = M^-1 for kXCols columns per CTA (identity columns staged in shared
// memory).  Blocked like the factorisation: per 32-row block, warp j solves
// the diagonal block for column j with shuffles (block rows preloaded into
// registers), then every thread updates one remaining row for all columns.
__global__ void __launch_bounds__(32 * kXCols) merge_inverse_kernel(DevView v, int first) {
    extern __shared__ __align__(16) double xs[];   // kXCols x 2g
    const MergeDesc D = v.merges[first + blockIdx.x];
    const int g2 = 2 * D.g;
    const int j0 = blockIdx.y * kXCols;
    if (j0 >= g2) return;                             // uniform per CTA
    const int nc = min(kXCols, g2 - j0);
    const double* M = v.LU + D.LU_off;
    const int* piv = v.piv + D.piv_off;
    const double* dinv = v.udinv + D.xb_off;
    double* X = v.W + D.LU_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NT = 32 * kXCols;
    for (int idx = tid; idx < nc * g2; idx += NT) xs[idx] = (idx % g2 == j0 + idx / g2) ? 1.0 : 0.0;
    __syncthreads();
    // forward: per panel, its exchanges, the unit lower diagonal block, then
    // the rows below
    for (int k0 = 0; k0 < g2; k0 += kNB) {
        const int nb = min(kNB, g2 - k0);
        if (warp < nc) {
            double* x = xs + warp * g2;
            double Lr[kNB];
#pragma unroll
            for (int c = 0; c < kNB; ++c)
                Lr[c] = (c < nb && lane < nb) ? M[(long long)(k0 + c) * g2 + k0 + lane] : 0.0;
            if (lane == 0) {
                for (int k = k0; k < k0 + nb; ++k) {
                    const int p = piv[k];
                    if (p != k) { const double a = x[p]; x[p] = x[k]; x[k] = a; }
                }
            }
            __syncwarp();
            double val = lane < nb ? x[k0 + lane] : 0.0;
#pragma unroll
            for (int c = 0; c < kNB; ++c) {
                const double xc = __shfl_sync(0xffffffffu, val, c);
                if (lane > c) val -= Lr[c] * xc;
            }
            if (lane < nb) x[k0 + lane] = val;
        }
        __syncthreads();
        for (int i = k0 + nb + tid; i < g2; i += NT) {
            double Li[kNB];
#pragma unroll
            for (int c = 0; c < kNB; ++c) Li[c] = c < nb ? M[(long long)(k0 + c) * g2 + i] : 0.0;
            for (int j = 0; j < nc; ++j) {
                const double* x = xs + j * g2 + k0;
                double acc = 0.0;
#pragma unroll
                for (int c = 0; c < kNB; ++c) acc += Li[c] * (c < nb ? x[c] : 0.0);
                xs[j * g2 + i] -= acc;
            }
        }
        __syncthreads();
    }
    // backward: U with the reciprocals of its diagonal, blocks from the bottom
    for (int blk = (g2 - 1) / kNB; blk >= 0; --blk) {
        const int k0 = blk * kNB, nb = min(kNB, g2 - k0);
        if (warp < nc) {
            double* x = xs + warp * g2;
            double Ur[kNB];
#pragma unroll
            for (int c = 0; c < kNB; ++c)
                Ur[c] = (c < nb && lane < nb) ? M[(long long)(k0 + c) * g2 + k0 + lane] : 0.0;
            const double dl = lane < nb ? dinv[k0 + lane] : 0.0;
            double val = lane < nb ? x[k0 + lane] : 0.0;
#pragma unroll
            for (int c = kNB - 1; c >= 0; --c) {
                if (lane == c) val *= dl;
                const double xc = __shfl_sync(0xffffffffu, val, c);
                if (lane < c) val -= Ur[c] * xc;
            }
            if (lane < nb) x[k0 + lane] = val;
        }
        __syncthreads();
        for (int i = tid; i < k0; i += NT) {
            double Ui[kNB];
#pragma unroll
            for (int c = 0; c < kNB; ++c) Ui[c] = c < nb ? M[(long long)(k0 + c) * g2 + i] : 0.0;
            for (int j = 0; j < nc; ++j) {
                const double* x = xs + j * g2 + k0;
                double acc = 0.0;
#pragma unroll
                for (int c = 0; c < kNB; ++c) acc += Ui[c] * (c < nb ? x[c] : 0.0);
                xs[j * g2 + i] -= acc;
            }
        }
        __syncthreads();
    }
    for (int idx = tid; idx < nc * g2; idx += NT) X[(long long)j0 * g2 + idx] = xs[idx];
}

// X = -W C with C = blockdiag(R^a_go, R^b_go): column j < o1 uses the first
// g columns of W, the others the last g.  A CTA computes 64 rows x 16
// columns; the gathered entries of C are staged in shared memory in chunks.
constexpr int kXRows = 64, kXColsOut = 16, kXChunk = 64;
__global__ void __launch_bounds__(256) merge_x_kernel(DevView v, int first) {
    __shared__ double Cs[kXChunk][kXColsOut];
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int g = N.g, g2 = N.g2, m = N.m;
    const int rt = (g2 + kXRows - 1) / kXRows;
    const int r0 = (blockIdx.y % rt) * kXRows, j0 = (blockIdx.y / rt) * kXColsOut;
    if (j0 >= m) return;                              // uniform per CTA
    const double* W = v.W + D.LU_off;
    double* X = v.X + D.X_off;
    const int tid = threadIdx.x, rl = tid % kXRows, cg = tid / kXRows;   // 4 groups of 4 columns
    const int r = r0 + rl;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    // columns of this CTA may straddle o1: treat the two halves separately
    for (int half = 0; half < 2; ++half) {
        const int jlo = half == 0 ? 0 : N.o1, jhi = half == 0 ? N.o1 : m;
        if (j0 + kXColsOut <= jlo || j0 >= jhi) continue;  // uniform
        for (int k0 = 0; k0 < g; k0 += kXChunk) {
            const int kn = min(kXChunk, g - k0);
            __syncthreads();
            for (int idx = tid; idx < kXChunk * kXColsOut; idx += 256) {
                const int kk = idx / kXColsOut, jj = idx % kXColsOut, j = j0 + jj;
                double c = 0.0;
                if (kk < kn && j >= jlo && j < jhi) {
                    c = half == 0 ? N.R1[N.gpos1[k0 + kk] * N.m1 + N.opos1[j]]
                                  : N.R2[N.gpos2[k0 + kk] * N.m2 + N.opos2[j - N.o1]];
                }
                Cs[kk][jj] = c;
            }
            __syncthreads();
            if (r < g2) {
                const double* wcol = W + (long long)(half * g + k0) * g2 + r;
                for (int kk = 0; kk < kn; ++kk) {
                    const double wv = wcol[(long long)kk * g2];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] += wv * Cs[kk][cg * 4 + q];
                }
            }
        }
    }
    if (r < g2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + cg * 4 + q;
            if (j < m) X[(long long)j * g2 + r] = -acc[q];
        }
    }
}

// R = blockdiag(R_oo) + blockdiag(R_og) X on kRTile^2 output tiles: row i
// of the tile uses the gathered row of R^a (i < o1) or R^b and the matching
// half of X; both are staged in shared memory in chunks of kRTile.
__global__ void __launch_bounds__(256) merge_rupdate_kernel(DevView v, int first) {
    __shared__ double Cs[kRTile][kRTile + 1];        // Cs[row][k]
    __shared__ double Xs[2][kRTile][kRTile + 1];     // Xs[half][k][col]
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int m = N.m, g = N.g, g2 = N.g2, o1 = N.o1;
    const int tiles = (m + kRTile - 1) / kRTile;
    if ((int)blockIdx.y >= tiles * tiles) return;
    const int i0 = (blockIdx.y % tiles) * kRTile, jt = (blockIdx.y / tiles) * kRTile;
    const double* X = v.X + D.X_off;
    double* Rp = v.R + D.R_off;
    const int tid = threadIdx.x;
    constexpr int TS = kRTile / 16;
    const int tr = (tid % 16) * TS, tc = (tid / 16) * TS;
    double acc[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < g; k0 += kRTile) {
        const int kn = min(kRTile, g - k0);
        __syncthreads();
        for (int idx = tid; idx < kRTile * kRTile; idx += 256) {
            const int rr = idx / kRTile, kk = idx % kRTile, i = i0 + rr;
            double c = 0.0;
            if (kk < kn && i < m)
                c = i < o1 ? N.R1[N.opos1[i] * N.m1 + N.gpos1[k0 + kk]]
                           : N.R2[N.opos2[i - o1] * N.m2 + N.gpos2[k0 + kk]];
            Cs[rr][kk] = c;
        }
        for (int idx = tid; idx < 2 * kRTile * kRTile; idx += 256) {
            const int half = idx / (kRTile * kRTile), rem = idx % (kRTile * kRTile);
            const int kk = rem % kRTile, jj = rem / kRTile, j = jt + jj;
            Xs[half][kk][jj] = (kk < kn && j < m) ? X[(long long)j * g2 + half * g + k0 + kk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < TS; ++a) {
            const int half = (i0 + tr + a) < o1 ? 0 : 1;
            for (int kk = 0; kk < kRTile; ++kk) {
                const double cv = Cs[tr + a][kk];
#pragma unroll
                for (int b = 0; b < TS; ++b) acc[a][b] += cv * Xs[half][kk][tc + b];
            }
        }
    }
#pragma unroll
    for (int a = 0; a < TS; ++a) {
        const int i = i0 + tr + a;
        if (i >= m) continue;
        const double* row = i < o1 ? N.R1 + N.opos1[i] * N.m1 : N.R2 + N.opos2[i - o1] * N.m2;
#pragma unroll
        for (int b = 0; b < TS; ++b) {
            const int j = jt + tc + b;
            if (j >= m) continue;
            double val = acc[a][b];
            if (i < o1 && j < o1) val += row[N.opos1[j]];
            if (i >= o1 && j >= o1) val += row[N.opos2[j - o1]];
            Rp[(long long)i * m + j] = val;
        }
    }
}

// Solve phase, bottom-up: the node's particular fluxes
// rbar = rbar_o + X^T rbar_gamma (Eqs. particular.1-2 with M symmetric); one
// warp per output, lanes split the sum over gamma.
constexpr int kUpOut = 32;
__global__ void __launch_bounds__(256) merge_up_kernel(DevView v, int first) {
    extern __shared__ __align__(16) double rg[];     // rbar_gamma (2g)
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int g = N.g, g2 = N.g2, m = N.m, o1 = N.o1;
    const int i0 = blockIdx.y * kUpOut;
    if (i0 >= m) return;                              // uniform per CTA
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double* rb1 = v.rbar + D.r1_off;
    const double* rb2 = v.rbar + D.r2_off;
    for (int r = tid; r < g2; r += 256) rg[r] = r < g ? rb1[N.gpos1[r]] : rb2[N.gpos2[r - g]];
    __syncthreads();
    const double* X = v.X + D.X_off;
    double* rbp = v.rbar + D.r_off;
    for (int i = i0 + warp; i < min(i0 + kUpOut, m); i += 8) {
        const double* xc = X + (long long)i * g2;
        double acc = 0.0;
        for (int k = lane; k < g2; k += 32) acc += xc[k] * rg[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) rbp[i] = acc + (i < o1 ? rb1[N.opos1[i]] : rb2[N.opos2[i - o1]]);
    }
}

// Solve phase, top-down: lambda_gamma = X lambda_o + W (-rbar_gamma) (with
// the pinning rows of an all-Neumann root applied to the right-hand side),
// scattered into the children's Robin data together with the node's own
// outer data.  A CTA covers 64 rows of gamma; four thread groups split the
// sums.
constexpr int kDownRows = 32, kDownGroups = 8;
__global__ void __launch_bounds__(256) merge_down_kernel(DevView v, int first) {
    extern __shared__ __align__(16) double rhs[];    // -rbar_gamma (2g)
    __shared__ double part[kDownGroups][kDownRows];
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int g = N.g, g2 = N.g2, m = N.m, o1 = N.o1;
    const int r0 = blockIdx.y * kDownRows;
    if (r0 >= g2) return;                                // uniform per CTA
    const int tid = threadIdx.x, rl = tid % kDownRows, grp = tid / kDownRows;
    const double* rb1 = v.rbar + D.r1_off;
    const double* rb2 = v.rbar + D.r2_off;
    for (int r = tid; r < g2; r += 256) rhs[r] = -(r < g ? rb1[N.gpos1[r]] : rb2[N.gpos2[r - g]]);
    __syncthreads();
    if (D.pinned && tid == 0) {
        const double a = rhs[0], b = rhs[g];
        rhs[g] = a - b;
        rhs[0] = 0.0;
    }
    __syncthreads();
    const double* lam_o = v.lam + D.r_off;
    const double* X = v.X + D.X_off;
    const double* W = v.W + D.LU_off;
    double* l1 = v.lam + D.r1_off;
    double* l2 = v.lam + D.r2_off;
    const int r = r0 + rl;
    double acc = 0.0;
    if (r < g2) {
        for (int j = grp; j < m; j += kDownGroups) acc += X[(long long)j * g2 + r] * lam_o[j];
        for (int k = grp; k < g2; k += kDownGroups) acc += W[(long long)k * g2 + r] * rhs[k];
    }
    part[grp][rl] = acc;
    __syncthreads();
    if (grp == 0 && r < g2) {
        double lg = 0.0;
#pragma unroll
        for (int q = 0; q < kDownGroups; ++q) lg += part[q][rl];
        if (r < g) l1[N.gpos1[r]] = lg;
        else l2[N.gpos2[r - g]] = lg;
    }
    if (blockIdx.y == 0) {
        for (int j = tid; j < m; j += 256) {
            if (j < o1) l1[N.opos1[j]] = lam_o[j];
            else l2[N.opos2[j - o1]] = lam_o[j];
        }
    }
}

constexpr int kMergeThreads = 256;
constexpr int kPanelThreads = 512;
constexpr int kPanelSmemBytes = 200 * 1024;
constexpr int kSmemG2 = 128;          // fused path: M in shared memory up to 128 x 128
constexpr int kBlockedBelow = 304;    // levels with fewer nodes take the blocked path

}  // namespace

bool merge_level_blocked(int count, int max_g2) { return max_g2 > kSmemG2 || count < kBlockedBelow; }

// phase ids (include/mrcm.h)
enum { kPhMergeSmall = 2, kPhLuPanel = 3, kPhLuUpdate = 4, kPhMergeInverse = 5, kPhMergeProducts = 6 };

struct HookScope {
    const PhaseHook& h;
    int phase;
    HookScope(const PhaseHook& h_, int p) : h(h_), phase(p) { if (h.begin) h.begin(h.ctx, p); }
    ~HookScope() { if (h.end) h.end(h.ctx, phase); }
};

cudaError_t launch_merge_build(const DevView& v, int first, int count, int max_g2, int max_m,
                               unsigned long long* amax_bits, cudaStream_t s, int* launches,
                               const PhaseHook& hook) {
    static_assert(kNB == kMergePanel, "flop model panel width");
    if (count == 0) return cudaSuccess;
    cudaError_t e;
    if (!merge_level_blocked(count, max_g2)) {
        HookScope hs(hook, kPhMergeSmall);
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
        HookScope hs(hook, kPhMergeProducts);
        const long long work = (long long)max_g2 * (max_g2 + max_m);
        int gy = (int)((work + 255) / 256);
        gy = gy < 1 ? 1 : (gy > 64 ? 64 : gy);
        merge_assemble_kernel<<<dim3(count, gy), 256, 0, s>>>(v, first, amax_bits);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int smem_rows = kPanelSmemBytes / ((kNB + 1) * (int)sizeof(double));
    e = cudaFuncSetAttribute(lu_panel_kernel<kPanelThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kPanelSmemBytes);
    if (e != cudaSuccess) return e;
    for (int k0 = 0; k0 < max_g2; k0 += kNB) {
        const int rows = max_g2 - k0;
        const bool staged = rows <= smem_rows;
        const size_t psm = (size_t)rows * (staged ? kNB + 1 : 1) * sizeof(double);
        {
            HookScope hs(hook, kPhLuPanel);
            lu_panel_kernel<kPanelThreads><<<count, kPanelThreads, psm, s>>>(v, first, k0, amax_bits,
                                                                              staged ? smem_rows : 0);
            ++*launches;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        const int rest = max_g2 - min(k0 + kNB, max_g2);
        if (rest <= 0) break;
        HookScope hs(hook, kPhLuUpdate);
        lu_trsm_kernel<<<dim3(count, (rest + kTrsmWarps - 1) / kTrsmWarps), 32 * kTrsmWarps, 0, s>>>(v, first, k0);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int tiles = (rest + kGemmTile - 1) / kGemmTile;
        lu_gemm_kernel<<<dim3(count, tiles * tiles), 256, 0, s>>>(v, first, k0);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        HookScope hs(hook, kPhMergeInverse);
        const size_t sm = (size_t)kXCols * max_g2 * sizeof(double);
        e = cudaFuncSetAttribute(merge_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        merge_inverse_kernel<<<dim3(count, (max_g2 + kXCols - 1) / kXCols), 32 * kXCols, sm, s>>>(v, first);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (max_m > 0) {
        HookScope hs(hook, kPhMergeProducts);
        const int rt = (max_g2 + kXRows - 1) / kXRows, ct = (max_m + kXColsOut - 1) / kXColsOut;
        merge_x_kernel<<<dim3(count, rt * ct), 256, 0, s>>>(v, first);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int tiles = (max_m + kRTile - 1) / kRTile;
        merge_rupdate_kernel<<<dim3(count, tiles * tiles), 256, 0, s>>>(v, first);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_merge_up(const DevView& v, int first, int count, int max_g2, int max_m, cudaStream_t s) {
    if (count == 0 || max_m == 0) return cudaSuccess;
    merge_up_kernel<<<dim3(count, (max_m + kUpOut - 1) / kUpOut), 256, (size_t)max_g2 * sizeof(double), s>>>(
        v, first);
    return cudaGetLastError();
}

cudaError_t launch_merge_down(const DevView& v, int first, int count, int max_g2, int, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    merge_down_kernel<<<dim3(count, (max_g2 + kDownRows - 1) / kDownRows), 256, (size_t)max_g2 * sizeof(double),
                        s>>>(v, first);
    return cudaGetLastError();
}

}  // namespace mrcm
