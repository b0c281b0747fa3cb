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
// One CTA per node; M is LU-factored with partial pivoting (rows swapped
// explicitly, pivots recorded for the solve phase).
#include "mrcm_internal.h"

namespace mrcm {
namespace {

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

template <int NT>
__device__ __forceinline__ void block_argmax(double val, int idx, double* sv, int* si, int& out_idx) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, val, o);
        const int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    if (lane == 0) { sv[wid] = val; si[wid] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = sv[0]; int bi = si[0];
        for (int w = 1; w < NT / 32; ++w)
            if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
        si[0] = bi;
    }
    __syncthreads();
    out_idx = si[0];
    __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) merge_build_kernel(DevView v, int first, int smem_g2) {
    extern __shared__ __align__(16) double sm[];
    __shared__ double red_v[NT / 32];
    __shared__ int red_i[NT / 32];
    __shared__ double s_maxabs;
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int g = N.g, g2 = N.g2, m = N.m, o1 = N.o1;
    const int tid = threadIdx.x;
    double* Mg = v.LU + D.LU_off;
    const bool in_smem = g2 <= smem_g2;
    double* M = in_smem ? sm : Mg;
    int* piv = v.piv + D.piv_off;
    double* X = v.X + D.X_off;

    // ---- assemble M and C ---------------------------------------------------
    double amax = 0.0;
    for (int idx = tid; idx < g2 * g2; idx += NT) {
        const int r = idx / g2, c = idx % g2;
        double val = 0.0;
        if (r < g && c < g) {
            val = N.R1[N.gpos1[r] * N.m1 + N.gpos1[c]];
            if (r == c) val += v.seg_D[v.gamma_segs[D.gamma_off + r]];
        } else if (r >= g && c >= g) {
            val = N.R2[N.gpos2[r - g] * N.m2 + N.gpos2[c - g]];
            if (r == c) val += v.seg_D[v.gamma_segs[D.gamma_off + r - g]];
        } else if (r < g && c - g == r) {
            val = -v.seg_D[v.gamma_segs[D.gamma_off + r]];
        } else if (r >= g && r - g == c) {
            val = -v.seg_D[v.gamma_segs[D.gamma_off + c]];
        }
        M[idx] = val;
        amax = fmax(amax, fabs(val));
    }
    for (int idx = tid; idx < g2 * m; idx += NT) {
        const int r = idx / m, c = idx % m;
        double val = 0.0;
        if (r < g && c < o1) val = N.R1[N.gpos1[r] * N.m1 + N.opos1[c]];
        else if (r >= g && c >= o1) val = N.R2[N.gpos2[r - g] * N.m2 + N.opos2[c - o1]];
        X[idx] = val;
    }
    {
        // block maximum of |M| (threshold of the singular-pivot test)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_down_sync(0xffffffffu, amax, o));
        if ((tid & 31) == 0) red_v[tid >> 5] = amax;
        __syncthreads();
        if (tid == 0) {
            double mx = 0.0;
            for (int w = 0; w < NT / 32; ++w) mx = fmax(mx, red_v[w]);
            s_maxabs = mx;
        }
        __syncthreads();
    }
    if (D.pinned) {
        for (int c = tid; c < g2; c += NT) {
            const double a = M[c], b = M[g * g2 + c];
            M[g * g2 + c] = a - b;
            M[c] = (c == 0 || c == g) ? 1.0 : 0.0;
        }
        __syncthreads();
    }
    const double thresh = 1e-14 * s_maxabs;

    // ---- LU with partial pivoting -------------------------------------------
    bool singular = false;
    for (int k = 0; k < g2; ++k) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < g2; i += NT) {
            const double a = fabs(M[i * g2 + k]);
            if (a > best) { best = a; bi = i; }
        }
        int p;
        block_argmax<NT>(best, bi, red_v, red_i, p);
        if (tid == 0) piv[k] = p;
        if (p != k) {
            for (int c = tid; c < g2; c += NT) {
                const double a = M[k * g2 + c];
                M[k * g2 + c] = M[p * g2 + c];
                M[p * g2 + c] = a;
            }
            __syncthreads();
        }
        const double pivot = M[k * g2 + k];
        if (!(fabs(pivot) > thresh)) singular = true;
        const double rcp = 1.0 / pivot;
        for (int i = k + 1 + tid; i < g2; i += NT) M[i * g2 + k] *= rcp;
        __syncthreads();
        const int nt = g2 - k - 1;
        for (int idx = tid; idx < nt * nt; idx += NT) {
            const int i = k + 1 + idx / nt, j = k + 1 + idx % nt;
            M[i * g2 + j] -= M[i * g2 + k] * M[k * g2 + j];
        }
        __syncthreads();
    }
    if (singular && tid == 0) atomicOr(v.status, kStatusSingular);

    // ---- X = -M^-1 C, one column per thread ----------------------------------
    for (int j = tid; j < m; j += NT) {
        for (int k = 0; k < g2; ++k) {
            const int p = piv[k];
            if (p != k) {
                const double a = X[k * m + j];
                X[k * m + j] = X[p * m + j];
                X[p * m + j] = a;
            }
        }
        for (int i = 1; i < g2; ++i) {
            double acc = X[i * m + j];
            for (int k = 0; k < i; ++k) acc -= M[i * g2 + k] * X[k * m + j];
            X[i * m + j] = acc;
        }
        for (int i = g2 - 1; i >= 0; --i) {
            double acc = X[i * m + j];
            for (int k = i + 1; k < g2; ++k) acc -= M[i * g2 + k] * X[k * m + j];
            X[i * m + j] = acc / M[i * g2 + i];
        }
        for (int i = 0; i < g2; ++i) X[i * m + j] = -X[i * m + j];
    }
    __syncthreads();

    // ---- node map R = blockdiag(R_oo) + blockdiag(R_og) X ---------------------
    double* Rp = v.R + D.R_off;
    for (int idx = tid; idx < m * m; idx += NT) {
        const int i = idx / m, j = idx % m;
        double acc = 0.0;
        if (i < o1) {
            const double* row = N.R1 + N.opos1[i] * N.m1;
            if (j < o1) acc = row[N.opos1[j]];
            for (int k = 0; k < g; ++k) acc += row[N.gpos1[k]] * X[k * m + j];
        } else {
            const double* row = N.R2 + N.opos2[i - o1] * N.m2;
            if (j >= o1) acc = row[N.opos2[j - o1]];
            for (int k = 0; k < g; ++k) acc += row[N.gpos2[k]] * X[(g + k) * m + j];
        }
        Rp[idx] = acc;
    }
    if (in_smem) {
        for (int idx = tid; idx < g2 * g2; idx += NT) Mg[idx] = M[idx];
    }
}

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
    if (tid == 0) {
        if (D.pinned) {
            const double a = rhs[0], b = rhs[g];
            rhs[g] = a - b;
            rhs[0] = 0.0;
        }
        for (int k = 0; k < g2; ++k) {
            const int p = piv[k];
            if (p != k) { const double a = rhs[k]; rhs[k] = rhs[p]; rhs[p] = a; }
        }
    }
    __syncthreads();
    for (int k = 0; k < g2; ++k) {
        const double xk = rhs[k];
        for (int i = k + 1 + tid; i < g2; i += NT) rhs[i] -= M[i * g2 + k] * xk;
        __syncthreads();
    }
    for (int k = g2 - 1; k >= 0; --k) {
        if (tid == 0) rhs[k] /= M[k * g2 + k];
        __syncthreads();
        const double xk = rhs[k];
        for (int i = tid; i < k; i += NT) rhs[i] -= M[i * g2 + k] * xk;
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
        for (int j = 0; j < m; ++j) acc += X[r * m + j] * lam_o[j];
        if (r < g) l1[N.gpos1[r]] = acc;
        else l2[N.gpos2[r - g]] = acc;
    }
    for (int j = tid; j < m; j += NT) {
        if (j < o1) l1[N.opos1[j]] = lam_o[j];
        else l2[N.opos2[j - o1]] = lam_o[j];
    }
}

constexpr int kMergeThreads = 256;
constexpr int kSmemG2 = 128;   // interface systems up to 128 x 128 factor in shared memory

}  // namespace

cudaError_t launch_merge_build(const DevView& v, int first, int count, int max_g2, int,
                               cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int smem_g2 = max_g2 <= kSmemG2 ? max_g2 : 0;
    const size_t sm = (size_t)smem_g2 * smem_g2 * sizeof(double);
    cudaFuncSetAttribute(merge_build_kernel<kMergeThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kSmemG2 * kSmemG2 * sizeof(double)));
    merge_build_kernel<kMergeThreads><<<count, kMergeThreads, sm, s>>>(v, first, smem_g2);
    return cudaGetLastError();
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
