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
//
// Quasi-definite form.  M is symmetric but indefinite.  With the scaled
// maps Rh^c = D^-1/2 R^c_gg D^-1/2 and the sum / difference variables
//     s = (xh + yh) / sqrt2,  d = (yh - xh) / sqrt2,   xh = D^1/2 lambda^a, yh = D^1/2 lambda^b,
// the system becomes T [d; s] = (scaled right-hand side) with
//     T = [[A_d, E], [E, -A_s]],  A_d = 2I + (Rh^a + Rh^b)/2,
//     A_s = -(Rh^a + Rh^b)/2,     E = (Rh^b - Rh^a)/2.
// A Robin-to-flux map with this beta satisfies -2D < R <= 0 (each leaf's map
// is B^T A^-1 B - W with W < 2D, and a merged map inherits the bound as the
// map of the union), so A_d is positive definite and A_s positive
// semidefinite: T is symmetric quasi-definite.  Its inverse is therefore
// computed by Gauss-Jordan elimination without pivoting, d block first
// (positive pivots, then the negative pivots of the Schur complement
// -(A_s + E A_d^-1 E)); no pivot search sits on the sequential chain.  The
// inverse is mapped back to W = M^-1 = D^-1/2 Q T^-1 Q^T D^-1/2 (Q the
// orthogonal sum / difference transform).
//
// The root of an all-Neumann problem has the constant null vector (s along
// D^1/2 1, d = 0).  Its s block is regularised by -v v^T, v = D^1/2 1 / |D^1/2 1|:
// for the consistent right-hand sides of such a problem the regularised
// inverse returns the solution with v^T s = 0, and the final zero-mean shift
// fixes the constant.
//
// Every solve pass then is a pair of matrix-vector products per node: M is
// symmetric, so blockdiag(R_og) xbar = -C^T M^-1 rbar_gamma = X^T rbar_gamma,
// giving the up-sweep rbar = rbar_o + X^T rbar_gamma, and the down-sweep
// lambda_gamma = X lambda_o + W (-rbar_gamma).  Iterative refinement
// (kernels_refine.cu) absorbs the rounding of an inverse-based solve.
//
// A root (no outer segments: no X, no merged map) may be kept as a block
// LDL^T factor of T instead (a third of the inversion's flops; by default
// for 2g >= 1024, mrcm_set_root_form); its solve passes then run block
// triangular sweeps (ldl_sweep_kernel and the factor-form branches of
// tree_up_kernel / tree_down_kernel).
//
// Storage: W column-major per node (entry (r, c) at c*2g + r); X column-major
// (2g x m).  Two launch shapes.  Levels with 2g <= 32: one group of 2g (padded
// to a power of two) lanes per node does the whole merge in registers
// (merge_small_kernel).  Larger systems: the form T is written into W, then a
// blocked Gauss-Jordan sweep (block kGJ) across many CTAs, the back
// transform, and X and R by output tiles.
#include "mrcm_internal.h"

#include <algorithm>

namespace mrcm {
namespace {

constexpr int kGJ = kMergeBlock; // block size of the blocked Gauss-Jordan sweep
constexpr int kGJTile = 32;       // output tile of the blocked update (kGJTile^2 per CTA)
constexpr int kSmallMax = 32;     // largest 2g merged by the per-node register kernel
constexpr int kNodeMax = 128;     // largest 2g inverted by the per-node kernel of the blocked path
constexpr int kRTile = 32;       // R update tile
constexpr double kTinyPivot = 1e-14;   // pivots of the scaled form are O(1)
constexpr double kRsqrt2 = 0.70710678118654752440;   // 1 / sqrt(2), the sum / difference transform

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

__device__ __forceinline__ double gamma_D(const DevView& v, const MergeDesc& D, int i) {
    return v.seg_D[v.gamma_segs[D.gamma_off + i]];
}

// Entry of T at (row r, column c), r, c in [0, 2g): d block first.  sd* =
// D^-1/2 and sq* = D^1/2 of the two gamma segments, inv_sum = 1 / sum D for
// the regularised all-Neumann root (0 otherwise).
__device__ __forceinline__ double t_entry(const NodeRefs& N, int r, int c, double sdi, double sdj, double sqi,
                                          double sqj, double inv_sum) {
    const int g = N.g;
    const bool dr = r < g, dc = c < g;
    const int i = dr ? r : r - g, j = dc ? c : c - g;
    // R is stored symmetric: read it along the column of j, so that
    // consecutive r (consecutive i) read consecutive entries
    const double ra = N.R1[N.gpos1[j] * N.m1 + N.gpos1[i]] * sdi * sdj;
    const double rb = N.R2[N.gpos2[j] * N.m2 + N.gpos2[i]] * sdi * sdj;
    if (dr && dc) return 0.5 * (ra + rb) + (i == j ? 2.0 : 0.0);
    if (!dr && !dc) return 0.5 * (ra + rb) - sqi * sqj * inv_sum;
    return 0.5 * (rb - ra);
}

// Expected pivot sign of step k: positive on the d block, negative on s.
__device__ __forceinline__ bool pivot_ok(double p, bool d_row) {
    return d_row ? (p > kTinyPivot) : (p < -kTinyPivot);
}
// The same test on the bit pattern (integer instructions only; an FP64
// compare takes a full FP64 instruction): sign as expected, magnitude above
// kTinyPivot and finite.
__device__ __forceinline__ bool pivot_ok_bits(double p, bool d_row) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(p);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const unsigned long long tiny = (unsigned long long)__double_as_longlong(kTinyPivot);
    return ((b >> 63) == (d_row ? 0ull : 1ull)) && mag > tiny && mag < 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool pivot_ok_bits(float p, bool d_row) {
    const unsigned int b = __float_as_uint(p);
    const unsigned int mag = b & 0x7fffffffu;
    const unsigned int tiny = __float_as_uint((float)kTinyPivot);
    return ((b >> 31) == (d_row ? 0u : 1u)) && mag > tiny && mag < 0x7f800000u;
}
// The interface matrix being inverted in place: the W storage itself in
// FP64, or the FP32 work array of the mixed form (same offsets).
template <class T> __device__ __forceinline__ T* gj_work(const DevView& v);
template <> __device__ __forceinline__ double* gj_work<double>(const DevView& v) { return v.W; }
template <> __device__ __forceinline__ float* gj_work<float>(const DevView& v) { return v.W32; }

// ---------------------------------------------------------------------------
// Per-node path for small systems (2g <= kSmallMax): one CTA per node, all in
// shared memory.  T (row-major), Gauss-Jordan without pivoting (one entry per
// thread and step, thread 0 forms the pivot reciprocal), the back transform
// into W (column-major), then X = -W B and R = R_oo + B^T X with B = C
// compacted to g x m (row k: gamma segment k of the child owning column j).
// Shared layout: T[g2*g2], Wc[g2*g2], Bs[g*mstride], Xs[g2*mstride].
constexpr int kSmallThreads = 256;      // CTA size for 2g up to kSmallMax (smaller systems: fewer)
// Body of the per-node merge; G2F > 0 fixes 2g at compile time (the sizes of
// a uniform tree's lower levels: its loops and the T index arithmetic then
// fold), 0 reads it from the descriptor.
// F: the arithmetic of the merge (double; float for the FP32 levels of the
// mixed form); the scalings, W, X and R are stored in double.
// NT: threads of the CTA (64 for 2g <= 8, 128 for 2g <= 16, else 256: the
// smallest systems keep every thread busy and more nodes resident per SM).
template <int G2F, class F, int NT>
__device__ __forceinline__ void merge_small_body(const DevView& v, const MergeDesc& D, const NodeRefs& N, int mstride,
                                                 F* sm, double* sd, double* sq, F* vrow,
                                                 double& s_inv_sum, int& s_bad) {
    constexpr int kG2Max = G2F ? G2F : (NT >= 256 ? kSmallMax : NT / 8);   // the launch's largest 2g
    constexpr int kSmallTri = (kG2Max * (kG2Max + 1) / 2 + NT - 1) / NT;     // kept T entries per thread
    const int g2 = G2F ? G2F : N.g2, g = g2 / 2, m = N.m, o1 = N.o1;
    const int tid = threadIdx.x;
    F* T = sm;
    F* Wc = T + g2 * g2;
    F* Bs = Wc + g2 * g2;
    F* Xs = Bs + g * mstride;
    if (tid < 32) {
        double dsum = 0.0;
        if (tid < g) {
            const double d = gamma_D(v, D, tid);
            sq[tid] = sqrt(d);
            sd[tid] = 1.0 / sq[tid];
            dsum = d;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        if (tid == 0) {
            s_inv_sum = (D.pinned && dsum > 0.0) ? 1.0 / dsum : 0.0;
            s_bad = 0;
        }
    }
    __syncthreads();
    for (int idx = tid; idx < g2 * g2; idx += NT) {
        const int r = idx / g2, c = idx % g2, i = r < g ? r : r - g, j = c < g ? c : c - g;
        T[idx] = (F)t_entry(N, r, c, sd[i], sd[j], sq[i], sq[j], s_inv_sum);
    }
    for (int k = 0; k < g; ++k) {
        const double* ra = N.R1 + N.gpos1[k] * N.m1;
        const double* rb = N.R2 + N.gpos2[k] * N.m2;
        for (int j = tid; j < m; j += NT)
            Bs[k * mstride + j] = (F)(j < o1 ? ra[N.opos1[j]] : rb[N.opos2[j - o1]]);
    }
    // Gauss-Jordan on T (d rows first: positive pivots, then negative).  T
    // is symmetric, and after step k the entries of an eliminated and a
    // remaining index are antisymmetric, all others symmetric; so only the
    // lower triangle r >= c is kept: a_rk = -T[k][r] for r < k, a_kc =
    // T[c][k] for c > k.  Per step warp 0 forms the reciprocal (rcp_nr) and
    // the scaled pivot row v_c = a_kc / p (v_k = 1 / p); every kept entry then
    // takes one FMA, the same for all of them (no divergent branches):
    //     T'_rc = x_r v_c + y_rc,  x_r = -a_rk (1 on the pivot row),
    //     y_rc = T_rc off the pivot row and column, 0 on them.
    int er[kSmallTri], ec[kSmallTri];
#pragma unroll
    for (int e = 0; e < kSmallTri; ++e) {
        const int idx = tid + e * NT;
        int r = (int)((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
        while ((r + 1) * (r + 2) / 2 <= idx) ++r;
        while (r * (r + 1) / 2 > idx) --r;
        er[e] = r;
        ec[e] = idx - r * (r + 1) / 2;
    }
    const int ntri = g2 * (g2 + 1) / 2;
    for (int k = 0; k < g2; ++k) {
        __syncthreads();
        if (tid < 32) {
            const F p = T[k * g2 + k];
            const F rp = rcp_nr(p);
            if (tid < g2) {
                const int c = tid;
                const F a_kc = c == k ? (F)1 : (c < k ? T[k * g2 + c] : T[c * g2 + k]);
                vrow[c] = a_kc * rp;
            }
            if (tid == 0 && !pivot_ok_bits(p, k < g)) s_bad = 1;
        }
        __syncthreads();
        F nv[kSmallTri];
#pragma unroll
        for (int e = 0; e < kSmallTri; ++e) {
            const int idx = tid + e * NT;
            if (idx >= ntri) break;
            const int r = er[e], c = ec[e];
            const F xr = r == k ? (F)1 : (r > k ? neg_bits(T[r * g2 + k]) : T[k * g2 + r]);
            const F y = (r == k || c == k) ? (F)0 : T[r * g2 + c];
            nv[e] = fma(xr, vrow[c], y);
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kSmallTri; ++e) {
            const int idx = tid + e * NT;
            if (idx >= ntri) break;
            T[er[e] * g2 + ec[e]] = nv[e];
        }
    }
    __syncthreads();
    if (tid == 0 && s_bad) atomicOr(v.status, kStatusSingular);
    // W = D^-1/2 Q T^-1 Q^T D^-1/2 (column-major Wc); T^-1 symmetric, kept
    // in the lower triangle
    for (int idx = tid; idx < g * g; idx += NT) {
        const int i = idx % g, j = idx / g;
        const F zdd = i >= j ? T[i * g2 + j] : T[j * g2 + i];
        const F zds = T[(g + j) * g2 + i];           // (d_i, s_j) = (s_j, d_i)
        const F zsd = T[(g + i) * g2 + j];
        const F zss = i >= j ? T[(g + i) * g2 + g + j] : T[(g + j) * g2 + g + i];
        const F sc = (F)(0.5 * sd[i] * sd[j]);
        Wc[j * g2 + i] = (zdd - zds - zsd + zss) * sc;
        Wc[(g + j) * g2 + i] = (zss + zsd - zds - zdd) * sc;
        Wc[j * g2 + g + i] = (zss + zds - zsd - zdd) * sc;
        Wc[(g + j) * g2 + g + i] = (zdd + zds + zsd + zss) * sc;
    }
    __syncthreads();
    double* Wg = v.W + D.W_off;
    for (int idx = tid; idx < g2 * g2; idx += NT) Wg[idx] = (double)Wc[idx];
    // X = -W B (columns of side a use W's a columns)
    double* Xg = v.X + D.X_off;
    for (int idx = tid; idx < g2 * m; idx += NT) {
        const int r = idx % g2, j = idx / g2;
        const F* wc = Wc + (j < o1 ? 0 : g) * g2 + r;
        F acc0 = 0, acc1 = 0;
        int k = 0;
        for (; k + 1 < g; k += 2) {
            acc0 = fma(wc[k * g2], Bs[k * mstride + j], acc0);
            acc1 = fma(wc[(k + 1) * g2], Bs[(k + 1) * mstride + j], acc1);
        }
        if (k < g) acc0 = fma(wc[k * g2], Bs[k * mstride + j], acc0);
        const F x = -(acc0 + acc1);
        Xg[idx] = (double)x;
        Xs[r * mstride + j] = x;
    }
    __syncthreads();
    // merged R = R_oo + B^T X (row i of side a uses the a rows of X); R is
    // symmetric (R_oo - B^T W B), so the lower triangle is formed and mirrored
    double* Rp = v.R + D.R_off;
    const int mtri = m * (m + 1) / 2;
    for (int idx = tid; idx < mtri; idx += NT) {
        int i = (int)((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
        while ((i + 1) * (i + 2) / 2 <= idx) ++i;
        while (i * (i + 1) / 2 > idx) --i;
        const int j = idx - i * (i + 1) / 2;
        const bool ia = i < o1;
        double roo = 0.0;       // loaded first, added last: its latency overlaps the sum
        if (ia && j < o1) roo = N.R1[N.opos1[i] * N.m1 + N.opos1[j]];
        if (!ia && j >= o1) roo = N.R2[N.opos2[i - o1] * N.m2 + N.opos2[j - o1]];
        const F* xh = Xs + (ia ? 0 : g) * mstride + j;
        F acc0 = 0, acc1 = 0;
        int k = 0;
        for (; k + 1 < g; k += 2) {
            acc0 = fma(Bs[k * mstride + i], xh[k * mstride], acc0);
            acc1 = fma(Bs[(k + 1) * mstride + i], xh[(k + 1) * mstride], acc1);
        }
        if (k < g) acc0 = fma(Bs[k * mstride + i], xh[k * mstride], acc0);
        const double val = roo + (double)(acc0 + acc1);
        Rp[(long long)i * m + j] = val;
        Rp[(long long)j * m + i] = val;
    }}

template <class F, int NT>
__global__ void __launch_bounds__(NT) merge_small_kernel(DevView v, int first, int mstride) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    F* sm = reinterpret_cast<F*>(sm_raw);
    __shared__ double sd[kSmallMax / 2], sq[kSmallMax / 2];
    __shared__ F vrow[kSmallMax];
    __shared__ double s_inv_sum;
    __shared__ int s_bad;
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    // uniform per CTA; a launch with NT threads holds systems up to 2g = NT / 8
    // (NT = 256: up to kSmallMax)
    if (N.g2 == 8) merge_small_body<8, F, NT>(v, D, N, mstride, sm, sd, sq, vrow, s_inv_sum, s_bad);
    else if (NT >= 128 && N.g2 == 16) merge_small_body<16, F, NT>(v, D, N, mstride, sm, sd, sq, vrow, s_inv_sum, s_bad);
    else if (NT >= 256 && N.g2 == 32) merge_small_body<32, F, NT>(v, D, N, mstride, sm, sd, sq, vrow, s_inv_sum, s_bad);
    else merge_small_body<0, F, NT>(v, D, N, mstride, sm, sd, sq, vrow, s_inv_sum, s_bad);
}

// ---------------------------------------------------------------------------
// Blocked path.  T into the W storage of each node (column-major).
__device__ __forceinline__ double block_sum256(double x, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    __syncthreads();
    return t;
}

// D^1/2 (scl[0, g)) and D^-1/2 (scl[g, 2g)) of a node's gamma segments in
// shared memory; returns sum D (256 threads).
__device__ double stage_gamma_scalings(const DevView& v, const MergeDesc& D, double* scl, double* red) {
    const int g = D.g;
    double part = 0.0;
    for (int i = threadIdx.x; i < g; i += 256) {
        const double d = gamma_D(v, D, i), sq = sqrt(d);
        scl[i] = sq;
        scl[g + i] = 1.0 / sq;
        part += d;
    }
    return block_sum256(part, red);
}


// Scratch of the blocked sweep, per node: two buffers for the inverse P of
// a diagonal block (kGJ x kGJ, row-major; block step k uses buffer k & 1),
// two buffers of the column vectors c_x = A(x, K) of the current block for
// every index x outside it (2g x kGJ, row x at x * kGJ), two buffers of
// u_x = P c_x^T (same layout), a flag word (the number of the last block
// whose P has been published) and a counter of the tile items that have
// written c of a next block.
// (In the mixed form's FP32 levels every value below is a float; the
// scratch buffer is the same, read through a float pointer.)
constexpr int kGJScratchHead = 2 * kGJ * kGJ;
__device__ __forceinline__ long long gj_scratch_stride(int nmax) {
    return kGJScratchHead + 4LL * nmax * kGJ + 2;
}
template <class T>
__device__ __forceinline__ T* gj_scratch(T* scratch, int slot, int nmax) {
    return scratch + (long long)slot * gj_scratch_stride(nmax);
}
template <class T>
__device__ __forceinline__ T* gj_P(T* sc, int step) { return sc + (step & 1) * kGJ * kGJ; }
template <class T>
__device__ __forceinline__ T* gj_cvec(T* sc, int step, int nmax) {
    return sc + kGJScratchHead + (long long)(step & 1) * nmax * kGJ;
}
template <class T>
__device__ __forceinline__ T* gj_uvec(T* sc, int step, int nmax) {
    return sc + kGJScratchHead + 2LL * nmax * kGJ + (long long)(step & 1) * nmax * kGJ;
}
template <class T>
__device__ __forceinline__ unsigned int* gj_flag(T* sc, int nmax) {
    return reinterpret_cast<unsigned int*>(sc + kGJScratchHead + 4LL * nmax * kGJ);
}
// number of tile items so far that wrote c of a next block (monotonic over
// the steps: each step has one per tile row of the node)
template <class T>
__device__ __forceinline__ unsigned int* gj_cready(T* sc, int nmax) { return gj_flag(sc, nmax) + 1; }

template <class T>
struct GJSmem {
    T Cr[kGJTile][kGJ + 1];    // c of the tile's rows
    T Ur[kGJTile][kGJ + 1];    // u of the tile's rows
    T Uc[kGJTile][kGJ + 1];    // u of the tile's columns
    T Ps[kGJ][kGJ + 1];        // a diagonal block being inverted, or a P
    T Pt[kGJ][kGJ + 1];        // second buffer of the inversion
    T rp[2];                   // pivot reciprocals (by step parity)
    T tt[2];                   // squared subdiagonal entry of the next pivot
};

// Inverse of a symmetric kGJ x kGJ block held in shared memory (lower
// triangle of Ps used; identity padding beyond nb), by the whole CTA (at
// least 224 threads): Gauss-Jordan without pivot search on the lower triangle
// (after a step, entries of an eliminated and a remaining index are
// antisymmetric, all others symmetric), ping-ponging between Ps and Pt.
//
// A warp-wide FP64 instruction holds its scheduler for about 64 cycles, so
// the pivots are a sequential chain of FP64 latencies.  Warp 0 runs that
// chain one step ahead of the rest: while warps 1-3, 5 and 6 apply step k - 1
// to the 136 entries (two FP64 instructions per entry, no divergent branches,
// sign flips on the bit pattern), warp 0 forms pivot k itself,
//     p_k = b_k - t_k r_(k-1),   b_k, t_k from the entries after step k - 2,
// where t_k, the square of entry (k, k - 1) after step k - 2 (both indices
// still remaining, so the row and column entries agree), is left in s_tt by
// the thread that produced it, and then its reciprocal r_k (rcp_nr) and the
// integer pivot test.  One CTA barrier per pivot hands r_k to the update and
// the fresh entries to warp 0.  On return Ps holds the full inverse.
// d_rows: rows of the block in the d part (positive pivots expected).
// Returns false (lane 0 of warp 0) on a pivot of the wrong sign or size.
template <class T>
__device__ bool gj_invert_block(T (*Ps)[kGJ + 1], T (*Pt)[kGJ + 1], T* s_rp, T* s_tt, int nb, int d_rows) {
    constexpr int kTri = kGJ * (kGJ + 1) / 2;
    static_assert(kTri <= 5 * 32 && (kGJ % 2) == 0, "five update warps; even number of steps");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rank = (warp >= 1 && warp <= 3) ? (warp - 1) * 32 + lane
                   : (warp == 5 || warp == 6) ? (warp - 2) * 32 + lane : kTri;
    int r = 0, c = 0;
    if (rank < kTri) {
        r = (int)((sqrtf(8.0f * rank + 1.0f) - 1.0f) * 0.5f);
        while ((r + 1) * (r + 2) / 2 <= rank) ++r;
        while (r * (r + 1) / 2 > rank) --r;
        c = rank - r * (r + 1) / 2;
    }
    T (*cur)[kGJ + 1] = Ps;      // entries after step kk - 2 (the input for kk <= 1)
    T (*nxt)[kGJ + 1] = Pt;
    T rp_prev = 0;
    bool ok = true;
    for (int kk = 0; kk <= kGJ; ++kk) {
        if (warp == 0) {
            if (kk < kGJ) {
                T p;
                if (kk == 0) {
                    p = cur[0][0];
                } else if (kk == 1) {
                    const T a = cur[1][0];
                    p = fma(-(a * a), rp_prev, cur[1][1]);
                } else {
                    p = fma(-s_tt[kk & 1], rp_prev, cur[kk][kk]);
                }
                const T rp = rcp_nr(p);
                if (lane == 0) {
                    s_rp[kk & 1] = rp;
                    if (kk < nb && !pivot_ok_bits(p, kk < d_rows)) ok = false;
                }
                rp_prev = rp;
            }
        } else if (rank < kTri && kk >= 1) {
            // step s = kk - 1: B'(r, c) = B(r, c) - B(r, s) B(s, c) r_s, with
            // the pivot row scaled by r_s, the pivot column by -r_s
            const int s = kk - 1;
            const T rp = s_rp[s & 1];
            const T xa = (r == s) ? (T)1 : (r > s ? neg_bits(cur[r][s]) : cur[s][r]);   // -B(r, s)
            const T xb = (c == s) ? (T)1 : (c < s ? cur[s][c] : cur[c][s]);             //  B(s, c)
            const T y = (r == s || c == s) ? (T)0 : cur[r][c];
            const T nv = fma(xa * xb, rp, y);
            nxt[r][c] = nv;
            if (r == kk + 1 && c == kk) s_tt[(kk + 1) & 1] = nv * nv;
        }
        __syncthreads();
        if (kk >= 1) {
            T (*t)[kGJ + 1] = cur;
            cur = nxt;
            nxt = t;
        }
    }
    // kGJ (even) swaps: the result is back in Ps; mirror the upper triangle
    {
        const int i = tid / kGJ, j = tid % kGJ;
        if (tid < kGJ * kGJ && i < j) Ps[i][j] = Ps[j][i];
    }
    __syncthreads();
    return ok;
}

// The sweep keeps only the lower triangle of the symmetric T: after step k
// an entry of an eliminated and a remaining index is antisymmetric, all
// others symmetric.  With K the current block, P = A_KK^-1, and for every
// index x outside K the column vector c_x = A(x, K) (read from the lower
// triangle: A(x, K) for x > K, -A(K, x) for x < K) and u_x = P c_x^T, one
// block step is
//     A_ij <- A_ij - s_j c_i . u_j   (i >= j outside K; s_j = -1 for j < K, +1 for j > K)
//     A(i, K) <- -u_i^T (i > K),  A(K, j) <- -u_j (j < K),  A_KK <- P.
// The tiles that hold the next block K1 as rows or as columns write the
// step's c for their indices and, once P of K1 is published, its u.

// c and u of block 0 for one (node, chunk of kGJTile indices x >= nb0).
template <class T>
__device__ void gj_first_cu_item(const DevView& v, const MergeDesc& D, int slot, int x0, T* scratch, int nmax,
                                 GJSmem<T>& S) {
    const int N = 2 * D.g;
    const int nb = min(kGJ, N);
    const T* A = gj_work<T>(v) + D.W_off;
    T* sc = gj_scratch(scratch, slot, nmax);
    const T* P0 = gj_P(sc, 0);
    T* cv = gj_cvec(sc, 0, nmax);
    T* uv = gj_uvec(sc, 0, nmax);
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kGJ * kGJ; idx += 256) S.Ps[idx / kGJ][idx % kGJ] = ldcg(P0 + idx);
    for (int idx = tid; idx < kGJTile * kGJ; idx += 256) {
        const int xl = idx % kGJTile, cc = idx / kGJTile, x = x0 + xl;
        const T c = (x < N && x >= nb && cc < nb) ? ldcg(A + (long long)cc * N + x) : (T)0;
        S.Cr[xl][cc] = c;
        if (x < N && x >= nb) cv[(long long)x * kGJ + cc] = c;
    }
    __syncthreads();
    for (int idx = tid; idx < kGJTile * kGJ; idx += 256) {
        const int xl = idx / kGJ, rr = idx % kGJ, x = x0 + xl;
        if (x >= N || x < nb) continue;
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int cc = 0; cc < kGJ; cc += 2) {
            a0 = fma(S.Ps[rr][cc], S.Cr[xl][cc], a0);
            a1 = fma(S.Ps[rr][cc + 1], S.Cr[xl][cc + 1], a1);
        }
        uv[(long long)x * kGJ + rr] = a0 + a1;
    }
    __syncthreads();
}

// Bounded wait of one CTA for a flag that another CTA of the same
// cooperative launch raises (at most `limit` polls, about a second by
// default: DevView::spin_limit); false on timeout (kStatusTimeout set).  Thread 0 polls with acquire loads, so what the
// raising CTA wrote before its release (fence + atomic) is visible to the
// whole CTA after the barrier that ends the wait.
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ bool wait_flag(const unsigned int* flag, unsigned int value, int* status, long long limit) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        long long spins = 0;
        while (ld_acquire_gpu(flag) < value) {
            if (++spins > limit) {
                ok = 0;
                atomicOr(status, kStatusTimeout);
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Block step k for one (node, lower output tile (ti >= tj)): the tile's part
// of the update above (entries r >= c; the block K1 x K1 is left to
// gj_next_diag_item), and c of step k + 1 for its indices when it holds K1
// as rows or columns (then the node's c counter is raised).
template <class T>
__device__ void gj_step_item(const DevView& v, const MergeDesc& D, int slot, int ti, int tj, int step,
                             T* scratch, int nmax, GJSmem<T>& S) {
    const int N = 2 * D.g;
    const int k0 = step * kGJ, nb = min(kGJ, N - k0);
    const int k1 = k0 + kGJ, nb1 = k1 < N ? min(kGJ, N - k1) : 0;
    const int r0 = ti * kGJTile, c0 = tj * kGJTile;
    T* A = gj_work<T>(v) + D.W_off;
    T* sc = gj_scratch(scratch, slot, nmax);
    const T* Pg = gj_P(sc, step);
    const T* cv = gj_cvec(sc, step, nmax);
    const T* uv = gj_uvec(sc, step, nmax);
    T* cn = gj_cvec(sc, step + 1, nmax);
    const int tid = threadIdx.x;
    const int tr = (tid % 16) * 2, tc = (tid / 16) * 2;
    // the tile's current entries, in flight while c and u are staged
    T old[2][2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int j = c0 + tc + b;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int i = r0 + tr + a;
            old[a][b] = (j < N && i < N && i >= j) ? ldcg(A + (long long)j * N + i) : (T)0;
        }
    }
    for (int idx = tid; idx < kGJTile * kGJ; idx += 256) {
        const int xl = idx / kGJ, cc = idx % kGJ;
        const int xi = r0 + xl, xj = c0 + xl;
        const bool okc = cc < nb;
        S.Cr[xl][cc] = (okc && xi < N && (xi < k0 || xi >= k0 + nb)) ? ldcg(cv + (long long)xi * kGJ + cc) : (T)0;
        S.Ur[xl][cc] = (okc && xi < N && (xi < k0 || xi >= k0 + nb)) ? ldcg(uv + (long long)xi * kGJ + cc) : (T)0;
        S.Uc[xl][cc] = (okc && xj < N && (xj < k0 || xj >= k0 + nb)) ? ldcg(uv + (long long)xj * kGJ + cc) : (T)0;
    }
    __syncthreads();
    T acc[2][2] = {{0, 0}, {0, 0}};
#pragma unroll
    for (int cc = 0; cc < kGJ; ++cc) {
        const T l0 = S.Cr[tr][cc], l1 = S.Cr[tr + 1][cc];
        const T u0 = S.Uc[tc][cc], u1 = S.Uc[tc + 1][cc];
        acc[0][0] = fma(l0, u0, acc[0][0]);
        acc[0][1] = fma(l0, u1, acc[0][1]);
        acc[1][0] = fma(l1, u0, acc[1][0]);
        acc[1][1] = fma(l1, u1, acc[1][1]);
    }
    const bool k1rows = nb1 > 0 && k1 >= r0 && k1 < r0 + kGJTile;
    const bool k1cols = nb1 > 0 && k1 >= c0 && k1 < c0 + kGJTile;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int j = c0 + tc + b;
        if (j >= N) continue;
        const bool jK = j >= k0 && j < k0 + nb;
        const bool jK1 = j >= k1 && j < k1 + nb1;
        T* col = A + (long long)j * N;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int i = r0 + tr + a;
            if (i >= N || i < j) continue;
            const bool iK = i >= k0 && i < k0 + nb;
            const bool iK1 = i >= k1 && i < k1 + nb1;
            T val;
            if (iK && jK) {
                val = ldcg(Pg + (i - k0) * kGJ + (j - k0));
            } else if (jK) {
                val = neg_bits(S.Ur[tr + a][j - k0]);     // block column, i > K
            } else if (iK) {
                val = neg_bits(S.Uc[tc + b][i - k0]);     // block row, j < K
            } else if (iK1 && jK1) {
                continue;                                 // the next diagonal block
            } else {
                // A_ij - s_j c_i . u_j with s_j = -1 below K
                val = j < k0 ? old[a][b] + acc[a][b] : old[a][b] - acc[a][b];
            }
            col[i] = val;
            if (jK1 && !iK1) cn[(long long)i * kGJ + (j - k1)] = val;                 // c_i = A(i, K1), i > K1
            if (iK1 && !jK1) cn[(long long)j * kGJ + (i - k1)] = neg_bits(val);       // c_j = -A(K1, j), j < K1
        }
    }
    if (k1rows || k1cols) {
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(gj_cready(sc, nmax), 1u);
    }
    __syncthreads();
}

// u of step k + 1 for one (node, run of indices [x0, x0 + len) outside K1):
// u_x = P_(k+1) c_x^T, once P_(k+1) is published and every tile row of the
// node has written its c (counter = (k + 1) tiles).  Sub-chunks of kUChunk
// indices, two threads per output entry, each summing half of the kGJ
// products.  Returns false when a wait timed out.
constexpr int kUChunk = 8;
template <class T>
__device__ bool gj_u_item(const DevView& v, const MergeDesc& D, int slot, int x0, int len, int step,
                          T* scratch, int nmax, GJSmem<T>& S) {
    const int N = 2 * D.g;
    const int k1 = (step + 1) * kGJ, nb1 = min(kGJ, N - k1);
    const int tiles = (N + kGJTile - 1) / kGJTile;
    T* sc = gj_scratch(scratch, slot, nmax);
    const T* Pn = gj_P(sc, step + 1);
    const T* cn = gj_cvec(sc, step + 1, nmax);
    T* un = gj_uvec(sc, step + 1, nmax);
    const int tid = threadIdx.x;
    static_assert(kUChunk * kGJ * 2 == 256 && kUChunk <= kGJTile, "two threads per output");
    const int o = tid >> 1, half = tid & 1;
    const int xl = o / kGJ, rr = o % kGJ;
    // the c are usually in before P: wait for them first and stage the
    // first run while P is awaited
    if (!wait_flag(gj_cready(sc, nmax), (unsigned int)((step + 1) * tiles), v.status, v.spin_limit)) return false;
    auto stage_c = [&](int xs) {
        for (int idx = tid; idx < kUChunk * kGJ; idx += 256) {
            const int yl = idx / kGJ, cc = idx % kGJ, y = xs + yl;
            const bool ok = y < N && (y < k1 || y >= k1 + nb1) && cc < nb1;
            S.Cr[yl][cc] = ok ? ldcg(cn + (long long)y * kGJ + cc) : (T)0;
        }
    };
    stage_c(x0);
    if (!wait_flag(gj_flag(sc, nmax), (unsigned int)(step + 1), v.status, v.spin_limit)) return false;
    for (int idx = tid; idx < kGJ * kGJ; idx += 256) S.Ps[idx / kGJ][idx % kGJ] = ldcg(Pn + idx);
    for (int xs = x0; xs < x0 + len; xs += kUChunk) {
        if (xs != x0) stage_c(xs);
        __syncthreads();
        const int x = xs + xl;
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int cc = half * (kGJ / 2); cc < (half + 1) * (kGJ / 2); cc += 2) {
            a0 = fma(S.Ps[rr][cc], S.Cr[xl][cc], a0);
            a1 = fma(S.Ps[rr][cc + 1], S.Cr[xl][cc + 1], a1);
        }
        T sum = a0 + a1;
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        if (half == 0 && x < N && (x < k1 || x >= k1 + nb1) && rr < nb1) un[(long long)x * kGJ + rr] = sum;
        __syncthreads();
    }
    return true;
}

// Block step k, for the next diagonal block K1 = [k1, k1 + nb1) of a node:
// its update A_ij - c_i . u_j (lower triangle; both indices above K), its
// inverse into the P buffer of step k + 1, then the node's flag is raised to
// k + 1.  Runs before any tile item of its CTA.  Returns false on a bad
// pivot.
template <class T>
__device__ bool gj_next_diag_item(const DevView& v, const MergeDesc& D, int slot, int step, T* scratch,
                                  int nmax, GJSmem<T>& S) {
    const int N = 2 * D.g;
    const int k0 = step * kGJ, nb = min(kGJ, N - k0);
    const int k1 = k0 + kGJ, nb1 = min(kGJ, N - k1);
    const T* A = gj_work<T>(v) + D.W_off;
    T* sc = gj_scratch(scratch, slot, nmax);
    const T* cv = gj_cvec(sc, step, nmax);
    const T* uv = gj_uvec(sc, step, nmax);
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kGJ * kGJ; idx += 256) {
        const int xl = idx / kGJ, cc = idx % kGJ;
        const bool ok = xl < nb1 && cc < nb;
        S.Cr[xl][cc] = ok ? ldcg(cv + (long long)(k1 + xl) * kGJ + cc) : (T)0;
        S.Uc[xl][cc] = ok ? ldcg(uv + (long long)(k1 + xl) * kGJ + cc) : (T)0;
    }
    __syncthreads();
    for (int idx = tid; idx < kGJ * kGJ; idx += 256) {
        const int pr = idx / kGJ, pc = idx % kGJ;
        T val = (pr == pc) ? (T)1 : (T)0;
        if (pr < nb1 && pc < nb1 && pr >= pc) {
            T a0 = 0, a1 = 0;
#pragma unroll
            for (int cc = 0; cc < kGJ; cc += 2) {
                a0 = fma(S.Cr[pr][cc], S.Uc[pc][cc], a0);
                a1 = fma(S.Cr[pr][cc + 1], S.Uc[pc][cc + 1], a1);
            }
            val = ldcg(A + (long long)(k1 + pc) * N + k1 + pr) - (a0 + a1);
        }
        if (pr >= pc) S.Ps[pr][pc] = val;
    }
    __syncthreads();
    const bool ok = gj_invert_block(S.Ps, S.Pt, S.rp, S.tt, nb1, D.g - k1);
    T* Pn = gj_P(sc, step + 1);
    for (int idx = tid; idx < kGJ * kGJ; idx += 256) Pn[idx] = S.Ps[idx / kGJ][idx % kGJ];
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicExch(gj_flag(sc, nmax), (unsigned int)(step + 1));
    return ok;
}

// Grid-wide barrier of a cooperative launch: a monotonic arrival counter
// (reset before the launch); round n ends when it reaches (n + 1) * grid.
// Data written by other CTAs before a barrier is read after it with L2-only
// loads (__ldcg).  Every wait is bounded (`limit` polls, about a second by
// default); a CTA that gives up sets kStatusTimeout and the caller returns.

__device__ bool grid_barrier(unsigned int* counter, unsigned int& round, int* status, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int target = (round + 1) * gridDim.x;
        __threadfence();
        atomicAdd(counter, 1u);
        long long spins = 0;
        while (ld_acquire_gpu(counter) < target) {
            if (++spins > limit) {
                ok = 0;
                atomicOr(status, kStatusTimeout);
                break;
            }
        }
        s_ok = ok;
    }
    ++round;
    __syncthreads();
    return s_ok != 0;
}

// Next item of a dynamically distributed loop: thread 0 takes a ticket from
// the launch's work counter (work; zeroed with the barrier counter before
// the launch) and the CTA reads it.  The tickets of one loop run from base;
// every CTA leaves the loop at its first ticket past the loop's items, so a
// loop of n items consumes n + gridDim.x tickets (the next loop's base).
__device__ __forceinline__ int grab_item(unsigned int* work, unsigned int base, int* s_item) {
    if (threadIdx.x == 0) *s_item = (int)(atomicAdd(work, 1u) - base);
    __syncthreads();
    const int item = *s_item;
    __syncthreads();
    return item;
}

// Lower tile of rank r among the tiles of one node at a block step: the
// tiles outside block row / column tk (the one holding K1), in row order,
// then the tk ones.
__device__ __forceinline__ void gj_lower_tile(int r, int tiles, int tk, int& ti, int& tj) {
    if (tk >= tiles) {
        ti = (int)((sqrtf(8.0f * r + 1.0f) - 1.0f) * 0.5f);
        while ((ti + 1) * (ti + 2) / 2 <= r) ++ti;
        while (ti * (ti + 1) / 2 > r) --ti;
        tj = r - ti * (ti + 1) / 2;
        return;
    }
    const int head = tiles * (tiles + 1) / 2 - tiles;
    if (r >= head) {
        const int q = r - head;                 // row tk (tj <= tk), then column tk (ti > tk)
        if (q <= tk) { ti = tk; tj = q; }
        else { ti = q; tj = tk; }
        return;
    }
    int cnt = 0;
    for (ti = 0; ti < tiles; ++ti) {
        if (ti == tk) continue;
        const int nrow = ti < tk ? ti + 1 : ti;  // tiles (ti, tj <= ti) with tj != tk
        if (r < cnt + nrow) {
            tj = r - cnt;
            if (ti > tk && tj >= tk) ++tj;
            return;
        }
        cnt += nrow;
    }
    tj = 0;
}

// T (the quasi-definite form) of one node for entries [e0, e1) of its
// column-major 2g x 2g storage, by one CTA (scalings staged in scl: 2g
// doubles).  A CTA may take several items in a row (levels with more nodes
// than CTAs): the closing barrier keeps the next item's staging off scl
// until every thread is done with it.
template <class T>
__device__ void form_item(const DevView& v, const MergeDesc& D, long long e0, long long e1, double* scl,
                          double* red) {
    const NodeRefs N = node_refs(v, D);
    const int g = N.g, g2 = N.g2;
    const double sum = stage_gamma_scalings(v, D, scl, red);
    const double inv_sum = (D.pinned && sum > 0.0) ? 1.0 / sum : 0.0;
    T* Tm = gj_work<T>(v) + D.W_off;
    for (long long idx = e0 + threadIdx.x; idx < e1; idx += 256) {
        int r, c;
        udivmod(idx, g2, c, r);
        const int i = r < g ? r : r - g, j = c < g ? c : c - g;
        Tm[idx] = (T)t_entry(N, r, c, scl[g + i], scl[g + j], scl[i], scl[j], inv_sum);
    }
    __syncthreads();     // the CTA's next item restages scl
}
// T^-1 -> W = D^-1/2 Q T^-1 Q^T D^-1/2 in place for the 2 x 2 block patterns
// (i, j), i, j < g, with pattern index in [e0, e1), by one CTA.
// (The mixed form's FP32 levels read T^-1 from the FP32 work array and write
// W in double; in FP64 the four entries are read and written in place.)
template <class T>
__device__ void backform_item(const DevView& v, const MergeDesc& D, long long e0, long long e1, double* scl,
                              double* red) {
    const int g = D.g, g2 = 2 * g;
    stage_gamma_scalings(v, D, scl, red);
    const double* sd = scl + g;
    const T* A = gj_work<T>(v) + D.W_off;
    double* Wd = v.W + D.W_off;
    for (long long idx = e0 + threadIdx.x; idx < e1; idx += 256) {
        int i, j;
        udivmod(idx, g, j, i);
        const long long odd = (long long)j * g2 + i;          // (d_i, d_j)
        const long long ods = (long long)(g + j) * g2 + i;    // (d_i, s_j)
        const long long osd = (long long)j * g2 + g + i;      // (s_i, d_j)
        const long long oss = (long long)(g + j) * g2 + g + i;
        const T zdd = ldcg(A + odd), zds = ldcg(A + ods), zsd = ldcg(A + osd), zss = ldcg(A + oss);
        const T sc = (T)(0.5 * sd[i] * sd[j]);
        Wd[odd] = (double)((zdd - zds - zsd + zss) * sc);   // W(a_i, a_j)
        Wd[ods] = (double)((zss + zsd - zds - zdd) * sc);   // W(a_i, b_j)
        Wd[osd] = (double)((zss + zds - zsd - zdd) * sc);   // W(b_i, a_j)
        Wd[oss] = (double)((zdd + zds + zsd + zss) * sc);   // W(b_i, b_j)
    }
    __syncthreads();     // the CTA's next item restages scl
}
// Items of an elementwise pass over every node of a level: each node's
// `per_node` entries split into runs of a multiple of 256, about one item
// per CTA over the level.
__device__ __forceinline__ long long level_run(long long per_node, int count) {
    const long long want = (gridDim.x + count - 1) / count;          // items per node
    long long run = (per_node + want - 1) / want;
    run = (run + 255) / 256 * 256;
    return run < 256 ? 256 : run;
}

// The whole blocked Gauss-Jordan sweep of one tree height in one cooperative
// launch, on the lower triangle: P_0 of every node; c and u of block 0; per
// block step one fused phase (the nodes' next diagonal blocks first, then
// their lower output tiles, the row / column tk ones leading, then the u
// of the next step in chunks over all CTAs) with a grid barrier after each;
// finally the lower triangle is mirrored so that W is stored in full.
// T: the arithmetic of the level (double; float for the FP32 levels of the
// mixed form, which sweep the FP32 work array and write W in double).
template <class T>
__global__ void __launch_bounds__(256, 4) gj_sweep_kernel(DevView v, int first, int count, int nmax, T* scratch,
                                                       unsigned int* counter) {
    __shared__ GJSmem<T> S;
    __shared__ int s_bad, s_item;
    __shared__ double red[8];
    extern __shared__ __align__(16) double scl[];           // 2g scalings (form / back-form)
    unsigned int* work = counter + 1;                       // ticket counter of the tile loops
    unsigned int wbase = 0;
    const int tiles = (nmax + kGJTile - 1) / kGJTile;
    const int nlower = tiles * (tiles + 1) / 2;
    const int nsteps = (nmax + kGJ - 1) / kGJ;
    const int tid = threadIdx.x;
    unsigned int round = 0;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // T of every node of the level into its W storage
    {
        const long long per = (long long)nmax * nmax, run = level_run(per, count);
        const long long runs = (per + run - 1) / run;
        for (long long item = blockIdx.x; item < count * runs; item += gridDim.x) {
            const int q = (int)(item / runs);
            const long long e0 = (item % runs) * run;
            const MergeDesc D = v.merges[first + q];
            const long long nT = 4LL * D.g * D.g;
            if (e0 >= nT) continue;                                  // uniform per CTA
            form_item<T>(v, D, e0, min(e0 + run, nT), scl, red);
        }
    }
    if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const MergeDesc D = v.merges[first + q];
        const int N = 2 * D.g, nb = min(kGJ, N);
        const T* A = gj_work<T>(v) + D.W_off;
        for (int idx = tid; idx < kGJ * kGJ; idx += 256) {
            const int pr = idx % kGJ, pc = idx / kGJ;
            S.Ps[pr][pc] = (pr < nb && pc < nb) ? ldcg(A + (long long)pc * N + pr) : (pr == pc ? (T)1 : (T)0);
        }
        __syncthreads();
        if (!gj_invert_block(S.Ps, S.Pt, S.rp, S.tt, nb, D.g)) s_bad = 1;
        T* sc = gj_scratch(scratch, q, nmax);
        T* P0 = gj_P(sc, 0);
        for (int idx = tid; idx < kGJ * kGJ; idx += 256) P0[idx] = S.Ps[idx / kGJ][idx % kGJ];
        if (tid == 0) {
            *gj_flag(sc, nmax) = 0u;
            *gj_cready(sc, nmax) = 0u;
        }
        __syncthreads();
    }
    if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    for (int item = blockIdx.x; item < count * tiles; item += gridDim.x) {
        const int q = item / tiles, x0 = (item % tiles) * kGJTile;
        const MergeDesc D = v.merges[first + q];
        if (x0 >= 2 * D.g) continue;                         // uniform per CTA
        gj_first_cu_item(v, D, q, x0, scratch, nmax, S);
    }
    if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    for (int step = 0; step < nsteps; ++step) {
        const int k0 = step * kGJ;
        const int tk = (k0 + kGJ) / kGJTile;                  // tile index of the next block
        // the diagonal items first, then the tiles; with several items per
        // CTA they are handed out as CTAs come free (a tile takes the same
        // time on any CTA, and a fixed share per CTA left some SMs a tile
        // behind the others at every step), with about one per CTA in a
        // fixed order (a ticket would only add its latency)
        const int nitems = count * (1 + nlower);
        const bool dyn = nitems >= 2 * (int)gridDim.x;
        for (int it0 = blockIdx.x;; it0 += gridDim.x) {
            const int item = dyn ? grab_item(work, wbase, &s_item) : it0;
            if (item >= nitems) break;
            if (item < count) {
                const MergeDesc D = v.merges[first + item];
                if (k0 + kGJ >= 2 * D.g) continue;
                if (!gj_next_diag_item(v, D, item, step, scratch, nmax, S)) s_bad = 1;
                continue;
            }
            // all nodes' tiles in row / column tk first (their c feeds the u
            // items), then the others
            const int it = item - count;
            const int tkc = tk < tiles ? tiles : 0;           // tiles per node in row / column tk
            const int head = nlower - tkc;
            int q, r;
            if (it < count * tkc) { q = it / tkc; r = head + it % tkc; }
            else { q = (it - count * tkc) / head; r = (it - count * tkc) % head; }
            int ti, tj;
            gj_lower_tile(r, tiles, tk, ti, tj);
            const MergeDesc D = v.merges[first + q];
            if (k0 >= 2 * D.g || ti * kGJTile >= 2 * D.g) continue;
            gj_step_item(v, D, q, ti, tj, step, scratch, nmax, S);
        }
        if (dyn) wbase += (unsigned int)nitems + gridDim.x;
        // u of step + 1 for every index outside the next block, spread over
        // all CTAs once their tiles are done
        // (runs sized so that one round of items covers the level)
        const int per = (count * nmax + (int)gridDim.x - 1) / (int)gridDim.x;
        const int ulen = max(kUChunk, (per + kUChunk - 1) / kUChunk * kUChunk);
        const int uchunks = (nmax + ulen - 1) / ulen;
        for (int item = blockIdx.x; item < count * uchunks; item += gridDim.x) {
            const int q = item / uchunks, x0 = (item % uchunks) * ulen;
            const MergeDesc D = v.merges[first + q];
            if (k0 + kGJ >= 2 * D.g || x0 >= 2 * D.g) continue;       // no next block, or past the end
            if (!gj_u_item(v, D, q, x0, min(ulen, 2 * D.g - x0), step, scratch, nmax, S)) return;
        }
        if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    }
    // mirror the lower triangle (strictly lower entries of the lower tiles)
    for (int item = blockIdx.x; item < count * nlower; item += gridDim.x) {
        const int q = item / nlower, r = item % nlower;
        int ti, tj;
        gj_lower_tile(r, tiles, tiles, ti, tj);
        const MergeDesc D = v.merges[first + q];
        const int N = 2 * D.g;
        if (ti * kGJTile >= N) continue;
        T* A = gj_work<T>(v) + D.W_off;
        for (int idx = tid; idx < kGJTile * kGJTile; idx += 256) {
            const int i = ti * kGJTile + idx % kGJTile, j = tj * kGJTile + idx / kGJTile;
            if (i < N && j < N && i > j) A[(long long)i * N + j] = ldcg(A + (long long)j * N + i);
        }
    }
    // T^-1 -> W of every node
    if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    {
        const long long per = (long long)(nmax / 2) * (nmax / 2), run = level_run(per, count);
        const long long runs = (per + run - 1) / run;
        for (long long item = blockIdx.x; item < count * runs; item += gridDim.x) {
            const int q = (int)(item / runs);
            const long long e0 = (item % runs) * run;
            const MergeDesc D = v.merges[first + q];
            const long long np = (long long)D.g * D.g;
            if (e0 >= np) continue;                                  // uniform per CTA
            backform_item<T>(v, D, e0, min(e0 + run, np), scl, red);
        }
    }
    __syncthreads();
    if (tid == 0 && s_bad) atomicOr(v.status, kStatusSingular);
}
// (row, column) of entry r of a row-packed lower triangle
__device__ __forceinline__ void tri_rc(int r, int& a, int& b) {
    a = (int)((sqrtf(8.0f * r + 1.0f) - 1.0f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= r) ++a;
    while (a * (a + 1) / 2 > r) --a;
    b = r - a * (a + 1) / 2;
}

// ---------------------------------------------------------------------------
// Per-node inversion for levels of many mid-sized systems (32 < 2g <= 128,
// at least half as many nodes as SMs): one CTA per node holds the lower triangle
// of T in shared memory (row-packed) and runs the Gauss-Jordan elimination
// of merge_small on it, a rank-one step per pivot (warp 0 forms the pivot's
// reciprocal, the pivot test and the scaled pivot row and column; every
// thread then updates its kept entries in place), then back-forms W into
// global memory.  No grid barriers, no global round trips of T: at these
// sizes the cooperative blocked sweep spends most of its time on its
// per-step synchronisation.  X and R follow with merge_x / merge_rupdate.
// NMAX: largest 2g of the instantiation; F: the arithmetic (double, or
// float for the mixed form's FP32 levels; W is stored in double).
template <int NMAX>
struct NodeTri {
    static constexpr int kTri = NMAX * (NMAX + 1) / 2;
    static constexpr int kPer = (kTri + 255) / 256;    // kept entries per thread
};
template <int NMAX, class F>
__global__ void __launch_bounds__(256) gj_node_kernel(DevView v, int first) {
    constexpr int kPer = NodeTri<NMAX>::kPer;
    extern __shared__ __align__(16) unsigned char nsm_raw[];
    F* T = reinterpret_cast<F*>(nsm_raw);                               // row-packed lower triangle
    __shared__ F xcol[NMAX], vrow[NMAX];
    __shared__ double scl[NMAX];                                        // D^1/2 (g), D^-1/2 (g)
    __shared__ double red[8];
    __shared__ int s_bad;
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs Nr = node_refs(v, D);
    const int g = D.g, n = 2 * g, ntri = n * (n + 1) / 2;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    const double sum = stage_gamma_scalings(v, D, scl, red);
    const double inv_sum = (D.pinned && sum > 0.0) ? 1.0 / sum : 0.0;
    // the thread's entries (r, c), r >= c, packed as r << 16 | c
    int rc[kPer];
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const int idx = tid + e * 256;
        int r = 0, c = 0;
        if (idx < ntri) tri_rc(idx, r, c);
        rc[e] = (r << 16) | c;
    }
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const int idx = tid + e * 256;
        if (idx >= ntri) break;
        const int r = rc[e] >> 16, c = rc[e] & 0xffff;
        const int i = r < g ? r : r - g, j = c < g ? c : c - g;
        T[idx] = (F)t_entry(Nr, r, c, scl[g + i], scl[g + j], scl[i], scl[j], inv_sum);
    }
    // Gauss-Jordan without pivoting (d rows first: positive pivots, then
    // negative); kept entries r >= c; after step k an entry of an eliminated
    // and a remaining index is antisymmetric: a_rk = -T(k, r) for r < k.
    for (int k = 0; k < n; ++k) {
        __syncthreads();
        if (tid < 32) {
            const F p = T[k * (k + 1) / 2 + k];
            const F rp = rcp_nr(p);
            for (int c = tid; c < n; c += 32) {
                // a_kc (row k) and -a_ck (column k) from the kept triangle
                const F akc = c == k ? (F)1 : (c < k ? T[k * (k + 1) / 2 + c] : T[c * (c + 1) / 2 + k]);
                vrow[c] = akc * rp;
                xcol[c] = c == k ? (F)1 : (c > k ? neg_bits(T[c * (c + 1) / 2 + k]) : T[k * (k + 1) / 2 + c]);
            }
            if (tid == 0 && !pivot_ok_bits(p, k < g)) s_bad = 1;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            const int idx = tid + e * 256;
            if (idx >= ntri) break;
            const int r = rc[e] >> 16, c = rc[e] & 0xffff;
            const F y = (r == k || c == k) ? (F)0 : T[idx];
            T[idx] = fma(xcol[r], vrow[c], y);
        }
    }
    __syncthreads();
    if (tid == 0 && s_bad) atomicOr(v.status, kStatusSingular);
    // W = D^-1/2 Q T^-1 Q^T D^-1/2, column-major, from the symmetric T^-1
    double* Wg = v.W + D.W_off;
    auto tinv = [&](int r, int c) -> F { return r >= c ? T[r * (r + 1) / 2 + c] : T[c * (c + 1) / 2 + r]; };
    for (int idx = tid; idx < g * g; idx += 256) {
        const int i = idx % g, j = idx / g;
        const F zdd = tinv(i, j), zds = tinv(i, g + j), zsd = tinv(g + i, j), zss = tinv(g + i, g + j);
        const F sc = (F)(0.5 * scl[g + i] * scl[g + j]);
        Wg[(long long)j * n + i] = (double)((zdd - zds - zsd + zss) * sc);
        Wg[(long long)(g + j) * n + i] = (double)((zss + zsd - zds - zdd) * sc);
        Wg[(long long)j * n + g + i] = (double)((zss + zds - zsd - zdd) * sc);
        Wg[(long long)(g + j) * n + g + i] = (double)((zdd + zds + zsd + zss) * sc);
    }
}

// ---------------------------------------------------------------------------
// Factor form of a root interface system (a level whose nodes have no outer
// segments: only lambda_gamma = -M^-1 rbar_gamma is ever needed, no X and no
// merged map).  The same blocked elimination as the sweep above, restricted
// to the trailing part: at block step k only entries with both indices past
// K are updated, which is a block LDL^T factorisation
//     T = Lt Dt Lt^T,  Lt unit block-lower (identity kGJ x kGJ diagonal
//     blocks),  Dt = blockdiag(A_KK) (the Schur complements met at the steps),
// with Lt(x, K) = u_x^T (u_x = A_KK^-1 c_x^T as above) and Dt_K^-1 = P_K.
// About N^3 / 3 flops instead of the N^3 of the inversion.  On exit the
// node's W storage holds, on and below the diagonal, Lt below the diagonal
// blocks and P_K = Dt_K^-1 in them (lower triangles; P_K is symmetric); a
// solve is then T^-1 b = Lt^-T P Lt^-1 b (two block triangular sweeps,
// tree_up / tree_down).  The quasi-definite T needs no pivot search here
// either: the diagonal blocks are inverted by gj_invert_block with its sign
// tests.

// Tile of rank r among the lower tiles (ti >= tj) of the trailing triangle
// of tiles [t0, tiles) at a block step: the tiles of column tk (the one that
// holds the next block K1, as columns) first, so that their c, which the u
// items wait for, come in early; then the others in row order.  tk - t0 is
// 0 or 1 (K, kGJ wide, starts in tile t0; K1 follows it); tkc = 0 when no
// node of the level has a next block (then plain row order).
__device__ __forceinline__ void ldl_trailing_tile(int r, int t0, int tiles, int tk, bool col_first, int& ti,
                                                  int& tj) {
    const int n = tiles - t0;
    int a, b;
    if (!col_first) {
        tri_rc(r, a, b);
        ti = t0 + a;
        tj = t0 + b;
        return;
    }
    const int kp = tk - t0;                       // 0 or 1
    if (r < n - kp) {                             // column tk, rows tk .. tiles-1
        ti = tk + r;
        tj = tk;
        return;
    }
    r -= n - kp;
    if (kp == 0) {                                // the rest: columns t0+1 .. (a triangle of n-1)
        tri_rc(r, a, b);
        ti = t0 + 1 + a;
        tj = t0 + 1 + b;
        return;
    }
    if (r < n) {                                  // column t0 (holds K), all its rows
        ti = t0 + r;
        tj = t0;
        return;
    }
    tri_rc(r - n, a, b);                          // columns t0+2 .. (a triangle of n-2)
    ti = t0 + 2 + a;
    tj = t0 + 2 + b;
}

// Tile items of the node whose c of the next block a u item waits for, summed
// over the block steps 0..step (each step: the tiles of column tk from row tk
// down, tiles_n - tk of them, tk = (step + 1) / 2 with kGJ = kGJTile / 2).
__device__ __forceinline__ unsigned int ldl_cready_target(int step, int tiles_n) {
    static_assert(2 * kGJ == kGJTile, "two blocks per tile");
    const unsigned int s1 = (unsigned int)step + 1u;
    return s1 * (unsigned int)tiles_n - (s1 * s1) / 4u;
}

// Block step k of the factorisation for one (node, lower output tile (ti >=
// tj) with columns reaching K): entries with both indices past K get
// A_ij - c_i . u_j (the next diagonal block K1 x K1 is left to
// gj_next_diag_item), the block column K below K gets Lt = u^T, the diagonal
// block K gets P_K; c of step k + 1 is written for the indices below K1.
template <class T>
__device__ void ldl_step_item(const DevView& v, const MergeDesc& D, int slot, int ti, int tj, int step,
                              T* scratch, int nmax, GJSmem<T>& S) {
    const int N = 2 * D.g;
    const int k0 = step * kGJ, nb = min(kGJ, N - k0);
    const int k1 = k0 + kGJ, nb1 = k1 < N ? min(kGJ, N - k1) : 0;
    const int r0 = ti * kGJTile, c0 = tj * kGJTile;
    T* A = gj_work<T>(v) + D.W_off;
    T* sc = gj_scratch(scratch, slot, nmax);
    const T* Pg = gj_P(sc, step);
    const T* cv = gj_cvec(sc, step, nmax);
    const T* uv = gj_uvec(sc, step, nmax);
    T* cn = gj_cvec(sc, step + 1, nmax);
    const int tid = threadIdx.x;
    const int tr = (tid % 16) * 2, tc = (tid / 16) * 2;
    const int kend = k0 + nb;                     // first index past K
    T old[2][2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int j = c0 + tc + b;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int i = r0 + tr + a;
            old[a][b] = (j < N && i < N && i >= j && j >= kend) ? ldcg(A + (long long)j * N + i) : (T)0;
        }
    }
    for (int idx = tid; idx < kGJTile * kGJ; idx += 256) {
        const int xl = idx / kGJ, cc = idx % kGJ;
        const int xi = r0 + xl, xj = c0 + xl;
        const bool okc = cc < nb;
        S.Cr[xl][cc] = (okc && xi < N && xi >= kend) ? ldcg(cv + (long long)xi * kGJ + cc) : (T)0;
        S.Ur[xl][cc] = (okc && xi < N && xi >= kend) ? ldcg(uv + (long long)xi * kGJ + cc) : (T)0;
        S.Uc[xl][cc] = (okc && xj < N && xj >= kend) ? ldcg(uv + (long long)xj * kGJ + cc) : (T)0;
    }
    __syncthreads();
    T acc[2][2] = {{0, 0}, {0, 0}};
#pragma unroll
    for (int cc = 0; cc < kGJ; ++cc) {
        const T l0 = S.Cr[tr][cc], l1 = S.Cr[tr + 1][cc];
        const T u0 = S.Uc[tc][cc], u1 = S.Uc[tc + 1][cc];
        acc[0][0] = fma(l0, u0, acc[0][0]);
        acc[0][1] = fma(l0, u1, acc[0][1]);
        acc[1][0] = fma(l1, u0, acc[1][0]);
        acc[1][1] = fma(l1, u1, acc[1][1]);
    }
    const bool k1cols = nb1 > 0 && k1 >= c0 && k1 < c0 + kGJTile;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int j = c0 + tc + b;
        if (j >= N || j < k0) continue;           // eliminated columns hold Lt already
        const bool jK = j < kend;
        const bool jK1 = j >= k1 && j < k1 + nb1;
        T* col = A + (long long)j * N;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int i = r0 + tr + a;
            if (i >= N || i < j) continue;
            const bool iK = i < kend;
            const bool iK1 = i >= k1 && i < k1 + nb1;
            T val;
            if (iK && jK) {
                val = ldcg(Pg + (i - k0) * kGJ + (j - k0));     // P_K = Dt_K^-1
            } else if (jK) {
                val = S.Ur[tr + a][j - k0];                     // Lt(i, K) = u_i^T
            } else if (iK1 && jK1) {
                continue;                                       // the next diagonal block
            } else {
                val = old[a][b] - acc[a][b];
            }
            col[i] = val;
            if (jK1 && !iK1) cn[(long long)i * kGJ + (j - k1)] = val;   // c_i = A(i, K1), i past K1
        }
    }
    if (k1cols) {
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(gj_cready(sc, nmax), 1u);
    }
    __syncthreads();
}

// u of step k + 1 for one (node, run of indices [x0, x0 + len) past K1):
// u_x = P_(k+1) c_x^T once P_(k+1) is published and every tile of column tk
// has written its c.  Returns false when a wait timed out.
template <class T>
__device__ bool ldl_u_item(const DevView& v, const MergeDesc& D, int slot, int x0, int len, int step,
                           T* scratch, int nmax, GJSmem<T>& S) {
    const int N = 2 * D.g;
    const int k1 = (step + 1) * kGJ, nb1 = min(kGJ, N - k1);
    const int tiles_n = (N + kGJTile - 1) / kGJTile;
    T* sc = gj_scratch(scratch, slot, nmax);
    const T* Pn = gj_P(sc, step + 1);
    const T* cn = gj_cvec(sc, step + 1, nmax);
    T* un = gj_uvec(sc, step + 1, nmax);
    const int tid = threadIdx.x;
    const int o = tid >> 1, half = tid & 1;
    const int xl = o / kGJ, rr = o % kGJ;
    if (!wait_flag(gj_cready(sc, nmax), ldl_cready_target(step, tiles_n), v.status, v.spin_limit)) return false;
    auto stage_c = [&](int xs) {
        for (int idx = tid; idx < kUChunk * kGJ; idx += 256) {
            const int yl = idx / kGJ, cc = idx % kGJ, y = xs + yl;
            const bool ok = y < N && y >= k1 + nb1 && cc < nb1;
            S.Cr[yl][cc] = ok ? ldcg(cn + (long long)y * kGJ + cc) : (T)0;
        }
    };
    stage_c(x0);
    if (!wait_flag(gj_flag(sc, nmax), (unsigned int)(step + 1), v.status, v.spin_limit)) return false;
    for (int idx = tid; idx < kGJ * kGJ; idx += 256) S.Ps[idx / kGJ][idx % kGJ] = ldcg(Pn + idx);
    for (int xs = x0; xs < x0 + len; xs += kUChunk) {
        if (xs != x0) stage_c(xs);
        __syncthreads();
        const int x = xs + xl;
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int cc = half * (kGJ / 2); cc < (half + 1) * (kGJ / 2); cc += 2) {
            a0 = fma(S.Ps[rr][cc], S.Cr[xl][cc], a0);
            a1 = fma(S.Ps[rr][cc + 1], S.Cr[xl][cc + 1], a1);
        }
        T sum = a0 + a1;
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        if (half == 0 && x < N && x >= k1 + nb1 && rr < nb1) un[(long long)x * kGJ + rr] = sum;
        __syncthreads();
    }
    return true;
}

// The factorisation of one root level in one cooperative launch: T of every
// node, P_0, c and u of block 0, then per block step the next diagonal
// blocks, the trailing tiles (column tk first) and the u of the next step
// past K1, with a grid barrier after each step.  T: the arithmetic of the
// level (double; float for an FP32 level of the mixed form, which factors in
// the FP32 work array and stores Lt and P in double at the end).
template <class T>
__global__ void __launch_bounds__(256, 4) ldl_sweep_kernel(DevView v, int first, int count, int nmax, T* scratch,
                                                        unsigned int* counter) {
    __shared__ GJSmem<T> S;
    __shared__ int s_bad, s_item;
    __shared__ double red[8];
    extern __shared__ __align__(16) double scl[];           // 2g scalings (form)
    unsigned int* work = counter + 1;                       // ticket counter of the tile loops
    unsigned int wbase = 0;
    const int tiles = (nmax + kGJTile - 1) / kGJTile;
    const int nsteps = (nmax + kGJ - 1) / kGJ;
    const int tid = threadIdx.x;
    unsigned int round = 0;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    {
        const long long per = (long long)nmax * nmax, run = level_run(per, count);
        const long long runs = (per + run - 1) / run;
        for (long long item = blockIdx.x; item < count * runs; item += gridDim.x) {
            const int q = (int)(item / runs);
            const long long e0 = (item % runs) * run;
            const MergeDesc D = v.merges[first + q];
            const long long nT = 4LL * D.g * D.g;
            if (e0 >= nT) continue;                                  // uniform per CTA
            form_item<T>(v, D, e0, min(e0 + run, nT), scl, red);
        }
    }
    if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const MergeDesc D = v.merges[first + q];
        const int N = 2 * D.g, nb = min(kGJ, N);
        const T* A = gj_work<T>(v) + D.W_off;
        for (int idx = tid; idx < kGJ * kGJ; idx += 256) {
            const int pr = idx % kGJ, pc = idx / kGJ;
            S.Ps[pr][pc] = (pr < nb && pc < nb) ? ldcg(A + (long long)pc * N + pr) : (pr == pc ? (T)1 : (T)0);
        }
        __syncthreads();
        if (!gj_invert_block(S.Ps, S.Pt, S.rp, S.tt, nb, D.g)) s_bad = 1;
        T* sc = gj_scratch(scratch, q, nmax);
        T* P0 = gj_P(sc, 0);
        for (int idx = tid; idx < kGJ * kGJ; idx += 256) P0[idx] = S.Ps[idx / kGJ][idx % kGJ];
        if (tid == 0) {
            *gj_flag(sc, nmax) = 0u;
            *gj_cready(sc, nmax) = 0u;
        }
        __syncthreads();
    }
    if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    for (int item = blockIdx.x; item < count * tiles; item += gridDim.x) {
        const int q = item / tiles, x0 = (item % tiles) * kGJTile;
        const MergeDesc D = v.merges[first + q];
        if (x0 >= 2 * D.g) continue;                         // uniform per CTA
        gj_first_cu_item(v, D, q, x0, scratch, nmax, S);
    }
    if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    for (int step = 0; step < nsteps; ++step) {
        const int k0 = step * kGJ;
        const int t0 = k0 / kGJTile;                          // tile column holding K
        const int tk = (k0 + kGJ) / kGJTile;                  // tile column holding K1
        const bool col_first = k0 + kGJ < nmax;
        const int n = tiles - t0;
        const int ntri = n * (n + 1) / 2;
        const int tkc = col_first ? tiles - tk : 0;           // column-tk tiles per node
        const int nitems = count * (1 + ntri);
        // handed out as CTAs come free at every step: the trailing triangle
        // shrinks, and its last steps gain most from the balance
        const bool dyn = true;
        for (int it0 = blockIdx.x;; it0 += gridDim.x) {
            const int item = dyn ? grab_item(work, wbase, &s_item) : it0;
            if (item >= nitems) break;
            if (item < count) {
                const MergeDesc D = v.merges[first + item];
                if (k0 + kGJ >= 2 * D.g) continue;
                if (!gj_next_diag_item(v, D, item, step, scratch, nmax, S)) s_bad = 1;
                continue;
            }
            const int it = item - count;
            int q, r;
            if (it < count * tkc) { q = it / tkc; r = it % tkc; }
            else { q = (it - count * tkc) / (ntri - tkc); r = tkc + (it - count * tkc) % (ntri - tkc); }
            int ti, tj;
            ldl_trailing_tile(r, t0, tiles, tk, col_first, ti, tj);
            const MergeDesc D = v.merges[first + q];
            if (k0 >= 2 * D.g || ti * kGJTile >= 2 * D.g) continue;
            ldl_step_item(v, D, q, ti, tj, step, scratch, nmax, S);
        }
        if (dyn) wbase += (unsigned int)nitems + gridDim.x;
        // u of step + 1 past the next block, spread over all CTAs
        const int xs0 = k0 + 2 * kGJ;                         // first index past K1
        if (xs0 < nmax) {
            const int span = nmax - xs0;
            const int per = (count * span + (int)gridDim.x - 1) / (int)gridDim.x;
            const int ulen = max(kUChunk, (per + kUChunk - 1) / kUChunk * kUChunk);
            const int uchunks = (span + ulen - 1) / ulen;
            for (int item = blockIdx.x; item < count * uchunks; item += gridDim.x) {
                const int q = item / uchunks, x0 = xs0 + (item % uchunks) * ulen;
                const MergeDesc D = v.merges[first + q];
                if (xs0 >= 2 * D.g || x0 >= 2 * D.g) continue;       // nothing past K1 in this node
                if (!ldl_u_item(v, D, q, x0, min(ulen, 2 * D.g - x0), step, scratch, nmax, S)) return;
            }
        }
        if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
    }
    // an FP32 level: Lt and P (on and below the diagonal) into the double storage
    if (sizeof(T) != sizeof(double)) {
        for (long long item = blockIdx.x; item < (long long)count * tiles * tiles; item += gridDim.x) {
            const int q = (int)(item / ((long long)tiles * tiles));
            const int rem = (int)(item % ((long long)tiles * tiles));
            const int ti = rem % tiles, tj = rem / tiles;
            const MergeDesc D = v.merges[first + q];
            const int N = 2 * D.g;
            if (ti < tj || ti * kGJTile >= N) continue;
            const T* A = gj_work<T>(v) + D.W_off;
            double* Wd = v.W + D.W_off;
            for (int idx = tid; idx < kGJTile * kGJTile; idx += 256) {
                const int i = ti * kGJTile + idx % kGJTile, j = tj * kGJTile + idx / kGJTile;
                if (i < N && j < N && i >= j) Wd[(long long)j * N + i] = (double)ldcg(A + (long long)j * N + i);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && s_bad) atomicOr(v.status, kStatusSingular);
}


// X = -W C with C = blockdiag(R^a_go, R^b_go): column j < o1 uses the first
// g columns of W, the others the last g.  A CTA computes 64 rows x 16
// columns; the gathered entries of C are staged in shared memory in chunks.
constexpr int kXColsOut = 16, kXChunk = 64;
// XROWS rows x kXColsOut columns of X per CTA: 32 unless the level has
// CTAs in great excess (then 64, fewer staged loads per product); with few
// long rows per node the smaller CTAs keep more SMs busy.
// F: the arithmetic (double; float for the FP32 levels of the mixed form,
// which read W and the children's maps in double and write X in double).
template <int XROWS, class F>
__global__ void __launch_bounds__(256) merge_x_kernel(DevView v, int first) {
    constexpr int kXRows = XROWS, kQ = kXRows * kXColsOut / 256;   // outputs per thread
    __shared__ F Cs[kXChunk][kXColsOut];
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int g = N.g, g2 = N.g2, m = N.m;
    const int rt = (g2 + kXRows - 1) / kXRows;
    const int r0 = (blockIdx.y % rt) * kXRows, j0 = (blockIdx.y / rt) * kXColsOut;
    if (j0 >= m) return;                              // uniform per CTA
    const double* W = v.W + D.W_off;
    double* X = v.X + D.X_off;
    const int tid = threadIdx.x, rl = tid % kXRows, cg = tid / kXRows;   // column groups of kQ
    const int r = r0 + rl;
    F acc[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) acc[q] = 0;
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
                Cs[kk][jj] = (F)c;
            }
            __syncthreads();
            if (r < g2) {
                const double* wcol = W + (long long)(half * g + k0) * g2 + r;
                for (int kk = 0; kk < kn; ++kk) {
                    const F wv = (F)wcol[(long long)kk * g2];
#pragma unroll
                    for (int q = 0; q < kQ; ++q) acc[q] += wv * Cs[kk][cg * kQ + q];
                }
            }
        }
    }
    if (r < g2) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int j = j0 + cg * kQ + q;
            if (j < m) X[(long long)j * g2 + r] = (double)(-acc[q]);
        }
    }
}

// R = blockdiag(R_oo) + blockdiag(R_og) X on (16 TS)^2 output tiles (the
// lower triangle, mirrored: R is symmetric): row i
// of the tile uses the gathered row of R^a (i < o1) or R^b and the matching
// half of X; both are staged in shared memory in chunks of kRTile.
// staged in shared memory in chunks of kRTile.  TS = 1 (16 x 16 tiles, one
// entry per thread) unless the level has tiles in great excess (then TS = 2,
// 32 x 32 tiles, 2 x 2 per thread): with few nodes per height the small
// tiles keep more SMs busy behind the long k loops.
template <int TS, class F>
__global__ void __launch_bounds__(256) merge_rupdate_kernel(DevView v, int first) {
    constexpr int kTile = 16 * TS;
    __shared__ F Cs[kTile][kRTile + 1];         // Cs[row][k]
    __shared__ F Xs[2][kRTile][kTile + 1];      // Xs[half][k][col]
    const MergeDesc D = v.merges[first + blockIdx.x];
    const NodeRefs N = node_refs(v, D);
    const int m = N.m, g = N.g, g2 = N.g2, o1 = N.o1;
    const int tiles = (m + kTile - 1) / kTile;
    if ((int)blockIdx.y >= tiles * (tiles + 1) / 2) return;
    // R is symmetric: lower-triangle tiles (ti >= tj) only, mirrored on write
    int ti = (int)((sqrtf(8.0f * blockIdx.y + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.y) ++ti;
    while (ti * (ti + 1) / 2 > (int)blockIdx.y) --ti;
    const int tj = blockIdx.y - ti * (ti + 1) / 2;
    const int i0 = ti * kTile, jt = tj * kTile;
    const double* X = v.X + D.X_off;
    double* Rp = v.R + D.R_off;
    const int tid = threadIdx.x;
    const int tr = (tid % 16) * TS, tc = (tid / 16) * TS;
    F acc[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) acc[a][b] = 0;
    for (int k0 = 0; k0 < g; k0 += kRTile) {
        const int kn = min(kRTile, g - k0);
        __syncthreads();
        for (int idx = tid; idx < kTile * kRTile; idx += 256) {
            const int rr = idx / kRTile, kk = idx % kRTile, i = i0 + rr;
            double c = 0.0;
            if (kk < kn && i < m)
                c = i < o1 ? N.R1[N.opos1[i] * N.m1 + N.gpos1[k0 + kk]]
                           : N.R2[N.opos2[i - o1] * N.m2 + N.gpos2[k0 + kk]];
            Cs[rr][kk] = (F)c;
        }
        for (int idx = tid; idx < 2 * kRTile * kTile; idx += 256) {
            const int half = idx / (kRTile * kTile), rem = idx % (kRTile * kTile);
            const int kk = rem % kRTile, jj = rem / kRTile, j = jt + jj;
            Xs[half][kk][jj] = (kk < kn && j < m) ? (F)X[(long long)j * g2 + half * g + k0 + kk] : (F)0;
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < TS; ++a) {
            const int half = (i0 + tr + a) < o1 ? 0 : 1;
            for (int kk = 0; kk < kRTile; ++kk) {
                const F cv = Cs[tr + a][kk];
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
            if (j >= m || j > i) continue;
            double val = (double)acc[a][b];
            if (i < o1 && j < o1) val += row[N.opos1[j]];
            if (i >= o1 && j >= o1) val += row[N.opos2[j - o1]];
            Rp[(long long)i * m + j] = val;
            Rp[(long long)j * m + i] = val;
        }
    }
}

// ---------------------------------------------------------------------------
// Block triangular sweeps with the factor Lt of a root level, in blocks of
// kSolveBlock unknowns (kSolveBlock / kGJ factor blocks), left-looking: the
// item of block K (one CTA) forms its right-hand side, subtracts the
// products with the blocks it depends on as each of them is published
// (a flag per block, bounded waits), solves its diagonal part of Lt
// (identity kGJ blocks, full kGJ x kGJ blocks below them: kSolveBlock / kGJ
// dependent sub-steps) and publishes its own unknowns.  Items run in the
// order of the dependencies (forward: K ascending; backward: K descending)
// over the CTAs of a cooperative launch, so an item only waits for items
// that come earlier in that order, and the chain is one block's products
// and its small solve per block instead of a grid barrier.
constexpr int kSolveBlock = kTriBlock;
constexpr int kSolveSub = kSolveBlock / kGJ;
constexpr int kSolvePairs = kSolveSub * (kSolveSub - 1) / 2;
static_assert(kSolveSub == 4, "four factor blocks per solve block");

struct TriSmem {
    double Ls[kSolvePairs][kGJ][kGJ + 1];   // the blocks (b, a), b > a, of the diagonal part
    double rhs[kSolveBlock];
    double sol[kSolveBlock];
    double dep[kSolveBlock];                // unknowns of the block being subtracted
    double part[4][kSolveBlock];
};
// pair index of the sub-block (b, a), b > a
__device__ __forceinline__ int tri_pair(int b, int a) { return b * (b - 1) / 2 + a; }

// Stages the diagonal part of Lt for the block [s0, s0 + kSolveBlock) of a
// node (rows past N read as 0).
__device__ __forceinline__ void tri_stage_diag(const double* Wn, int N, int s0, TriSmem& S) {
    for (int idx = threadIdx.x; idx < kSolvePairs * kGJ * kGJ; idx += 256) {
        const int pr = idx / (kGJ * kGJ), e = idx % (kGJ * kGJ), rr = e % kGJ, cc = e / kGJ;
        int b = 1;
        while (tri_pair(b + 1, 0) <= pr) ++b;
        const int a = pr - tri_pair(b, 0);
        const int row = s0 + b * kGJ + rr, col = s0 + a * kGJ + cc;
        S.Ls[pr][rr][cc] = row < N ? __ldcg(Wn + (long long)col * N + row) : 0.0;
    }
}

// Publishes a block's unknowns: the stores, a fence, then the flag.
__device__ __forceinline__ void tri_publish(unsigned int* flag) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(flag, 1u);
}

// Forward item: y_K = Lt_KK^-1 (rhat_K - sum_{J<K} Lt_KJ y_J) for block K of
// one node of a root level; rhat = Q^T S rbar_gamma is formed here from the
// children's particular fluxes; y goes to out (v.fwd).  Returns false when
// a wait timed out.
__device__ bool tri_forward_item(const DevView& v, const MergeDesc& D, int K, unsigned int* flags,
                                 TriSmem& S) {
    const int tid = threadIdx.x, N = 2 * D.g, g = D.g, s0 = K * kSolveBlock;
    const int nbk = min(kSolveBlock, N - s0);
    const double* Wn = v.W + D.W_off;
    double* out = v.fwd + 2LL * D.gamma_off;
    if (tid < kSolveBlock) {
        double r = 0.0;
        if (tid < nbk) {
            const int x = s0 + tid, i = x < g ? x : x - g;
            const NodeRefs Nr = node_refs(v, D);
            const double ra = __ldcg(v.rbar + D.r1_off + Nr.gpos1[i]);
            const double rb = __ldcg(v.rbar + D.r2_off + Nr.gpos2[i]);
            const double sc = kRsqrt2 / sqrt(gamma_D(v, D, i));
            r = x < g ? sc * (rb - ra) : sc * (ra + rb);
        }
        S.rhs[tid] = r;
    }
    tri_stage_diag(Wn, N, s0, S);
    const int rr = tid % kSolveBlock, grp = tid / kSolveBlock;
    for (int J = 0; J < K; ++J) {
        // this thread's entries of Lt_KJ are loaded before the wait (they do
        // not depend on it), so the chain holds only the products
        double lt[kGJ];
        const double* col = Wn + (long long)(J * kSolveBlock + grp * kGJ) * N + s0 + rr;
#pragma unroll
        for (int jj = 0; jj < kGJ; ++jj) lt[jj] = rr < nbk ? __ldcg(col + (long long)jj * N) : 0.0;
        if (!wait_flag(flags + J, 1u, v.status, v.spin_limit)) return false;
        if (tid < kSolveBlock) S.dep[tid] = __ldcg(out + J * kSolveBlock + tid);
        __syncthreads();
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
        for (int jj = 0; jj < kGJ; jj += 4) {
            a0 = fma(lt[jj], S.dep[grp * kGJ + jj], a0);
            a1 = fma(lt[jj + 1], S.dep[grp * kGJ + jj + 1], a1);
            a2 = fma(lt[jj + 2], S.dep[grp * kGJ + jj + 2], a2);
            a3 = fma(lt[jj + 3], S.dep[grp * kGJ + jj + 3], a3);
        }
        S.part[grp][rr] = (a0 + a1) + (a2 + a3);
        __syncthreads();
        if (tid < kSolveBlock) S.rhs[tid] -= (S.part[0][tid] + S.part[1][tid]) + (S.part[2][tid] + S.part[3][tid]);
    }
    __syncthreads();
    if (tid < kGJ) S.sol[tid] = S.rhs[tid];
    __syncthreads();
    const int sr = tid / kGJ, p = tid % kGJ;
    for (int b = 1; b < kSolveSub; ++b) {
        double acc = 0.0;
        for (int a = 0; a < b; ++a) acc = fma(S.Ls[tri_pair(b, a)][sr][p], S.sol[a * kGJ + p], acc);
#pragma unroll
        for (int w = kGJ / 2; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w, kGJ);
        if (p == 0) S.sol[b * kGJ + sr] = S.rhs[b * kGJ + sr] - acc;
        __syncthreads();
    }
    if (tid < nbk) out[s0 + tid] = S.sol[tid];
    tri_publish(flags + K);
    __syncthreads();
    return true;
}

// Backward item: x_K = Lt_KK^-T (z_K - sum_{J>K} Lt_JK^T x_J) with z = P y
// (the inverse diagonal blocks of the factor on the forward result, formed
// here); x goes to out (rgam).  Returns false when a wait timed out.
__device__ bool tri_backward_item(const DevView& v, const MergeDesc& D, int K, unsigned int* flags,
                                  TriSmem& S) {
    const int tid = threadIdx.x, N = 2 * D.g, s0 = K * kSolveBlock;
    const int nbk = min(kSolveBlock, N - s0), nblk = (N + kSolveBlock - 1) / kSolveBlock;
    const double* Wn = v.W + D.W_off;
    const double* y = v.fwd + 2LL * D.gamma_off;
    double* out = v.rgam + 2LL * D.gamma_off;
    if (tid < kSolveBlock) {
        double z = 0.0;
        if (tid < nbk) {
            const int r = s0 + tid, k0 = r - r % kGJ, nb = min(kGJ, N - k0);
            for (int cc = 0; cc < nb; ++cc) {
                const int col = k0 + cc;
                const double pv = r >= col ? Wn[(long long)col * N + r] : Wn[(long long)r * N + col];
                z = fma(pv, __ldcg(y + col), z);
            }
        }
        S.rhs[tid] = z;
    }
    tri_stage_diag(Wn, N, s0, S);
    // kGJ lanes over the rows of block J, one column of block K per lane group
    const int lane = tid % kGJ, cg = tid / kGJ;           // 16 column groups
    for (int J = nblk - 1; J > K; --J) {
        const int nbj = min(kSolveBlock, N - J * kSolveBlock);
        // this thread's entries of Lt_JK (4 columns x 4 rows), loaded before
        // the wait
        double lt[kSolveBlock / 16][kSolveBlock / kGJ];
#pragma unroll
        for (int c4 = 0; c4 < kSolveBlock / 16; ++c4) {
            const int cc = cg + 16 * c4;
            const double* col = Wn + (long long)(s0 + cc) * N + J * kSolveBlock;
#pragma unroll
            for (int r4 = 0; r4 < kSolveBlock / kGJ; ++r4) {
                const int ii = lane + r4 * kGJ;
                lt[c4][r4] = (cc < nbk && ii < nbj) ? __ldcg(col + ii) : 0.0;
            }
        }
        if (!wait_flag(flags + J, 1u, v.status, v.spin_limit)) return false;
        if (tid < kSolveBlock) S.dep[tid] = tid < nbj ? __ldcg(out + J * kSolveBlock + tid) : 0.0;
        __syncthreads();
#pragma unroll
        for (int c4 = 0; c4 < kSolveBlock / 16; ++c4) {
            const int cc = cg + 16 * c4;
            double acc = 0.0;
#pragma unroll
            for (int r4 = 0; r4 < kSolveBlock / kGJ; ++r4) acc = fma(lt[c4][r4], S.dep[lane + r4 * kGJ], acc);
#pragma unroll
            for (int w = kGJ / 2; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w, kGJ);
            if (lane == 0) S.part[0][cc] = acc;
        }
        __syncthreads();
        if (tid < kSolveBlock) S.rhs[tid] -= S.part[0][tid];
    }
    __syncthreads();
    if (tid < kGJ) S.sol[(kSolveSub - 1) * kGJ + tid] = S.rhs[(kSolveSub - 1) * kGJ + tid];
    __syncthreads();
    const int sc = tid / kGJ, p = tid % kGJ;
    for (int b = kSolveSub - 2; b >= 0; --b) {
        double acc = 0.0;
        for (int a = b + 1; a < kSolveSub; ++a) acc = fma(S.Ls[tri_pair(a, b)][p][sc], S.sol[a * kGJ + p], acc);
#pragma unroll
        for (int w = kGJ / 2; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w, kGJ);
        if (p == 0) S.sol[b * kGJ + sc] = S.rhs[b * kGJ + sc] - acc;
        __syncthreads();
    }
    if (tid < nbk) out[s0 + tid] = S.sol[tid];
    tri_publish(flags + K);
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// Solve-phase tree sweeps (Algorithm 1's upward pass of the particular
// fluxes and its downward pass of the interface unknowns), every tree height
// in one cooperative launch with a grid barrier between heights.  Each
// height's dot products are spread over the whole grid, so that the top of
// the tree (few nodes, long rows of W and X) keeps enough loads in flight.

// Lanes per output of the up sweep: a power of two, up to 32, so that each
// lane has about kUpTerms terms (FP64 products are costly per warp
// instruction: they are spread thin, and padded ones are avoided).
constexpr int kUpTerms = 4;
constexpr long long kTreePrefetchMax = 64LL << 20;   // half the L2
__device__ __forceinline__ int tree_up_lanes(int g2) {
    int l = 1;
    while (l < 32 && l * kUpTerms < g2) l <<= 1;
    return l;
}

// Hint one 128-byte line of global memory into L2.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
// Every line of [p, p + bytes) into L2, spread over the grid's threads.
__device__ __forceinline__ void prefetch_range_l2(const void* p, long long bytes, long long t0, long long stride) {
    const char* c = static_cast<const char*>(p);
    for (long long off = t0 * 128; off < bytes; off += stride * 128) prefetch_l2(c + off);
}

// rbar_node(i) = sum_k X(k, i) rbar_gamma(k) + rbar of outer segment i
// (i < m, k < 2g).  Per height: rbar_gamma of every node gathered from the
// children into rgam, a grid barrier, then the dot products on contiguous
// rgam (no dependent gathers inside them).
__global__ void __launch_bounds__(256) tree_up_kernel(DevView v, TreeLevels L, unsigned int* counter) {
    __shared__ TriSmem TS;
    const int tid = threadIdx.x, lane = tid & 31;
    const long long stride = (long long)gridDim.x * 256;
    const long long t0 = (long long)blockIdx.x * 256 + tid;
    unsigned int round = 0;
    // The static data of both sweeps (descriptors, index maps, X, W) into L2
    // first, in the order of use, when it fits there with room to spare: each
    // height is then a short chain of dependent loads, and cold misses would
    // set its pace.  Larger trees (X and W of a 4096^2 field: ~1 GB) would
    // only stream W through L2 ahead of a sweep that does not read it.
    prefetch_range_l2(v.merges, L.n_merges * (long long)sizeof(MergeDesc), t0, stride);
    prefetch_range_l2(v.node_map, L.map_len * (long long)sizeof(int), t0, stride);
    if ((L.x_len + L.w_len) * (long long)sizeof(double) <= kTreePrefetchMax) {
        prefetch_range_l2(v.X, L.x_len * (long long)sizeof(double), t0, stride);
        prefetch_range_l2(v.W, L.w_len * (long long)sizeof(double), t0, stride);
    }
    for (int h = 0; h < L.height; ++h) {
        const int first = L.first[h], count = L.count[h], g2max = L.g2[h], mmax = L.m[h];
        if (count == 0) continue;                           // uniform over the grid
        if (L.form[h]) {
            // a root level in the factor form (no outer segments): y =
            // Lt^-1 Q^T S rbar_gamma into fwd, block by block (left-looking)
            const int nsb = (g2max + kSolveBlock - 1) / kSolveBlock;
            unsigned int* fl = v.tri_flags;
            for (long long t = t0; t < (long long)count * nsb; t += stride) fl[t] = 0u;
            if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
            for (int item = blockIdx.x; item < count * nsb; item += gridDim.x) {
                const int K = item / count, q = item % count;
                const MergeDesc D = v.merges[first + q];
                if (K * kSolveBlock >= 2 * D.g) continue;                  // uniform per CTA
                if (!tri_forward_item(v, D, K, fl + (long long)q * nsb, TS)) return;
            }
            if (h + 1 < L.height && !grid_barrier(counter, round, v.status, v.spin_limit)) return;
            continue;
        }
        for (long long t = t0; t < (long long)count * g2max; t += stride) {
            int q, k;
            udivmod(t, g2max, q, k);
            const MergeDesc D = v.merges[first + q];
            if (k >= 2 * D.g) continue;
            const NodeRefs N = node_refs(v, D);
            v.rgam[2LL * D.gamma_off + k] = k < N.g ? __ldcg(v.rbar + D.r1_off + N.gpos1[k])
                                                    : __ldcg(v.rbar + D.r2_off + N.gpos2[k - N.g]);
        }
        if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
        if (mmax == 0) continue;                            // (the root) uniform
        const int lanes = tree_up_lanes(g2max);
        const unsigned int gmask = (lanes == 32 ? 0xffffffffu : ((1u << lanes) - 1u) << (lane & ~(lanes - 1)));
        const long long total = (long long)count * mmax * lanes;
        for (long long t = t0; t < total; t += stride) {
            int o, sub, q, i;
            udivmod(t, lanes, o, sub);
            udivmod(o, mmax, q, i);
            const MergeDesc D = v.merges[first + q];
            const int g2 = 2 * D.g;
            const double* rg = v.rgam + 2LL * D.gamma_off;
            double acc = 0.0;
            if (i < D.m) {
                // blocks of kUpTerms terms per lane (one block up to
                // 2g = 32 kUpTerms), all loads issued before the products
                const double* xc = v.X + D.X_off + (long long)i * g2;
                double a0 = 0.0, a1 = 0.0;
                int kb = sub;
                for (; kb + (kUpTerms - 1) * lanes < g2; kb += kUpTerms * lanes) {
                    double xv[kUpTerms], rv[kUpTerms];
#pragma unroll
                    for (int u = 0; u < kUpTerms; ++u) {
                        xv[u] = xc[kb + u * lanes];
                        rv[u] = __ldcg(rg + kb + u * lanes);
                    }
#pragma unroll
                    for (int u = 0; u < kUpTerms; u += 2) {
                        a0 = fma(xv[u], rv[u], a0);
                        a1 = fma(xv[u + 1], rv[u + 1], a1);
                    }
                }
                for (; kb < g2; kb += lanes) a0 = fma(xc[kb], __ldcg(rg + kb), a0);
                acc = a0 + a1;
            }
            for (int w = lanes >> 1; w > 0; w >>= 1) acc += __shfl_xor_sync(gmask, acc, w, lanes);
            if (sub == 0 && i < D.m) {
                const NodeRefs N = node_refs(v, D);
                const double ro = i < N.o1 ? __ldcg(v.rbar + D.r1_off + N.opos1[i])
                                           : __ldcg(v.rbar + D.r2_off + N.opos2[i - N.o1]);
                v.rbar[D.r_off + i] = acc + ro;
            }
        }
        if (h + 1 < L.height && !grid_barrier(counter, round, v.status, v.spin_limit)) return;
    }
}

// lambda_gamma(r) = sum_j X(r, j) lambda_o(j) - sum_k W(r, k) rbar_gamma(k),
// scattered to the children, whose outer lambda are copied from the node;
// rbar_gamma is read from rgam, which the up sweep of the same pass wrote.
// Data written by other CTAs of the launch (lambda, partial sums) is read
// with L2-only loads: a line left in L1 from an earlier height may be stale.
// Thread per (node, row r, term chunk), the chunk taken in blocks of
// kDownTerms terms whose loads are all in flight together; with several
// chunks the partial sums go to scratch and a second phase adds them in
// chunk order.
constexpr int kDownTerms = 8;
__global__ void __launch_bounds__(256) tree_down_kernel(DevView v, TreeLevels L, double* scratch,
                                                        unsigned int* counter) {
    __shared__ TriSmem TS;
    const int tid = threadIdx.x;
    const long long stride = (long long)gridDim.x * 256;
    const long long t0 = (long long)blockIdx.x * 256 + tid;
    unsigned int round = 0;
    for (int h = L.height - 1; h >= 0; --h) {
        const int first = L.first[h], count = L.count[h], g2max = L.g2[h], mmax = L.m[h], nkc = L.nkc[h];
        if (count == 0) continue;                           // uniform over the grid
        if (L.form[h]) {
            // a root level in the factor form: x = Lt^-T P y (P: the inverse
            // diagonal blocks of the factor, y from the up sweep) into rgam,
            // block by block from the last, then lambda_gamma = -S Q x to the
            // children
            const int nsb = (g2max + kSolveBlock - 1) / kSolveBlock;
            unsigned int* fl = v.tri_flags + v.tri_flag_n;
            for (long long t = t0; t < (long long)count * nsb; t += stride) fl[t] = 0u;
            if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
            for (int item = blockIdx.x; item < count * nsb; item += gridDim.x) {
                const int K = nsb - 1 - item / count, q = item % count;
                const MergeDesc D = v.merges[first + q];
                if (K * kSolveBlock >= 2 * D.g) continue;                  // uniform per CTA
                if (!tri_backward_item(v, D, K, fl + (long long)q * nsb, TS)) return;
            }
            if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
            const int gmax = g2max / 2;
            for (long long t = t0; t < (long long)count * gmax; t += stride) {
                int q, i;
                udivmod(t, gmax, q, i);
                const MergeDesc D = v.merges[first + q];
                if (i >= D.g) continue;
                const NodeRefs N = node_refs(v, D);
                const double* x = v.rgam + 2LL * D.gamma_off;
                const double xd = __ldcg(x + i), xs = __ldcg(x + D.g + i);
                const double sc = kRsqrt2 / sqrt(gamma_D(v, D, i));
                v.lam[D.r1_off + N.gpos1[i]] = sc * (xd - xs);
                v.lam[D.r2_off + N.gpos2[i]] = -(sc * (xd + xs));
            }
            if (h > 0 && !grid_barrier(counter, round, v.status, v.spin_limit)) return;
            continue;
        }
        const int kc_len = L.kcl[h];
        const long long rows = (long long)count * nkc * g2max;
        // the rows, then the children's outer lambda (copied from the node),
        // in one index space so that their load chains overlap
        for (long long t = t0; t < rows + (long long)count * mmax; t += stride) {
            if (t >= rows) {
                int q, j;
                udivmod(t - rows, mmax, q, j);
                const MergeDesc D = v.merges[first + q];
                if (j >= D.m) continue;
                const NodeRefs N = node_refs(v, D);
                const double lo = __ldcg(v.lam + D.r_off + j);
                if (j < N.o1) v.lam[D.r1_off + N.opos1[j]] = lo;
                else v.lam[D.r2_off + N.opos2[j - N.o1]] = lo;
                continue;
            }
            int r, qk, q, kc;
            udivmod(t, g2max, qk, r);
            udivmod(qk, nkc, q, kc);
            const MergeDesc D = v.merges[first + q];
            const NodeRefs N = node_refs(v, D);
            if (r >= N.g2) continue;
            const double* lam_o = v.lam + D.r_off;
            const double* X = v.X + D.X_off;
            const double* W = v.W + D.W_off;
            const int lo = kc * kc_len, hi = min(lo + kc_len, N.m + N.g2);
            const double* rg = v.rgam + 2LL * D.gamma_off;
            double a[4] = {0.0, 0.0, 0.0, 0.0};
            int jb = lo;
            for (; jb + kDownTerms <= hi; jb += kDownTerms) {
                // one block of terms: every load issued before the products
                double mv[kDownTerms], cv[kDownTerms];
#pragma unroll
                for (int u = 0; u < kDownTerms; ++u) {
                    const int j = jb + u;
                    const bool xpart = j < N.m;
                    mv[u] = xpart ? X[(long long)j * N.g2 + r] : W[(long long)(j - N.m) * N.g2 + r];
                    cv[u] = xpart ? __ldcg(lam_o + j) : neg_bits(__ldcg(rg + (j - N.m)));
                }
#pragma unroll
                for (int u = 0; u < kDownTerms; ++u) a[u & 3] = fma(mv[u], cv[u], a[u & 3]);
            }
            for (; jb < hi; ++jb) {
                const bool xpart = jb < N.m;
                const double mvv = xpart ? X[(long long)jb * N.g2 + r] : W[(long long)(jb - N.m) * N.g2 + r];
                const double cvv = xpart ? __ldcg(lam_o + jb) : neg_bits(__ldcg(rg + (jb - N.m)));
                a[jb & 3] = fma(mvv, cvv, a[jb & 3]);
            }
            const double part = (a[0] + a[1]) + (a[2] + a[3]);
            if (nkc == 1) {
                if (r < N.g) v.lam[D.r1_off + N.gpos1[r]] = part;
                else v.lam[D.r2_off + N.gpos2[r - N.g]] = part;
            } else {
                scratch[t] = part;
            }
        }
        if (nkc > 1) {
            if (!grid_barrier(counter, round, v.status, v.spin_limit)) return;
            // G lanes per row add the chunk partials, then a shuffle tree
            const int G = nkc < 32 ? nkc : 32;
            const int lane = tid & 31;
            const unsigned int gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (lane & ~(G - 1)));
            for (long long t = t0; t < (long long)count * g2max * G; t += stride) {
                int o, sub, q, r;
                udivmod(t, G, o, sub);
                udivmod(o, g2max, q, r);
                const MergeDesc D = v.merges[first + q];
                const double* ps = scratch + (long long)q * nkc * g2max + r;
                double lg = 0.0;
                if (r < 2 * D.g)
                    for (int kc = sub; kc < nkc; kc += G) lg += __ldcg(ps + (long long)kc * g2max);
                for (int w = G >> 1; w > 0; w >>= 1) lg += __shfl_xor_sync(gmask, lg, w, G);
                if (sub == 0 && r < 2 * D.g) {
                    const NodeRefs N = node_refs(v, D);
                    if (r < N.g) v.lam[D.r1_off + N.gpos1[r]] = lg;
                    else v.lam[D.r2_off + N.gpos2[r - N.g]] = lg;
                }
            }
        }
        if (h > 0 && !grid_barrier(counter, round, v.status, v.spin_limit)) return;
    }
}


}  // namespace

constexpr size_t kSmallSmemMax = 160 * 1024;
constexpr int kSweepSmemPad = 120 * 1024;   // > half an SM's shared memory

// shared memory of the per-node path for a level
static size_t small_smem(int max_g2, int max_m) {
    const size_t mstride = (size_t)(max_m | 1);
    return sizeof(double) * (2 * (size_t)max_g2 * max_g2 + (size_t)(max_g2 / 2) * mstride + (size_t)max_g2 * mstride);
}

bool merge_level_blocked(int, int max_g2, int max_m) {
    return max_g2 > kSmallMax || small_smem(max_g2, max_m) > kSmallSmemMax;
}

size_t merge_scratch_doubles(int count, int max_g2, int max_m) {
    if (!merge_level_blocked(count, max_g2, max_m)) return 0;
    return (size_t)count * (2 * kGJ * kGJ + 4 * (size_t)max_g2 * kGJ + 2);
}

// phase ids (include/mrcm.h)
enum { kPhMergeSmall = 2, kPhGjSweep = 3, kPhMergeForm = 4, kPhMergeX = 5, kPhMergeR = 6, kPhRootFactor = 13 };

struct HookScope {
    const PhaseHook& h;
    int phase;
    HookScope(const PhaseHook& h_, int p) : h(h_), phase(p) { if (h.begin) h.begin(h.ctx, p); }
    ~HookScope() { if (h.end) h.end(h.ctx, phase); }
};

template <class F>
static cudaError_t launch_small(const DevView& v, int first, int count, int max_g2, int max_m, cudaStream_t s) {
    const int mstride = max_m | 1;          // odd: rows of B and X start in different banks
    const size_t sm = small_smem(max_g2, max_m);
    auto go = [&](auto kern, int nt) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmemMax);
        if (e != cudaSuccess) return e;
        kern<<<count, nt, sm, s>>>(v, first, mstride);
        return cudaGetLastError();
    };
    if (max_g2 <= 8) return go(merge_small_kernel<F, 64>, 64);
    if (max_g2 <= 16) return go(merge_small_kernel<F, 128>, 128);
    return go(merge_small_kernel<F, kSmallThreads>, kSmallThreads);
}

// The three launches of a blocked level, each with its tuning choice (0:
// the heuristic below).  Every choice computes the same numbers: a tile,
// an X block or an R tile is formed by the same thread arithmetic whichever
// CTA shape runs it, so the tuner may pick any of them.
template <class F>
static cudaError_t sweep_launch(const DevView& v, int first, int count, int max_g2, double* scratch, void* barrier,
                                int sms, int per_sm, bool factor, cudaStream_t s) {
    cudaError_t e;
    const void* kern = factor ? (const void*)ldl_sweep_kernel<F> : (const void*)gj_sweep_kernel<F>;
    // Default one CTA per SM (the padded dynamic shared memory keeps a
    // second one off): the CTAs that invert the next diagonal blocks, which
    // lie on the sequential chain of the sweep, then own their SM's FP64
    // pipe.  Two or three per SM let one CTA's staging loads overlap the
    // others' tile updates, which pays where the tiles of a step outnumber
    // the CTAs many times over (the largest systems).
    if (per_sm < 1) per_sm = 1;              // the heuristic: one CTA per SM
    size_t dyn = kSweepSmemPad;
    if (per_sm >= 2) {
        dyn = std::max<size_t>((size_t)max_g2 * sizeof(double), 16);
        int fit = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, 256, dyn)) != cudaSuccess) return e;
        if (fit < per_sm) {
            per_sm = fit >= 2 ? fit : 1;
            if (per_sm == 1) dyn = kSweepSmemPad;
        }
    }
    const int tiles = (max_g2 + kGJTile - 1) / kGJTile;
    const long long items = (long long)count * (1 + tiles * (tiles + 1) / 2);
    int grid = (int)std::min<long long>(items, (long long)sms * per_sm);
    grid = grid < 1 ? 1 : grid;
    // the grid barrier's arrival counter and the tile loops' ticket counter
    if ((e = cudaMemsetAsync(barrier, 0, 2 * sizeof(unsigned int), s)) != cudaSuccess) return e;
    unsigned int* bar = reinterpret_cast<unsigned int*>(barrier);
    DevView vv = v;
    int f = first, c = count, n = max_g2;
    F* scr = reinterpret_cast<F*>(scratch);
    void* args[] = {&vv, &f, &c, &n, &scr, &bar};
    return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(256), args, dyn, s);
}
// A blocked level of many mid-sized systems takes the per-node inversion
// (gj_node_kernel): one CTA per node, no per-step grid barriers; from half
// as many nodes as SMs on, a node's whole elimination on one SM is shorter
// than the sweep's chain of block steps over the level.  A fixed rule (not
// a tuning choice, so that tuned launch shapes keep the bits of the result).
static bool node_level(int count, int max_g2, int sms) { return max_g2 <= kNodeMax && 2 * count >= sms; }
template <class F>
static cudaError_t node_launch(const DevView& v, int first, int count, int max_g2, cudaStream_t s) {
    cudaError_t e;
    if (max_g2 <= 64) {
        const size_t sm = sizeof(F) * NodeTri<64>::kTri;
        if ((e = cudaFuncSetAttribute(gj_node_kernel<64, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess)
            return e;
        gj_node_kernel<64, F><<<count, 256, sm, s>>>(v, first);
    } else {
        const size_t sm = sizeof(F) * NodeTri<kNodeMax>::kTri;
        if ((e = cudaFuncSetAttribute(gj_node_kernel<kNodeMax, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm)) != cudaSuccess)
            return e;
        gj_node_kernel<kNodeMax, F><<<count, 256, sm, s>>>(v, first);
    }
    return cudaGetLastError();
}
template <class F>
static cudaError_t x_launch(const DevView& v, int first, int count, int max_g2, int max_m, int sms, int rows,
                            cudaStream_t s) {
    const int ct = (max_m + kXColsOut - 1) / kXColsOut;
    const int rt64 = (max_g2 + 63) / 64;
    if (rows == 0) rows = (long long)count * rt64 * ct >= 64LL * sms ? 64 : 32;
    if (rows == 64) {
        merge_x_kernel<64, F><<<dim3(count, rt64 * ct), 256, 0, s>>>(v, first);
    } else {
        const int rt32 = (max_g2 + 31) / 32;
        merge_x_kernel<32, F><<<dim3(count, rt32 * ct), 256, 0, s>>>(v, first);
    }
    return cudaGetLastError();
}
template <class F>
static cudaError_t r_launch(const DevView& v, int first, int count, int max_m, int sms, int tile, cudaStream_t s) {
    const int rt32 = (max_m + 31) / 32;
    if (tile == 0) tile = (long long)count * rt32 * (rt32 + 1) / 2 >= 64LL * sms ? 32 : 16;
    if (tile == 32) {
        merge_rupdate_kernel<2, F><<<dim3(count, rt32 * (rt32 + 1) / 2), 256, 0, s>>>(v, first);
    } else {
        const int rt16 = (max_m + 15) / 16;
        merge_rupdate_kernel<1, F><<<dim3(count, rt16 * (rt16 + 1) / 2), 256, 0, s>>>(v, first);
    }
    return cudaGetLastError();
}

static cudaError_t device_sms(int* sms) {
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    return cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
}

template <class F>
static cudaError_t sweep_attributes() {
    cudaError_t e = cudaFuncSetAttribute(gj_sweep_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSweepSmemPad);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(ldl_sweep_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmemPad);
}

template <class F>
static cudaError_t launch_merge_build_t(const DevView& v, int first, int count, int max_g2, int max_m, bool factor,
                                        const MergeTune& tune, double* scratch, void* barrier, cudaStream_t s,
                                        int* launches, const PhaseHook& hook) {
    if (count == 0) return cudaSuccess;
    cudaError_t e;
    // per call, so that every device the library runs on gets its own SM
    // count and the sweep's shared-memory attribute (cheap host calls; a
    // captured build makes them once)
    int sms = 0;
    if ((e = device_sms(&sms)) != cudaSuccess) return e;
    if ((e = sweep_attributes<F>()) != cudaSuccess) return e;
    if (!merge_level_blocked(count, max_g2, max_m)) {
        HookScope hs(hook, kPhMergeSmall);
        e = launch_small<F>(v, first, count, max_g2, max_m, s);
        ++*launches;
        return e;
    }
    factor = factor && max_m == 0;
    {
        HookScope hs(hook, factor ? kPhRootFactor : kPhGjSweep);
        if (!factor && node_level(count, max_g2, sms))
            e = node_launch<F>(v, first, count, max_g2, s);
        else
            e = sweep_launch<F>(v, first, count, max_g2, scratch, barrier, sms, tune.sweep_per_sm, factor, s);
        ++*launches;
        if (e != cudaSuccess) return e;
    }
    if (max_m > 0) {
        {
            HookScope hs(hook, kPhMergeX);
            e = x_launch<F>(v, first, count, max_g2, max_m, sms, tune.x_rows, s);
            ++*launches;
            if (e != cudaSuccess) return e;
        }
        HookScope hs(hook, kPhMergeR);
        e = r_launch<F>(v, first, count, max_m, sms, tune.r_tile, s);
        ++*launches;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_merge_build(const DevView& v, int first, int count, int max_g2, int max_m, bool fp32,
                               bool factor, const MergeTune& tune, double* scratch, void* barrier, cudaStream_t s,
                               int* launches, const PhaseHook& hook) {
    if (fp32)
        return launch_merge_build_t<float>(v, first, count, max_g2, max_m, factor, tune, scratch, barrier, s,
                                           launches, hook);
    return launch_merge_build_t<double>(v, first, count, max_g2, max_m, factor, tune, scratch, barrier, s, launches,
                                        hook);
}

// Times fn (one launch, already valid to repeat) `reps` times on s with
// events; the best run in ms.
template <class Fn>
static cudaError_t best_time(cudaStream_t s, int reps, cudaEvent_t e0, cudaEvent_t e1, Fn&& fn, float* best) {
    *best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaError_t e;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
        if ((e = fn()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
        *best = std::min(*best, ms);
    }
    return cudaSuccess;
}

template <class F>
static cudaError_t tune_level_t(const DevView& v, int first, int count, int max_g2, int max_m, bool factor,
                                double* scratch, void* barrier, cudaStream_t s, int reps, MergeTune* out) {
    *out = MergeTune{};
    if (count == 0 || !merge_level_blocked(count, max_g2, max_m)) return cudaSuccess;
    int sms = 0;
    cudaError_t e;
    if ((e = device_sms(&sms)) != cudaSuccess) return e;
    if ((e = sweep_attributes<F>()) != cudaSuccess) return e;
    factor = factor && max_m == 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 1e30f;
    for (int per_sm : {1, 2, 3, 4}) {
        if (!factor && node_level(count, max_g2, sms)) break;        // the per-node kernel: no shape to pick
        float t = 0.f;
        e = best_time(s, reps, e0, e1, [&] {
            return sweep_launch<F>(v, first, count, max_g2, scratch, barrier, sms, per_sm, factor, s);
        }, &t);
        if (e != cudaSuccess) break;
        if (t < best) { best = t; out->sweep_per_sm = per_sm; }
    }
    if (e == cudaSuccess && max_m > 0) {
        best = 1e30f;
        for (int rows : {32, 64}) {
            float t = 0.f;
            e = best_time(s, reps, e0, e1, [&] { return x_launch<F>(v, first, count, max_g2, max_m, sms, rows, s); },
                          &t);
            if (e != cudaSuccess) break;
            if (t < best) { best = t; out->x_rows = rows; }
        }
    }
    if (e == cudaSuccess && max_m > 0) {
        best = 1e30f;
        for (int tile : {16, 32}) {
            float t = 0.f;
            e = best_time(s, reps, e0, e1, [&] { return r_launch<F>(v, first, count, max_m, sms, tile, s); }, &t);
            if (e != cudaSuccess) break;
            if (t < best) { best = t; out->r_tile = tile; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

cudaError_t tune_merge_level(const DevView& v, int first, int count, int max_g2, int max_m, bool fp32, bool factor,
                             double* scratch, void* barrier, cudaStream_t s, int reps, MergeTune* out) {
    if (fp32) return tune_level_t<float>(v, first, count, max_g2, max_m, factor, scratch, barrier, s, reps, out);
    return tune_level_t<double>(v, first, count, max_g2, max_m, factor, scratch, barrier, s, reps, out);
}

cudaError_t tree_grid(int* grid) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tree_down_kernel, 256, 0)) != cudaSuccess) return e;
    int per_up = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_up, tree_up_kernel, 256, 0)) != cudaSuccess) return e;
    per = std::min(std::min(per, per_up), 2);
    *grid = std::max(1, sms * std::max(per, 1));
    return cudaSuccess;
}

long long tree_plan_chunks(TreeLevels& L, int grid) {
    // A warp-wide FP64 instruction holds its scheduler for many cycles, so a
    // height's products have to be spread over the whole grid: the terms of
    // a row are split into chunks (a power of two of them) until rows x
    // chunks fills the grid's threads, keeping at least 8 terms per chunk.
    const long long threads = (long long)grid * 256;
    long long need = 0;
    for (int h = 0; h < L.height; ++h) {
        const long long rows = (long long)L.count[h] * L.g2[h];
        const int T = L.m[h] + L.g2[h];
        int nkc = 1;
        while (rows * nkc * 2 <= threads && (T + 2 * nkc - 1) / (2 * nkc) >= 8) nkc *= 2;
        L.nkc[h] = nkc;
        L.kcl[h] = ((T + nkc - 1) / nkc + 7) / 8 * 8;
        if (nkc > 1) need = std::max(need, rows * nkc);
    }
    return need;
}

cudaError_t launch_tree_up(const DevView& v, const TreeLevels& L, int grid, void* barrier, cudaStream_t s) {
    if (L.height == 0) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaMemsetAsync(barrier, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
    DevView vv = v;
    TreeLevels ll = L;
    unsigned int* bar = reinterpret_cast<unsigned int*>(barrier);
    void* args[] = {&vv, &ll, &bar};
    return cudaLaunchCooperativeKernel((const void*)tree_up_kernel, dim3(grid), dim3(256), args, 0, s);
}

cudaError_t launch_tree_down(const DevView& v, const TreeLevels& L, int grid, double* scratch, void* barrier,
                             cudaStream_t s) {
    if (L.height == 0) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaMemsetAsync(barrier, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
    DevView vv = v;
    TreeLevels ll = L;
    unsigned int* bar = reinterpret_cast<unsigned int*>(barrier);
    void* args[] = {&vv, &ll, &scratch, &bar};
    return cudaLaunchCooperativeKernel((const void*)tree_down_kernel, dim3(grid), dim3(256), args, 0, s);
}

}  // namespace mrcm
