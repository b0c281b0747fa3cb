// Leaf kernels: the local Robin problems of every finest-level subdomain.
//
// arXiv 2009.07965, Eqs. (11.2)-(12.2) on one leaf with lumped RT0 (two-point
// fluxes).  On a skeleton face e of segment t the Robin term gives the
// outward flux F_e = rho_e (p_c - lambda_t), lambda_t = P_t - beta_t U_t
// (n_t . n^i), so the interface data of the MMBF problems (Eqs.
// 11Hhatbasisa / 11Hhatbasisb) enter only through one Robin datum per
// segment.  With the leaf pressure matrix A (SPD: two-point couplings plus
// the Robin / Dirichlet diagonal) and B[c, s] = rho_e for the face e of cell
// c in segment s:
//     p = A^-1 (bbar + B lambda),   F_s = (B^T A^-1 B - W) lambda + B^T A^-1 bbar,
// W_s = sum_{e in s} rho_e.  The Robin-to-flux map R = B^T A^-1 B - W holds
// the traces of all MMBFs of the leaf (coefficient-tracking remark, Section
// 3.2); bbar carries the source and external boundary data (Eqs. addu, addp).
//
// Layout and mapping.  16 threads own one leaf (two leaves per warp, four
// per CTA so that a 64 x 64-leaf grid fits in one wave); cells are ordered x
// fastest, so A is banded with half-bandwidth w (leaf width).  A = L D L^T
// is factored right-looking over a circular window of w+2 band rows in
// shared memory; each step also advances the multi-right-hand-side forward
// solve Z = L^-1 B and accumulates R += z_k z_k^T / d_k, so no column of L is
// read twice.  The columns of B are taken in the order of their first
// nonzero row, so the structurally zero upper part of Z is skipped and the
// remaining work is spread evenly over the 16 lanes (a masked FP64 lane
// costs as much as a busy one).  The multipliers L, 1/d and Z are written to
// global memory for the solve phase.
#include "mrcm_internal.h"

namespace mrcm {
namespace {

constexpr int kWin = kMaxLeafSide + 2;   // circular window rows

// T: the arithmetic of the factorisation (double; float in the mixed form).
template <int MMAX, class T>
struct LeafBuildSmem {
    T win[kWin][kMaxLeafSide + 1];       // win[row % (w+2)][o] = A[row][row - o]
    T zw[kWin][MMAX + 1];                // rows of Z being updated (ordered columns)
    T R[MMAX][MMAX + 1];                 // lower triangle of B^T A^-1 B (ordered)
    double W[MMAX];                      // sum of rho per segment (ordered)
    T lcol[kMaxLeafSide];                // column k of L below the diagonal
    T zk[MMAX];                          // row k of Z (ordered)
    T uk[MMAX];                          // row k of Z / d_k (ordered)
    int order[MMAX];                     // ordered column q -> local segment
    int pos[MMAX];                       // local segment -> ordered column
    int start[MMAX];                     // first row with a nonzero, per ordered column
    double dg[kLeafThreads];             // diagonal entries of the next rows to enter (row % 16)
};

// (row, col) of entry idx of a lower triangle stored row by row.
__device__ __forceinline__ void tri_index(int idx, int& r, int& c) {
    r = (int)((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= idx) ++r;
    while (r * (r + 1) / 2 > idx) --r;
    c = idx - r * (r + 1) / 2;
}

// Face coefficients around local cell (i, j) of leaf L.
struct CellFaces {
    double w_, e_, s_, n_;   // coefficient seen from the cell: west, east, south, north
    double tx, ty;           // couplings to the west / south neighbour inside the leaf
};

__device__ __forceinline__ CellFaces cell_faces(const DevView& v, const LeafDesc& L, int i, int j) {
    const GridDesc& G = v.grids[L.grid];
    const int gi = L.i0 + i, gj = L.j0 + j;
    const long long fx = G.fx0 + gi + (long long)(G.nx + 1) * gj;
    const long long fy = G.fy0 + gi + (long long)G.nx * gj;
    CellFaces c;
    c.w_ = v.cxU[fx];
    c.e_ = v.cxL[fx + 1];
    c.s_ = v.cyU[fy];
    c.n_ = v.cyL[fy + G.nx];
    c.tx = (i > 0) ? v.cxL[fx] : 0.0;
    c.ty = (j > 0) ? v.cyL[fy] : 0.0;
    return c;
}

// Local segments of the Robin faces of cell (i, j), -1 where the face is not
// on the skeleton.
__device__ __forceinline__ void cell_robin_segments(const DevView& v, const LeafDesc& L, int i, int j,
                                                    int& sw, int& se, int& ss, int& sn) {
    sw = (i == 0 && L.side_off[0] >= 0) ? L.side_off[0] + j / v.gy : -1;
    se = (i == L.w - 1 && L.side_off[1] >= 0) ? L.side_off[1] + j / v.gy : -1;
    ss = (j == 0 && L.side_off[2] >= 0) ? L.side_off[2] + i / v.gx : -1;
    sn = (j == L.h - 1 && L.side_off[3] >= 0) ? L.side_off[3] + i / v.gx : -1;
}

// Diagonal entry of row `row` of the leaf matrix: the sum of the cell's face
// coefficients.
__device__ __forceinline__ double row_diag(const DevView& v, const LeafDesc& L, int row) {
    const CellFaces f = cell_faces(v, L, row % L.w, row / L.w);
    return (f.w_ + f.e_) + (f.s_ + f.n_);
}

// Row `row` of the band into the window and its Robin columns into zw.  The
// diagonal entry comes from S.dg (formed 16 rows at a time, one row per
// lane: an FP64 instruction costs a whole warp's issue however few lanes it
// uses), or is formed here when `fresh` (the rows before the elimination).
template <int MMAX, class T>
__device__ __forceinline__ void init_row(const DevView& v, const LeafDesc& L, LeafBuildSmem<MMAX, T>& S,
                                         int row, int t, bool fresh) {
    const int w = L.w, m = L.m;
    const int i = row % w, j = row / w;
    const int slot = row % (w + 2);
    const CellFaces f = cell_faces(v, L, i, j);
    for (int o = t; o <= w; o += kLeafThreads) {
        double a = 0.0;
        if (o == 0) a = fresh ? (f.w_ + f.e_) + (f.s_ + f.n_) : S.dg[row % kLeafThreads];
        if (o == 1 && i > 0) a = neg_bits(f.tx);
        if (o == w && j > 0) a = neg_bits(f.ty);   // w == 1: the y neighbour sits at offset 1
        S.win[slot][o] = (T)a;
    }
    int sw, se, ss, sn;
    cell_robin_segments(v, L, i, j, sw, se, ss, sn);
    for (int q = t; q < m; q += kLeafThreads) {
        const int s = S.order[q];
        double b = 0.0;
        if (s == sw) b = f.w_;
        if (s == se) b = f.e_;
        if (s == ss) b = f.s_;
        if (s == sn) b = f.n_;
        S.zw[slot][q] = (T)b;
    }
}

// Sum of the Robin coefficients rho_e over the faces of local segment s,
// seen from the leaf's own cells (the diagonal W_s of B^T A^-1 B - W).
__device__ __forceinline__ double segment_rho_sum(const DevView& v, const LeafDesc& L, int s) {
    int side = 0;
    for (int d = 1; d < 4; ++d)
        if (L.side_off[d] >= 0 && s >= L.side_off[d]) side = d;
    const int p = s - L.side_off[side];
    const int len = side < 2 ? L.h : L.w, g = side < 2 ? v.gy : v.gx;
    const GridDesc& G = v.grids[L.grid];
    const double* cxL = v.cxL + G.fx0;
    const double* cxU = v.cxU + G.fx0;
    const double* cyL = v.cyL + G.fy0;
    const double* cyU = v.cyU + G.fy0;
    double sum = 0.0;
    for (int e = p * g; e < min((p + 1) * g, len); ++e) {
        if (side == 0) sum += cxU[(long long)L.i0 + (long long)(G.nx + 1) * (L.j0 + e)];
        else if (side == 1) sum += cxL[(long long)(L.i0 + L.w) + (long long)(G.nx + 1) * (L.j0 + e)];
        else if (side == 2) sum += cyU[(long long)(L.i0 + e) + (long long)G.nx * L.j0];
        else sum += cyL[(long long)(L.i0 + e) + (long long)G.nx * (L.j0 + L.h)];
    }
    return sum;
}

// First row of the leaf whose cell touches local segment s (the first
// nonzero of column s of B).
__device__ __forceinline__ int segment_start_row(const DevView& v, const LeafDesc& L, int s) {
    const int w = L.w, h = L.h;
    if (L.side_off[3] >= 0 && s >= L.side_off[3]) return (h - 1) * w + (s - L.side_off[3]) * v.gx;
    if (L.side_off[2] >= 0 && s >= L.side_off[2]) return (s - L.side_off[2]) * v.gx;
    if (L.side_off[1] >= 0 && s >= L.side_off[1]) return (s - L.side_off[1]) * v.gy * w + w - 1;
    return (s - L.side_off[0]) * v.gy * w;
}

// Body of the leaf build for one leaf; WF > 0 fixes the leaf to WF x WF
// cells at compile time (the full leaf), 0 reads the size from the
// descriptor (truncated leaves).  T: arithmetic and storage of the factors
// (double, or float in the mixed form; the map R is stored in double).
template <int MMAX, int WF, class T>
__device__ __forceinline__ void leaf_build_body(const DevView& v, LeafBuildSmem<MMAX, T>& S, const LeafDesc& L,
                                                int t, unsigned mask) {
    const int w = WF ? WF : L.w, n = WF ? WF * WF : L.w * L.h, m = L.m, W2 = w + 2;
    T* Lg = leaf_L<T>(v) + L.L_off;          // n x 16 multipliers
    T* Dg = Lg + (long long)n * kLeafThreads;   // n reciprocal pivots
    T* Zg = leaf_Z<T>(v) + L.Z_off;          // n x m, column-major (local segment order)

    // Columns of B ordered by their first nonzero row: column q of Z stays
    // zero above start[q], so only the first c_k ordered columns take part
    // in step k of the forward solve and of the R accumulation.
    if (t == 0) {
        for (int s = 0; s < m; ++s) {
            const int st = segment_start_row(v, L, s);
            int q = s;
            while (q > 0 && S.start[q - 1] > st) {
                S.start[q] = S.start[q - 1];
                S.order[q] = S.order[q - 1];
                --q;
            }
            S.start[q] = st;
            S.order[q] = s;
        }
        for (int q = 0; q < m; ++q) S.pos[S.order[q]] = q;
    }
    __syncwarp(mask);

    for (int idx = t; idx < m * (MMAX + 1); idx += kLeafThreads) S.R[idx / (MMAX + 1)][idx % (MMAX + 1)] = (T)0;
    const int first = min(w, n - 1);
    for (int r = 0; r <= first; ++r) init_row(v, L, S, r, t, true);
    __syncwarp(mask);

    // per-thread index patterns of the two triangles (band update: rows a >=
    // b of the w x w trailing block; R update: r >= c of the active columns),
    // fixed for the whole elimination: entry idx = t + 16 e
    constexpr int kBandEnt = (kMaxLeafSide * (kMaxLeafSide + 1) / 2 + kLeafThreads - 1) / kLeafThreads;
    constexpr int kREnt = (MMAX * (MMAX + 1) / 2 + kLeafThreads - 1) / kLeafThreads;
    constexpr bool kRPre = kREnt <= 12;       // keep the R pattern in registers when it is small
    constexpr int kRReg = kRPre ? kREnt : 1;
    int band_a[kBandEnt], band_b[kBandEnt], tri_r[kRReg], tri_c[kRReg];
#pragma unroll
    for (int e = 0; e < kBandEnt; ++e) tri_index(t + e * kLeafThreads, band_a[e], band_b[e]);
    if constexpr (kRPre) {
#pragma unroll
        for (int e = 0; e < kREnt; ++e) tri_index(t + e * kLeafThreads, tri_r[e], tri_c[e]);
    }

    bool bad_pivot = false;
    int ck = 0;                      // active ordered columns
    int sk = 0;                      // window slot of row k (k mod W2)
    for (int k = 0; k < n; ++k) {
        // diagonals of the rows entering the window in steps k .. k + 15 (read
        // after the warp barrier of phase A)
        if ((k & (kLeafThreads - 1)) == 0) {
            const int r = k + w + 1 + t;
            if (r < n) S.dg[r % kLeafThreads] = row_diag(v, L, r);
        }
        while (ck < m && S.start[ck] <= k) ++ck;
        const int s1 = sk + 1 == W2 ? 0 : sk + 1;        // slot of row k + 1
        // ---- phase A: pivot, multipliers, row k of Z -------------------------
        const T dk = S.win[sk][0];
        // dk > 0 and finite, tested on the bit pattern (no FP64 compare)
        bad_pivot |= !positive_finite_bits(dk);
        const T rcp = rcp_nr(dk);
        const int wk = min(w, n - 1 - k);
        if (t < wk) {
            int sl = s1 + t;
            sl -= sl >= W2 ? W2 : 0;
            const T l = S.win[sl][1 + t] * rcp;
            S.lcol[t] = l;
            Lg[(long long)k * kLeafThreads + t] = l;
        }
        if (t == 0) Dg[k] = rcp;
        for (int q = t; q < ck; q += kLeafThreads) {
            const T z = S.zw[sk][q];
            S.zk[q] = z;
            S.uk[q] = z * rcp;
        }
        __syncwarp(mask);
        for (int s = t; s < m; s += kLeafThreads) {
            const int q = S.pos[s];
            Zg[(long long)s * n + k] = q < ck ? S.zk[q] : (T)0;
        }
        // ---- phase B: trailing band update, Z update, R update, new row -----
        const int ntri_w = wk * (wk + 1) / 2;
#pragma unroll
        for (int e = 0; e < kBandEnt; ++e) {
            if (t + e * kLeafThreads >= ntri_w) break;
            const int a = band_a[e], b = band_b[e];
            int ra = s1 + a, rb = s1 + b;
            ra -= ra >= W2 ? W2 : 0;
            rb -= rb >= W2 ? W2 : 0;
            T& x = S.win[ra][a - b];
            x = fma(-S.lcol[a], S.win[rb][1 + b], x);
        }
        if (ck > 0) {
            // (row a, column q) of entry idx = a ck + q, stepped by 16 entries
            const int nz = wk * ck, da = kLeafThreads / ck, dq = kLeafThreads - da * ck;
            int a = t / ck, q = t - a * ck;
            for (int idx = t; idx < nz; idx += kLeafThreads) {
                int ra = s1 + a;
                ra -= ra >= W2 ? W2 : 0;
                T& x = S.zw[ra][q];
                x = fma(-S.lcol[a], S.zk[q], x);
                a += da;
                q += dq;
                if (q >= ck) {
                    q -= ck;
                    ++a;
                }
            }
        }
        const int ntri_m = ck * (ck + 1) / 2;
        if constexpr (kRPre) {
#pragma unroll
            for (int e = 0; e < kREnt; ++e) {
                if (t + e * kLeafThreads >= ntri_m) break;
                const int r = tri_r[e], c = tri_c[e];
                S.R[r][c] = fma(S.zk[r], S.uk[c], S.R[r][c]);
            }
        } else {
            for (int idx = t; idx < ntri_m; idx += kLeafThreads) {
                int r, c;
                tri_index(idx, r, c);
                S.R[r][c] = fma(S.zk[r], S.uk[c], S.R[r][c]);
            }
        }
        if (k + w + 1 < n) init_row(v, L, S, k + w + 1, t, false);
        __syncwarp(mask);
        sk = s1;
    }
    if (bad_pivot) atomicOr(v.status, kStatusSingular);
    // W_s = sum of rho over the faces of segment s (seen from this leaf)
    for (int q = t; q < m; q += kLeafThreads) S.W[q] = segment_rho_sum(v, L, S.order[q]);
    __syncwarp(mask);
    double* Rg = v.R + L.R_off;
    for (int idx = t; idx < m * m; idx += kLeafThreads) {
        const int r = S.pos[idx / m], c = S.pos[idx % m];
        double val = (r >= c) ? (double)S.R[r][c] : (double)S.R[c][r];
        if (r == c) val -= S.W[r];
        Rg[idx] = val;
    }}

// Residency: the FP64 full-leaf variant holds 31 KB of shared memory per
// CTA, so 7 CTAs fit an SM; the register cap keeps all 7 resident (one wave
// of 1064 CTAs covers the 4096 leaves of a 1024^2 grid).
template <int MMAX, int LPB, class T>
__global__ void __launch_bounds__(kLeafThreads * LPB, MMAX == 16 ? (sizeof(T) == 8 ? 7 : 8) : 1)
leaf_build_kernel(DevView v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x & (kLeafThreads - 1);
    const int slot_leaf = threadIdx.x / kLeafThreads;
    const int leaf = blockIdx.x * LPB + slot_leaf;
    if (leaf >= v.nleaf) return;     // uniform over the 16 threads of the leaf
    const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
    LeafBuildSmem<MMAX, T>& S = reinterpret_cast<LeafBuildSmem<MMAX, T>*>(smem_raw)[slot_leaf];
    const LeafDesc L = v.leaves[leaf];
    if (L.w == kMaxLeafSide && L.h == kMaxLeafSide)
        leaf_build_body<MMAX, kMaxLeafSide, T>(v, S, L, t, mask);
    else
        leaf_build_body<MMAX, 0, T>(v, S, L, t, mask);
}

// ---------------------------------------------------------------------------
// Solve phase.  Right-hand side of the particular problem (Eqs. addu/addp):
// source plus Dirichlet and Neumann data of the leaf's domain-boundary faces.
__device__ __forceinline__ double particular_rhs(const DevView& v, const LeafDesc& L, const double* q,
                                                 const double* bc_val, int row) {
    const GridDesc& G = v.grids[L.grid];
    const int i = row % L.w, j = row / L.w;
    const int gi = L.i0 + i, gj = L.j0 + j;
    double b = q[G.c0 + (long long)gj * G.nx + gi];
    if (!bc_val) return b;
    const double* bv = bc_val + G.b0;
    if (gi == 0) {
        const double g = bv[gj];
        b += G.bc[0] ? v.cxU[G.fx0 + (long long)(G.nx + 1) * gj] * g : -G.hy * g;
    }
    if (gi == G.nx - 1) {
        const double g = bv[G.ny + gj];
        b += G.bc[1] ? v.cxL[G.fx0 + G.nx + (long long)(G.nx + 1) * gj] * g : -G.hy * g;
    }
    if (gj == 0) {
        const double g = bv[2 * G.ny + gi];
        b += G.bc[2] ? v.cyU[G.fy0 + gi] * g : -G.hx * g;
    }
    if (gj == G.ny - 1) {
        const double g = bv[2 * G.ny + G.nx + gi];
        b += G.bc[3] ? v.cyL[G.fy0 + gi + (long long)G.nx * G.ny] * g : -G.hx * g;
    }
    return b;
}

struct LeafSolveSmem {
    double y[kMaxLeafSide * kMaxLeafSide];             // right-hand side, swept in place
};

// Depth of the register ring that prefetches the band multipliers of the
// sweeps (rows streamed from HBM ahead of the sequential elimination chain).
constexpr int kSweepAhead = 16;

// Body of the particular solve for one leaf; NF, WF > 0 fix the row count
// and the band width at compile time (the full kMaxLeafSide^2 leaf: the
// sweep's bounds and end tests then fold away, which makes it ~3x faster),
// 0 reads them from the descriptor (truncated leaves).  TS: storage type of
// the factors (float in the mixed form); the sweep itself runs in FP64.
template <int NF, int WF, class TS>
__device__ __forceinline__ void leaf_particular_body(const DevView& v, const double* __restrict__ q,
                                                     const double* __restrict__ bc_val, bool with_sadj,
                                                     LeafSolveSmem& S, const LeafDesc& L, int t, unsigned mask) {
    const int w = WF ? WF : L.w, n = NF ? NF : L.w * L.h, m = L.m;
    const TS* Lg = leaf_L<TS>(v) + L.L_off;
    const TS* Dg = Lg + (long long)n * kLeafThreads;
    const TS* Zg = leaf_Z<TS>(v) + L.Z_off;
    double* zb = v.leafzb + L.zb_off;

    // forward sweep zbar = L^-1 bbar (unit lower band); the right-hand side
    // is formed for all rows first, the multipliers stream through a
    // register ring kSweepAhead steps ahead of their use
    for (int r = t; r < n; r += kLeafThreads) S.y[r] = particular_rhs(v, L, q, bc_val, r);
    __syncwarp(mask);
    double ring[kSweepAhead];
#pragma unroll
    for (int d = 0; d < kSweepAhead; ++d) ring[d] = (d < n && t < min(w, n - 1 - d)) ? Lg[(long long)d * kLeafThreads + t] : 0.0;
    for (int k0 = 0; k0 < n; k0 += kSweepAhead) {
#pragma unroll
        for (int d = 0; d < kSweepAhead; ++d) {
            const int k = k0 + d;
            if (k >= n) break;
            const double lk = ring[d];
            const int kn = k + kSweepAhead;
            ring[d] = (kn < n && t < min(w, n - 1 - kn)) ? Lg[(long long)kn * kLeafThreads + t] : 0.0;
            const double zk = S.y[k];
            if (t < min(w, n - 1 - k)) S.y[k + 1 + t] = fma(-lk, zk, S.y[k + 1 + t]);
            __syncwarp(mask);
        }
    }
    for (int k = t; k < n; k += kLeafThreads) zb[k] = S.y[k];
    // y = D^-1 zbar ; rbar = Z^T y  (= B^T A^-1 bbar): the 16 lanes share
    // every column of Z (consecutive rows, coalesced) and reduce by shuffles;
    // the lane's y stay in registers and all of its kRows loads of a column
    // are in flight together
    constexpr int kRows = kMaxLeafSide * kMaxLeafSide / kLeafThreads;
    double yv[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int k = t + r * kLeafThreads;
        yv[r] = k < n ? S.y[k] * (double)Dg[k] : 0.0;
    }
    double* rb = v.rbar + L.r_off;
    for (int s = 0; s < m; ++s) {
        const TS* zc = Zg + (long long)s * n;
        double zv[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int k = t + r * kLeafThreads;
            zv[r] = k < n ? (double)zc[k] : 0.0;
        }
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
        for (int r = 0; r < kRows; r += 4) {
            a0 = fma(zv[r], yv[r], a0);
            a1 = fma(zv[r + 1], yv[r + 1], a1);
            a2 = fma(zv[r + 2], yv[r + 2], a2);
            a3 = fma(zv[r + 3], yv[r + 3], a3);
        }
        double acc = (a0 + a1) + (a2 + a3);
#pragma unroll
        for (int o = kLeafThreads / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
        // a right-hand side sigma on this segment's interface row,
        // F - D (lambda_other - lambda_own) = sigma, acts as rbar - sigma
        if (t == 0) rb[s] = with_sadj ? acc - v.sadj[L.r_off + s] : acc;
    }}

template <int LPB, class TS>
__global__ void __launch_bounds__(kLeafThreads * LPB)
leaf_particular_kernel(DevView v, const double* __restrict__ q, const double* __restrict__ bc_val,
                       bool with_sadj) {
    __shared__ LeafSolveSmem smem[LPB];
    const int t = threadIdx.x & (kLeafThreads - 1);
    const int slot_leaf = threadIdx.x / kLeafThreads;
    const int leaf = blockIdx.x * LPB + slot_leaf;
    if (leaf >= v.nleaf) return;
    const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
    LeafSolveSmem& S = smem[slot_leaf];
    const LeafDesc L = v.leaves[leaf];
    if (L.w == kMaxLeafSide && L.h == kMaxLeafSide)
        leaf_particular_body<kMaxLeafSide * kMaxLeafSide, kMaxLeafSide, TS>(v, q, bc_val, with_sadj, S, L, t,
                                                                            mask);
    else
        leaf_particular_body<0, 0, TS>(v, q, bc_val, with_sadj, S, L, t, mask);
}

// p = A^-1 (bbar + B lambda) = L^-T D^-1 (zbar + Z lambda), written into the
// state (p_hi, p_lo) or added to it in double-double (refinement corrections).
// Body of the final solve for one leaf; NF, WF as for the particular solve.
template <int NF, int WF, class TS>
__device__ __forceinline__ void leaf_pressure_body(const DevView& v, bool accumulate, LeafSolveSmem& S,
                                                   double* lam, const LeafDesc& L, int t, unsigned mask) {
    const int w = WF ? WF : L.w, n = NF ? NF : L.w * L.h, m = L.m;
    const TS* Lg = leaf_L<TS>(v) + L.L_off;
    const TS* Dg = Lg + (long long)n * kLeafThreads;
    const TS* Zg = leaf_Z<TS>(v) + L.Z_off;
    const double* zb = v.leafzb + L.zb_off;
    for (int s = t; s < m; s += kLeafThreads) lam[s] = v.lam[L.r_off + s];
    __syncwarp(mask);
    // y = D^-1 (zbar + Z lambda), Z column-major: the lane's rows
    // k = t + 16 r accumulate together, one column at a time, so that
    // kRows independent loads are in flight per lane
    constexpr int kRows = kMaxLeafSide * kMaxLeafSide / kLeafThreads;
    double acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int k = t + r * kLeafThreads;
        acc[r] = k < n ? zb[k] : 0.0;
    }
    for (int s = 0; s < m; ++s) {
        const double ls = lam[s];
        const TS* zc = Zg + (long long)s * n;
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const int k = t + r * kLeafThreads;
            if (k < n) acc[r] = fma((double)zc[k], ls, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int k = t + r * kLeafThreads;
        if (k < n) S.y[k] = acc[r] * (double)Dg[k];
    }
    __syncwarp(mask);
    // backward sweep L^T p = y in place, right-looking from the last row,
    // reading row k of L from the column layout (L[k][k-1-t] is multiplier t
    // of column k-1-t, at Lg[16 (k-1-t) + t]: a diagonal of the layout, whose
    // lines the next steps read again from L1); the multipliers stream
    // through a register ring kSweepAhead steps ahead
    double ring[kSweepAhead];
#pragma unroll
    for (int d = 0; d < kSweepAhead; ++d) {
        const int k = n - 1 - d;
        ring[d] = (k >= 1 && t < min(w, k)) ? Lg[(long long)(k - 1 - t) * kLeafThreads + t] : 0.0;
    }
    for (int k0 = n - 1; k0 >= 0; k0 -= kSweepAhead) {
#pragma unroll
        for (int d = 0; d < kSweepAhead; ++d) {
            const int k = k0 - d;
            if (k < 0) break;
            const double lk = ring[d];
            const int kn = k - kSweepAhead;
            ring[d] = (kn >= 1 && t < min(w, kn)) ? Lg[(long long)(kn - 1 - t) * kLeafThreads + t] : 0.0;
            const double pk = S.y[k];
            if (t < min(w, k)) S.y[k - 1 - t] = fma(-lk, pk, S.y[k - 1 - t]);   // entry L[k][k-1-t]
            __syncwarp(mask);
        }
    }
    const GridDesc& G = v.grids[L.grid];
    for (int k = t; k < n; k += kLeafThreads) {
        const int i = k % w, j = k / w;
        const long long c = G.c0 + (long long)(L.j0 + j) * G.nx + L.i0 + i;
        if (accumulate) {
            const DD x = dd_add(DD{v.p_hi[c], v.p_lo[c]}, DD{S.y[k], 0.0});
            v.p_hi[c] = x.h;
            v.p_lo[c] = x.l;
        } else {
            v.p_hi[c] = S.y[k];
            v.p_lo[c] = 0.0;
        }
    }}

template <int LPB, class TS>
__global__ void __launch_bounds__(kLeafThreads * LPB)
leaf_pressure_kernel(DevView v, bool accumulate) {
    __shared__ LeafSolveSmem smem[LPB];
    __shared__ double lam_s[LPB][64];
    const int t = threadIdx.x & (kLeafThreads - 1);
    const int slot_leaf = threadIdx.x / kLeafThreads;
    const int leaf = blockIdx.x * LPB + slot_leaf;
    if (leaf >= v.nleaf) return;
    const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
    LeafSolveSmem& S = smem[slot_leaf];
    double* lam = lam_s[slot_leaf];
    const LeafDesc L = v.leaves[leaf];
    if (L.w == kMaxLeafSide && L.h == kMaxLeafSide)
        leaf_pressure_body<kMaxLeafSide * kMaxLeafSide, kMaxLeafSide, TS>(v, accumulate, S, lam, L, t, mask);
    else
        leaf_pressure_body<0, 0, TS>(v, accumulate, S, lam, L, t, mask);
}

constexpr int kRedBlocks = 256;

__global__ void mean_partial_kernel(const double* __restrict__ ph, const double* __restrict__ pl, long long n,
                                    double* red) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc += ph[i] + pl[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) red[blockIdx.x] = sh[0];
}

// Subtracts the mean of the rounded cell pressures from p and P, in
// double-double (the shift is exact up to its own rounding).
template <bool kPlain>
__global__ void mean_subtract_kernel(DevView v, long long n) {
    __shared__ double mean;
    if (threadIdx.x < 32) {
        // fixed-order warp reduction of the block partial sums: every block
        // obtains the identical mean
        double acc = 0.0;
        for (int b = threadIdx.x; b < kRedBlocks; b += 32) acc += v.red[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) mean = acc / (double)n;
    }
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (kPlain) {
        // no low parts: shift the high parts
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) v.p_hi[i] -= mean;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v.nseg; i += stride) {
            v.segP[i] -= mean;
            v.seg_lam_dd[2 * i].x -= mean;
            v.seg_lam_dd[2 * i + 1].x -= mean;
        }
        return;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const DD x = dd_add(DD{v.p_hi[i], v.p_lo[i]}, DD{-mean, 0.0});
        v.p_hi[i] = x.h;
        v.p_lo[i] = x.l;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v.nseg; i += stride) {
        const DD x = dd_add(DD{v.segP[i], v.segP_lo[i]}, DD{-mean, 0.0});
        v.segP[i] = x.h;
        v.segP_lo[i] = x.l;
        // the Robin data P -/+ beta U move with P
        for (int side = 0; side < 2; ++side) {
            const double2 l = v.seg_lam_dd[2 * i + side];
            const DD y = dd_add(DD{l.x, l.y}, DD{-mean, 0.0});
            v.seg_lam_dd[2 * i + side] = make_double2(y.h, y.l);
        }
    }
}

}  // namespace

template <class T>
static cudaError_t launch_leaf_build_t(const DevView& v, int max_m, cudaStream_t s) {
    if (max_m <= 16) {
        constexpr int LPB = 4;
        const size_t sm = sizeof(LeafBuildSmem<16, T>) * LPB;
        cudaFuncSetAttribute(leaf_build_kernel<16, LPB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        leaf_build_kernel<16, LPB, T><<<(v.nleaf + LPB - 1) / LPB, kLeafThreads * LPB, sm, s>>>(v);
    } else {
        constexpr int LPB = 2;
        const size_t sm = sizeof(LeafBuildSmem<64, T>) * LPB;
        cudaFuncSetAttribute(leaf_build_kernel<64, LPB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        leaf_build_kernel<64, LPB, T><<<(v.nleaf + LPB - 1) / LPB, kLeafThreads * LPB, sm, s>>>(v);
    }
    return cudaGetLastError();
}

cudaError_t launch_leaf_build(const DevView& v, int max_m, cudaStream_t s) {
    return v.leaf32 ? launch_leaf_build_t<float>(v, max_m, s) : launch_leaf_build_t<double>(v, max_m, s);
}

cudaError_t launch_leaf_particular(const DevView& v, const double* q, const double* bc_val,
                                   bool with_sadj, cudaStream_t s) {
    constexpr int LPB = 8;
    const int grid = (v.nleaf + LPB - 1) / LPB;
    if (v.leaf32)
        leaf_particular_kernel<LPB, float><<<grid, kLeafThreads * LPB, 0, s>>>(v, q, bc_val, with_sadj);
    else
        leaf_particular_kernel<LPB, double><<<grid, kLeafThreads * LPB, 0, s>>>(v, q, bc_val, with_sadj);
    return cudaGetLastError();
}

cudaError_t launch_leaf_pressure(const DevView& v, bool accumulate, cudaStream_t s) {
    constexpr int LPB = 8;
    const int grid = (v.nleaf + LPB - 1) / LPB;
    if (v.leaf32)
        leaf_pressure_kernel<LPB, float><<<grid, kLeafThreads * LPB, 0, s>>>(v, accumulate);
    else
        leaf_pressure_kernel<LPB, double><<<grid, kLeafThreads * LPB, 0, s>>>(v, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_mean_shift(const DevView& v, bool plain, cudaStream_t s) {
    const long long n = v.ncell;      // all-Neumann problems: single-grid contexts only
    mean_partial_kernel<<<kRedBlocks, 256, 0, s>>>(v.p_hi, v.p_lo, n, v.red);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (plain)
        mean_subtract_kernel<true><<<kRedBlocks, 256, 0, s>>>(v, n);
    else
        mean_subtract_kernel<false><<<kRedBlocks, 256, 0, s>>>(v, n);
    return cudaGetLastError();
}

}  // namespace mrcm
