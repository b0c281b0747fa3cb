// Internal declarations shared by the CUDA translation units of libmrcm.
// Not part of the public ABI (see include/mrcm.h).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace mrcm {

// Largest leaf side handled by the leaf kernels (cells).
constexpr int kMaxLeafSide = 16;
// Threads cooperating on one leaf.
constexpr int kLeafThreads = 16;
// Device status word bits (host maps them to MRCM_ERR_* codes).
enum : int {
    kStatusBadK = 1,
    kStatusSingular = 2,
    kStatusTimeout = 4,
    kStatusBadIndex = 8,
    kStatusInconsistent = 16,   // all-Neumann data violate the compatibility condition
};
// Polls of a bounded inter-CTA wait before it gives up (about a second).
constexpr long long kDefaultSpinLimit = 5000000;
// Relative tolerance of the all-Neumann compatibility condition
// |sum q - sum |e| g_N| <= kCompatTol (sum |q| + sum |e| |g_N|).
constexpr double kCompatTol = 1e-14;

// One grid of a context: a context holds one problem, or a batch of
// independent problems (realisations) whose leaves, segments and merge
// trees are planned together and whose arrays are concatenated grid after
// grid (cells x fastest within a grid; x-faces, y-faces and boundary values
// likewise).
struct GridDesc {
    int nx, ny;        // cells
    double hx, hy;     // cell size
    int bc[4];         // side types x-, x+, y-, y+ (1: Dirichlet)
    long long c0;      // first cell of the grid in the cell arrays
    long long fx0;     // first x-face ((nx+1) ny of them)
    long long fy0;     // first y-face (nx (ny+1))
    long long b0;      // first boundary value (2 (nx + ny))
};

// Geometry of one leaf, uploaded once by mrcm_setup.
struct LeafDesc {
    int i0, j0;        // first cell (within its grid)
    int w, h;          // size in cells (<= 16)
    int m;             // interface segments of the leaf
    int grid;          // the grid it belongs to
    int side_off[4];   // local index of the first segment of side x-, x+, y-,
                       // y+ (-1 when the side lies on the domain boundary)
    int seg_off;       // offset of the leaf's segment ids in leaf_segs
    long long L_off;   // band factor: n x 16 multipliers by column (step k: rows
                       // k+1..k+16), then n reciprocal pivots
    long long Z_off;   // Z = L^-1 B: n rows x m
    long long zb_off;  // particular forward solve: n values
    long long R_off;   // node R (m x m) of the leaf
    long long r_off;   // node rbar / lambda (m values each, separate arrays)
};

// A 3D grid (one problem per 3D context): arrays are x fastest, then y,
// then z.  Faces: x-faces (k ny + j)(nx + 1) + i, y-faces (k (ny + 1) + j)
// nx + i, z-faces (k ny + j) nx + i with k in [0, nz].  Boundary values per
// side x-, x+, y-, y+, z-, z+ concatenated, the x sides (nz, ny), the y
// sides (nz, nx), the z sides (ny, nx), first index slowest.
struct Grid3 {
    int nx, ny, nz;
    double hx, hy, hz;
    int bc[6];                  // side types (1: Dirichlet)
};

// Largest leaf block of the 3D path (cells) and its segment count: a
// seg_x x seg_y x seg_z block of at most 64 cells, at most 16 faces per side.
constexpr int kLeaf3Cells = 64;
constexpr int kLeaf3Segs = 96;

// One 3D leaf block.  The blocks tile the grid with the interface patch shape,
// so a patch between two subdomains is the whole shared side of two blocks;
// inside a subdomain every face between two blocks is a segment of its own
// (a fine-face interface, on which the Robin coupling is exact for any beta).
struct LeafDesc3 {
    int i0, j0, k0;             // first cell
    int w[3];                   // cells per axis
    int m;                      // segments of the block
    int seg_off;                // offset of its segment ids in leaf_segs
    int side_off[6];            // local index of the first segment of side x-, x+,
                                // y-, y+, z-, z+ (-1: the side is on the domain boundary)
    int side_fine[6];           // 1: one segment per face; 0: one patch for the side
    long long L_off;            // n x n: L below the diagonal (row-major), 1/d on it
    long long Z_off;            // Z = L^-1 B: m columns of n
    long long zb_off;           // particular forward solve: n values
    long long R_off, r_off;     // node R (m x m) and rbar / lambda (m)
};

// One internal tree node (a merge of two children).
struct MergeDesc {
    int node;          // node id
    int c1, c2;        // children node ids (c1: lower half = side a of gamma)
    int g;             // gamma segments
    int m;             // outer segments of the node (= o1 + o2)
    int o1;            // outer segments inherited from c1
    int m1, m2;        // children's segment counts
    int map_off;       // gpos1[g], gpos2[g], opos1[o1], opos2[m-o1] in node_map
    int gamma_off;     // global ids of the gamma segments in gamma_segs
    int pinned;        // 1: root of an all-Neumann problem (P of gamma[0] = 0)
    long long R_off, R1_off, R2_off;   // node / children R
    long long r_off, r1_off, r2_off;   // node / children rbar (and lambda)
    long long W_off;   // 2g x 2g inverse W = M^-1 (column-major), or the factor of
                       // a factor-form root level
    long long X_off;   // 2g x m coefficients X = -M^-1 C (column-major)
};

// Device-side view of the plan and workspace.
struct DevView {
    double alpha;
    long long ncell, nxface, nyface, nbc;   // totals over the grids
    int ngrid;
    const GridDesc* grids;
    int nleaf, nseg;
    int sx, sy, gx, gy;
    // inputs copied / derived
    const double* K;        // ncell
    double* rx;             // nx*ny half-cell resistances hx / (2 K)
    double* ry;             //                               hy / (2 K)
    double* seg_beta;       // nseg
    double* seg_D;          // nseg: |t| / (2 beta_t)
    double* cxL;            // (nx+1)*ny face coefficient seen from the lower cell
    double* cxU;            //            ... seen from the upper cell
    double* cyL;            // nx*(ny+1)
    double* cyU;
    // segment geometry
    const int* seg_axis; const int* seg_line; const int* seg_lo; const int* seg_len;
    const int* seg_a; const int* seg_b; const int* seg_face_off;
    const int* seg_grid;          // grid of each segment (line and lo are grid-local)
    const long long* seg_lam_a;   // offset in lam of segment t in the leaf on side a
    const long long* seg_lam_b;   //                                   ... side b
    const int* xface_seg;         // (nx+1)*ny: segment of each x-face, -1 off the skeleton
    const int* yface_seg;         // nx*(ny+1): segment of each y-face
    double2* seg_lam_dd;          // per segment: Robin data of side a, of side b
                                  // (P -/+ beta U of the refined state, double-double)
    // leaves and tree
    const LeafDesc* leaves;
    const int* leaf_segs;
    const MergeDesc* merges;    // all internal nodes, grouped by height
    const int* node_map;
    const int* gamma_segs;
    // workspace
    double* leafL;      // band factors
    double* leafZ;      // Z per leaf
    float* leafL32;     // the same in FP32 (mixed precision: leaf work in FP32)
    float* leafZ32;
    int mixed;          // 1: the mixed form (the merges of FP32 levels in FP32)
    int leaf32;         // 1: leaf factors in FP32 (mixed form, mrcm_set_mixed_leaves)
    int res_dd;         // 1: refinement residuals in double-double, 0: in FP64 (mrcm_set_residual)
    double* leafzb;     // particular forward solves
    double* R;          // node maps (leaves and internal nodes)
    double* rbar;       // node particular fluxes
    double* rgam;       // per merge, rbar of its 2g gamma unknowns gathered from
                        // the children (at 2 * gamma_off), written by the up sweep
    double* lam;        // node Robin data (top-down)
    double* fwd;        // per merge of a factor-form root level (2g at 2 * gamma_off):
                        // y = Lt^-1 rhat of the up sweep
    unsigned int* tri_flags;   // block flags of the factor form's triangular sweeps:
    long long tri_flag_n;      // tri_flag_n for the forward sweep, then as many backward
    double* X;
    double* W;          // per merge (W_off layout): the explicit inverse of the
                        // interface matrix, or for a factor-form root level its
                        // block LDL^T factor (Lt below the diagonal blocks, their
                        // inverses in them; on and below the diagonal)
    float* W32;         // FP32 work array of the mixed form's blocked levels (W_off layout)
    double* segP;       // refined interface unknowns P_t, U_t (high parts)
    double* segU;
    double* segP_lo;    // ... and low parts of the double-double state
    double* segU_lo;
    double* p_hi;       // refined cell pressures, double-double
    double* p_lo;
    double* rcell;      // cell residuals (refinement)
    double* sadj;       // per leaf segment: right-hand side of its interface row
    double* red;        // reduction scratch (mean pressure)
    unsigned long long* res_max;  // max |residual| per refinement step (double bits)
    int* status;        // device status word
    long long spin_limit;         // polls of a bounded inter-CTA wait (mrcm_set_wait_limit)
    // 3D contexts (dim == 3): the grid, the blocks, the z-faces and the second
    // tangential extent of each segment (seg_lo / seg_len hold the first)
    int dim;
    Grid3 g3;
    long long nzface;
    const LeafDesc3* leaves3;
    const int* zface_seg;         // segment of each z-face, -1 off the skeleton
    const int* seg_lo2;
    const int* seg_len2;
    double* czL;                  // z-face coefficients seen from the lower / upper cell
    double* czU;
};

#ifdef __CUDACC__
// The grid holding entry x of the concatenated cell (KIND 0), x-face (1) or
// y-face (2) arrays: binary search over the grids' first entries (one grid:
// no search).
template <int KIND>
__device__ __forceinline__ int grid_of(const DevView& v, long long x) {
    int lo = 0, hi = v.ngrid - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const GridDesc& G = v.grids[mid];
        const long long o = KIND == 0 ? G.c0 : (KIND == 1 ? G.fx0 : G.fy0);
        if (o <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Double-double arithmetic: TwoSum (Knuth) and FMA-based TwoProd are
// error-free; a value is the unevaluated sum h + l with |l| <= ulp(h)/2.
struct DD {
    double h, l;
};
__device__ __forceinline__ DD dd_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DD dd_two_prod(double a, double b) {
    const double p = __dmul_rn(a, b);
    return {p, __fma_rn(a, b, -p)};
}
__device__ __forceinline__ DD dd_add(DD x, DD y) {
    const DD s = dd_two_sum(x.h, y.h);
    return dd_two_sum(s.h, __dadd_rn(s.l, __dadd_rn(x.l, y.l)));
}
__device__ __forceinline__ DD dd_mul_d(DD x, double b) {
    const DD p = dd_two_prod(x.h, b);
    return dd_two_sum(p.h, __fma_rn(x.l, b, p.l));
}
__device__ __forceinline__ DD dd_neg(DD x) { return {-x.h, -x.l}; }

// Reciprocal from a single-precision seed refined by one third-order step of
// the Newton-Raphson family (Muller et al., Handbook of Floating-Point
// Arithmetic, Sec. 5.3): with x the seed and e = 1 - p x, 1/p = x / (1 - e) =
// x (1 + e + e^2 + ...), and the series is cut after e^2.  The seed is the
// approximate FP32 reciprocal (at most 1 ulp off) of p's sign, exponent and
// leading 23 mantissa bits, moved between formats with integer operations
// (conversion instructions run on the slower FP64 path), so |e| < 2^-21.9 and
// the dropped terms are below 2^-65 relative: the result is within an ulp of
// 1/p.  Three dependent FP64 instructions (e, e + e^2, x + x (e + e^2))
// instead of the longer IEEE division sequence, which matters where a
// reciprocal sits on a sequential chain (pivots).  Outside the exponent range
// of FP32 it falls back to the division.
__device__ __forceinline__ double rcp_nr(double p) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(p);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    if (e < -120 || e > 120) return 1.0 / p;
    const unsigned int fb = (unsigned int)(bits >> 32 & 0x80000000u) | ((unsigned int)(e + 127) << 23) |
                            (unsigned int)(bits >> 29 & 0x7fffffu);
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(fb)));
    const unsigned int rb = __float_as_uint(rf);
    const int er = (int)((rb >> 23) & 0xff) - 127;
    const unsigned long long xb = ((unsigned long long)(rb & 0x80000000u) << 32) |
                                  ((unsigned long long)(er + 1023) << 52) | ((unsigned long long)(rb & 0x7fffffu) << 29);
    const double x = __longlong_as_double((long long)xb);
    const double e0 = fma(-p, x, 1.0);
    const double s = fma(e0, e0, e0);
    return fma(x, s, x);
}
// Quotient and remainder of a non-negative index by a positive divisor in
// 32-bit unsigned arithmetic (every index of the workspace is below 2^32;
// a 64-bit division is a long emulated sequence).
__device__ __forceinline__ void udivmod(long long x, int d, int& q, int& r) {
    const unsigned ux = (unsigned)x, ud = (unsigned)d;
    const unsigned uq = ux / ud;
    q = (int)uq;
    r = (int)(ux - uq * ud);
}
// -x by flipping the sign bit: an FP64 negation that is not an FMA operand
// modifier (inside a select, say) costs a full FP64 instruction.
__device__ __forceinline__ double neg_bits(double x) {
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000u, __double2loint(x));
}
__device__ __forceinline__ double dd_round(DD x) { return __dadd_rn(x.h, x.l); }
// FP32 counterparts used by the mixed-precision instantiations of the leaf
// and merge kernels: the IEEE reciprocal (a single instruction in FP32) and
// the sign flip on the bit pattern.
__device__ __forceinline__ float rcp_nr(float p) { return __frcp_rn(p); }
__device__ __forceinline__ float neg_bits(float x) { return __int_as_float(__float_as_int(x) ^ (int)0x80000000u); }
// positive and finite, tested on the bit pattern
__device__ __forceinline__ bool positive_finite_bits(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool positive_finite_bits(float x) {
    const int b = __float_as_int(x);
    return b > 0 && b < 0x7f800000;
}
// L2-only loads for either precision
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
// the leaf factor arrays of either precision
template <class T> __device__ __forceinline__ T* leaf_L(const DevView& v);
template <> __device__ __forceinline__ double* leaf_L<double>(const DevView& v) { return v.leafL; }
template <> __device__ __forceinline__ float* leaf_L<float>(const DevView& v) { return v.leafL32; }
template <class T> __device__ __forceinline__ T* leaf_Z(const DevView& v);
template <> __device__ __forceinline__ double* leaf_Z<double>(const DevView& v) { return v.leafZ; }
template <> __device__ __forceinline__ float* leaf_Z<float>(const DevView& v) { return v.leafZ32; }
#endif

// MRCM_OK for cudaSuccess; otherwise records e as the calling thread's last
// CUDA error (mrcm_last_cuda_error) and returns MRCM_ERR_OOM or
// MRCM_ERR_CUDA.
int cuda_status(cudaError_t e);

// ---- launchers (return cudaGetLastError() of the launch) -----------------
cudaError_t launch_check_K(const DevView& v, cudaStream_t s);
// r[i] = rcp_nr(x[i]) (self-check of the kernels' reciprocal)
cudaError_t launch_reciprocal(const double* x, double* r, long long n, cudaStream_t s);
cudaError_t launch_cell_resist(const DevView& v, cudaStream_t s);
cudaError_t launch_seg_beta(const DevView& v, cudaStream_t s);
cudaError_t launch_face_coef(const DevView& v, cudaStream_t s);
cudaError_t launch_leaf_build(const DevView& v, int max_m, cudaStream_t s);
// particular solve: q and bc_val are the data; bc_val == nullptr means zero
// external data; with_sadj subtracts the interface right-hand sides.
cudaError_t launch_leaf_particular(const DevView& v, const double* q, const double* bc_val,
                                   bool with_sadj, cudaStream_t s);
// p = A^-1 (bbar + B lambda) per leaf into the double-double state
// (p_hi, p_lo): set, or accumulate (double-double add of the correction).
cudaError_t launch_leaf_pressure(const DevView& v, bool accumulate, cudaStream_t s);
// interface unknowns from the two Robin data of each segment (set or add)
cudaError_t launch_lam_to_PU(const DevView& v, bool accumulate, cudaStream_t s);
// residual of the discrete equations in double-double; fills rcell, sadj
cudaError_t launch_residual(const DevView& v, const double* q, const double* bc_val, int step,
                            cudaStream_t s);
// cell pressures and face fluxes from the double-double state; iface
// optional; plain: the state has no low parts (no refinement step ran), the
// fluxes are formed in plain FP64
cudaError_t launch_face_fluxes(const DevView& v, const double* bc_val, double* p, double* Fx,
                               double* Fy, double* iface, bool plain, cudaStream_t s);
// Learned basis surrogate (kernels_surrogate.cu): leaf lists are device
// arrays of leaf ids (each checked; leaves with more than 16 segments are
// refused); fields are float [item][16][256], patches bf16 [item][18][18][16].
// The 3D path (kernels_3d.cu): coefficients, the leaf blocks' local Robin
// problems, their solve-phase passes and the face fluxes.
cudaError_t launch_coef3(const DevView& v, cudaStream_t s);
cudaError_t launch_leaf3_build(const DevView& v, cudaStream_t s);
cudaError_t launch_leaf3_particular(const DevView& v, const double* q, const double* bc_val, bool with_sadj,
                                    cudaStream_t s);
cudaError_t launch_leaf3_pressure(const DevView& v, bool accumulate, cudaStream_t s);
cudaError_t launch_residual3(const DevView& v, const double* q, const double* bc_val, int step, cudaStream_t s);
cudaError_t launch_face_fluxes3(const DevView& v, const double* bc_val, double* p, double* Fx, double* Fy,
                                double* Fz, double* iface, cudaStream_t s);
cudaError_t launch_leaf_fields(const DevView& v, const int* ids, int count, float* psi, cudaStream_t s);
cudaError_t launch_leaf_patches(const DevView& v, const int* ids, int count, void* x, cudaStream_t s);
cudaError_t launch_leaf_gate(const DevView& v, const int* ids, int count, const float* psi, double* res,
                             cudaStream_t s);
cudaError_t launch_leaf_apply(const DevView& v, const int* ids, int count, const float* psi, const double* res,
                              double tau, int* accepted, cudaStream_t s);
cudaError_t launch_conv_fwd(const void* x, int count, int cin, int cout, int pad, int relu, const void* w,
                            const float* b, void* ybf, float* yf, cudaStream_t s);
cudaError_t launch_conv_wgrad(const void* x, const void* dy, int count, int cin, int cout, int pad, float* dw,
                              float* db, cudaStream_t s);
cudaError_t launch_flip_weights(const void* w, int cout, int cin, void* w2, cudaStream_t s);
cudaError_t launch_relu_grad(const float* dpost, const void* y, long long n, int mask, void* dpre, cudaStream_t s);
cudaError_t launch_mse_grad(const float* pred, const float* target, int count, float* dpred, float* loss,
                            cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, void* pbf, long long n, float lr, float b1,
                        float b2, float eps, int t, cudaStream_t s);
// all-Neumann data: sets kStatusInconsistent unless the sources balance the
// boundary outflow to kCompatTol (double-double sums; scratch in v.red)
cudaError_t launch_compat_check(const DevView& v, const double* q, const double* bc_val, cudaStream_t s);
// zero-mean shift of the state's p and P (all-Neumann problems); plain as
// above (the shift is applied to the high parts only)
cudaError_t launch_mean_shift(const DevView& v, bool plain, cudaStream_t s);
// Brackets each launch group of a phase (the phase ids of include/mrcm.h).
struct PhaseHook {
    void* ctx;
    void (*begin)(void* ctx, int phase);
    void (*end)(void* ctx, int phase);
};
// one tree height of merges; scratch: merge_scratch_doubles(count, max_g2,
// max_m) values; barrier: kMergeBarrierBytes of device memory (reset by the
// call); *launches is increased by the number of kernels launched
// Launch shapes of one blocked merge level (0 everywhere: the built-in
// heuristic).  sweep_per_sm: CTAs per SM of the cooperative sweep (1-4);
// x_rows: rows of X per CTA (32, 64); r_tile: side of an R tile (16, 32).
struct MergeTune {
    int sweep_per_sm = 0, x_rows = 0, r_tile = 0;
};
// fp32: the mixed form's FP32 arithmetic for this level (T of the blocked
// sweep in v.W32; W, X and R stored in double either way).  factor: a
// blocked level without outer segments (a root level) keeps the block
// LDL^T factor of its interface system instead of the inverse.
cudaError_t launch_merge_build(const DevView& v, int first, int count, int max_g2, int max_m, bool fp32,
                               bool factor, const MergeTune& tune, double* scratch, void* barrier, cudaStream_t s,
                               int* launches, const PhaseHook& hook);
// Times every launch shape of one blocked level (its children's maps must
// be built: the launches are repeated and recompute the same numbers) and
// returns the fastest per launch; `reps` timed runs each.
cudaError_t tune_merge_level(const DevView& v, int first, int count, int max_g2, int max_m, bool fp32, bool factor,
                             double* scratch, void* barrier, cudaStream_t s, int reps, MergeTune* out);
constexpr size_t kMergeBarrierBytes = 64;
bool merge_level_blocked(int count, int max_g2, int max_m);
size_t merge_scratch_doubles(int count, int max_g2, int max_m);
constexpr int kMergeBlock = 16;      // block size of the blocked Gauss-Jordan sweep (flop model)
constexpr int kTriBlock = 64;        // solve blocks of the factor form's triangular sweeps
// MRCM_ROOT_AUTO factors root systems from this 2g on: below it the root's
// elimination is bound by its sequential chain of pivot blocks (the same
// length in both forms), and the inverse's solve passes are the shorter.
constexpr int kRootFactorMinG2 = 1024;

// The merge levels of the tree for the fused up / down sweeps of the solve
// (passed by value as a kernel argument; index h - 1 for height h).
constexpr int kMaxTreeLevels = 48;
struct TreeLevels {
    int height;
    int first[kMaxTreeLevels], count[kMaxTreeLevels], g2[kMaxTreeLevels], m[kMaxTreeLevels];
    int nkc[kMaxTreeLevels];   // down sweep: term chunks per row, a power of two (1: no partial sums)
    int kcl[kMaxTreeLevels];   // down sweep: terms per chunk (a multiple of 8)
    int form[kMaxTreeLevels];  // 1: a root level in the factor form (block triangular sweeps)
    // extents of the static data the sweeps read (prefetched into L2)
    long long x_len, w_len;    // doubles of X and W
    long long n_merges, map_len;
};
// Grid of the fused tree sweeps on the current device (CTAs of 256 threads).
cudaError_t tree_grid(int* grid);
// Fills nkc for a grid of `grid` CTAs; returns the scratch doubles the down
// sweep needs (partial sums of the levels with nkc > 1).
long long tree_plan_chunks(TreeLevels& L, int grid);
// rbar of every merge, leaves' parents to the root, in one cooperative
// launch (grid barrier on `barrier` between heights).
cudaError_t launch_tree_up(const DevView& v, const TreeLevels& L, int grid, void* barrier, cudaStream_t s);
// lambda of every merge's gamma, root to the leaves' parents, in one
// cooperative launch; scratch: tree_plan_chunks doubles.
cudaError_t launch_tree_down(const DevView& v, const TreeLevels& L, int grid, double* scratch, void* barrier,
                             cudaStream_t s);

}  // namespace mrcm
