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
};

// Geometry of one leaf, uploaded once by mrcm_setup.
struct LeafDesc {
    int i0, j0;        // first cell
    int w, h;          // size in cells (<= 16)
    int m;             // interface segments of the leaf
    int side_off[4];   // local index of the first segment of side x-, x+, y-,
                       // y+ (-1 when the side lies on the domain boundary)
    int seg_off;       // offset of the leaf's segment ids in leaf_segs
    long long L_off;   // band factor: n rows x 16 multipliers, then n 1/d
    long long Z_off;   // Z = L^-1 B: n rows x m
    long long zb_off;  // particular forward solve: n values
    long long R_off;   // node R (m x m) of the leaf
    long long r_off;   // node rbar / lambda (m values each, separate arrays)
    long long fs_off;  // unused
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
    long long LU_off;  // 2g x 2g LU factors (row-major, in place)
    long long piv_off; // 2g pivot rows (int)
    long long X_off;   // 2g x m coefficients X = -M^-1 C
    long long xb_off;  // 2g particular coefficients
};

// Device-side view of the plan and workspace.
struct DevView {
    int nx, ny;
    double hx, hy, alpha;
    int bc[4];
    int nleaf, nseg;
    int sx, sy, gx, gy;
    // inputs copied / derived
    const double* K;        // nx*ny
    double* seg_beta;       // nseg
    double* seg_D;          // nseg: |t| / (2 beta_t)
    double* cxL;            // (nx+1)*ny face coefficient seen from the lower cell
    double* cxU;            //            ... seen from the upper cell
    double* cyL;            // nx*(ny+1)
    double* cyU;
    // segment geometry
    const int* seg_axis; const int* seg_line; const int* seg_lo; const int* seg_len;
    const int* seg_a; const int* seg_b; const int* seg_face_off;
    // leaves and tree
    const LeafDesc* leaves;
    const int* leaf_segs;
    const MergeDesc* merges;    // all internal nodes, grouped by height
    const int* node_map;
    const int* gamma_segs;
    // workspace
    double* leafL;      // band factors
    double* leafZ;      // Z per leaf
    double* leafzb;     // particular forward solves
    double* R;          // node maps (leaves and internal nodes)
    double* rbar;       // node particular fluxes
    double* lam;        // node Robin data (top-down)
    double* LU;         // merge factors
    int* piv;
    double* X;
    double* xbar;
    double* skel;       // one-sided skeleton fluxes: 2 per skeleton face
    double* red;        // reduction scratch (mean pressure)
    int* status;        // device status word
};

// ---- launchers (return cudaGetLastError() of the launch) -----------------
cudaError_t launch_check_K(const DevView& v, cudaStream_t s);
cudaError_t launch_seg_beta(const DevView& v, cudaStream_t s);
cudaError_t launch_face_coef(const DevView& v, cudaStream_t s);
cudaError_t launch_leaf_build(const DevView& v, int max_m, cudaStream_t s);
cudaError_t launch_leaf_particular(const DevView& v, const double* q, const double* bc_val,
                                   int max_m, cudaStream_t s);
cudaError_t launch_leaf_final(const DevView& v, const double* q, const double* bc_val,
                              double* p, double* Fx, double* Fy, int max_m, cudaStream_t s);
cudaError_t launch_skeleton_fluxes(const DevView& v, double* Fx, double* Fy, double* iface,
                                   cudaStream_t s);
cudaError_t launch_mean_shift(const DevView& v, double* p, cudaStream_t s);
cudaError_t launch_merge_build(const DevView& v, int first, int count, int max_g2, int max_m,
                               cudaStream_t s);
cudaError_t launch_merge_up(const DevView& v, int first, int count, int max_g2, cudaStream_t s);
cudaError_t launch_merge_down(const DevView& v, int first, int count, int max_g2, cudaStream_t s);

}  // namespace mrcm
