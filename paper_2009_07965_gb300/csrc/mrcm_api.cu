// libmrcm: C ABI, planning of the decomposition and launch orchestration.
//
// Host side of the Recursive MRCM (arXiv 2009.07965): leaves and interface
// segments (Section 2, Eqs. decomp.1-2; Section 4, intermediate scale
// H-bar), the binary hierarchy of Section 3.1 (Eqs. dd.l, dd.2, interface.1)
// and the order of the batched kernel launches that carry out Algorithm 1.
// All arithmetic on problem data happens in the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <map>
#include <unordered_map>
#include <vector>

#include "mrcm_internal.h"
#include "../../include/mrcm.h"

using namespace mrcm;

namespace {

constexpr int kMaxRefine = 16;

struct Plan {
    double alpha = 0;
    int sx = 0, sy = 0, gx = 0, gy = 0;
    // the grids (one problem, or a batch of independent realisations)
    std::vector<GridDesc> grids;
    std::vector<int> grid_Nlx, grid_Nly, grid_leaf0;   // leaf grid and first leaf of each grid
    long long ncell = 0, nxface = 0, nyface = 0, nbc = 0;
    bool pure_neumann = false;           // a single grid with no Dirichlet side
    int nleaf = 0;
    std::vector<LeafDesc> leaves;
    std::vector<int> leaf_segs;
    // segments
    std::vector<int> seg_axis, seg_line, seg_lo, seg_len, seg_a, seg_b, seg_face_off, seg_grid;
    int nseg = 0;
    long long nskel_faces = 0;
    std::vector<int> xface_seg, yface_seg;   // segment of each x- / y-face, -1 off the skeleton
    // tree (nodes 0..nleaf-1 are the leaves)
    struct Node {
        int box[4];
        int height = 0, c1 = -1, c2 = -1, parent = -1, leaf = -1;
        std::vector<int> segs;   // outer segments in R order
        std::vector<int> gamma;  // gamma segments (internal nodes)
        std::vector<int> map;    // gpos1, gpos2, opos1, opos2
        int o1 = 0;
    };
    std::vector<Node> nodes;
    std::vector<int> roots;              // one per grid
    std::vector<char> root_pinned;       // per node: root of an all-Neumann problem
    int height = 0;
    std::vector<MergeDesc> merges;       // grouped by height (ascending)
    std::vector<int> level_first, level_count, level_max_g2, level_max_m;  // index by height-1
    std::vector<int> node_map, gamma_segs;
    int max_m_leaf = 0, max_g2 = 0;
    // storage sizes (doubles / ints)
    long long nR = 0, nr = 0, nW = 0, nX = 0, nL = 0, nZ = 0, nzb = 0;
    std::vector<long long> node_R_off, node_r_off;
    std::vector<long long> seg_lam_a, seg_lam_b;   // lam offsets of each segment in its two leaves
    // flop model
    long long leaf_flops = 0, merge_flops = 0, solve_flops = 0;
    // reference flop model of a direct method (LU-based merges, banded
    // Cholesky leaves): the roofline numerator independent of this
    // implementation's choices
    double model_build = 0, model_sweep = 0;
    double phase_build[MRCM_PHASE_COUNT] = {};   // per build call
    double phase_pass[MRCM_PHASE_COUNT] = {};    // per solve pass
    // the above count root levels in the inverse form; where a root level
    // takes the factor form these differences are added: [0] every root
    // level (MRCM_ROOT_FACTOR), [1] the levels MRCM_ROOT_AUTO factors
    double root_build[2][MRCM_PHASE_COUNT] = {}, root_pass[2][MRCM_PHASE_COUNT] = {};
    double root_merge[2] = {}, root_solve[2] = {}, root_model_sweep[2] = {};
    double residual_flops = 0, finish_flops = 0;
    // 3D contexts: the grid, the blocks (leaves), the second tangential
    // extent of each segment and the z-face map
    int dim = 2;
    Grid3 g3{};
    int sz = 0, gz = 0;
    std::vector<LeafDesc3> leaves3;
    std::vector<int> seg_lo2, seg_len2, zface_seg;
    long long nzface = 0;
};

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// A tree node merging c1 and c2 (c1 on side a of every gamma segment): gamma =
// the segments the two share; the node's outer segments are c1's others,
// then c2's, and the node map records where each sits in the children.
int add_merge_node(Plan& P, int c1, int c2, const int box[4]) {
    Plan::Node nd;
    for (int k = 0; k < 4; ++k) nd.box[k] = box[k];
    nd.c1 = c1; nd.c2 = c2;
    nd.height = 1 + std::max(P.nodes[c1].height, P.nodes[c2].height);
    const std::vector<int>& s1 = P.nodes[c1].segs;
    const std::vector<int>& s2 = P.nodes[c2].segs;
    std::unordered_map<int, int> pos2;
    for (int k = 0; k < (int)s2.size(); ++k) pos2[s2[k]] = k;
    std::vector<int> gpos1, gpos2, opos1, opos2;
    std::vector<char> in_gamma2(s2.size(), 0);
    for (int k = 0; k < (int)s1.size(); ++k) {
        auto it = pos2.find(s1[k]);
        if (it != pos2.end()) {
            nd.gamma.push_back(s1[k]);
            gpos1.push_back(k);
            gpos2.push_back(it->second);
            in_gamma2[it->second] = 1;
        } else {
            opos1.push_back(k);
            nd.segs.push_back(s1[k]);
        }
    }
    nd.o1 = (int)opos1.size();
    for (int k = 0; k < (int)s2.size(); ++k)
        if (!in_gamma2[k]) { opos2.push_back(k); nd.segs.push_back(s2[k]); }
    nd.map = gpos1;
    nd.map.insert(nd.map.end(), gpos2.begin(), gpos2.end());
    nd.map.insert(nd.map.end(), opos1.begin(), opos1.end());
    nd.map.insert(nd.map.end(), opos2.begin(), opos2.end());
    const int id = (int)P.nodes.size();
    P.nodes.push_back(nd);
    P.nodes[c1].parent = id;
    P.nodes[c2].parent = id;
    return id;
}

// Root pins and the storage offsets of every node's R and rbar.
void finish_tree(Plan& P) {
    P.root_pinned.assign(P.nodes.size(), 0);
    if (P.pure_neumann) P.root_pinned[P.roots[0]] = 1;
    const int nnode = (int)P.nodes.size();
    P.node_R_off.resize(nnode);
    P.node_r_off.resize(nnode);
    for (int v = 0; v < nnode; ++v) {
        const long long m = (long long)P.nodes[v].segs.size();
        P.node_R_off[v] = P.nR;
        P.nR += m * m;
        P.node_r_off[v] = P.nr;
        P.nr += m;
    }
}

void finish_merges(Plan& P);

int make_plan(Plan& P) {
    const int ngrid = (int)P.grids.size();
    // per grid: leaf grid, offsets in the concatenated arrays
    P.grid_Nlx.resize(ngrid);
    P.grid_Nly.resize(ngrid);
    P.grid_leaf0.resize(ngrid);
    P.ncell = P.nxface = P.nyface = P.nbc = 0;
    P.nleaf = 0;
    for (int gi = 0; gi < ngrid; ++gi) {
        GridDesc& G = P.grids[gi];
        G.c0 = P.ncell;
        G.fx0 = P.nxface;
        G.fy0 = P.nyface;
        G.b0 = P.nbc;
        P.ncell += (long long)G.nx * G.ny;
        P.nxface += (long long)(G.nx + 1) * G.ny;
        P.nyface += (long long)G.nx * (G.ny + 1);
        P.nbc += 2LL * (G.nx + G.ny);
        P.grid_Nlx[gi] = ceil_div(G.nx, P.sx);
        P.grid_Nly[gi] = ceil_div(G.ny, P.sy);
        P.grid_leaf0[gi] = P.nleaf;
        P.nleaf += P.grid_Nlx[gi] * P.grid_Nly[gi];
    }
    P.pure_neumann = ngrid == 1 && !(P.grids[0].bc[0] || P.grids[0].bc[1] || P.grids[0].bc[2] || P.grids[0].bc[3]);
    P.leaves.resize(P.nleaf);
    std::vector<int> leaf_grid(P.nleaf);
    std::vector<int> xplus_first(P.nleaf, -1), yplus_first(P.nleaf, -1);
    // leaves and the segments on their + sides, grid by grid (segment
    // lines and positions are grid-local)
    for (int gi = 0; gi < ngrid; ++gi) {
        const GridDesc& G = P.grids[gi];
        const int Nlx = P.grid_Nlx[gi], Nly = P.grid_Nly[gi], l0 = P.grid_leaf0[gi];
        for (int J = 0; J < Nly; ++J)
            for (int I = 0; I < Nlx; ++I) {
                const int id = l0 + I + Nlx * J;
                LeafDesc& L = P.leaves[id];
                std::memset(&L, 0, sizeof(L));
                L.i0 = I * P.sx;
                L.j0 = J * P.sy;
                L.w = std::min(P.sx, G.nx - L.i0);
                L.h = std::min(P.sy, G.ny - L.j0);
                L.grid = gi;
                leaf_grid[id] = gi;
            }
        for (int J = 0; J < Nly; ++J)
            for (int I = 0; I < Nlx; ++I) {
                const int id = l0 + I + Nlx * J;
                const LeafDesc& L = P.leaves[id];
                if (I + 1 < Nlx) {
                    xplus_first[id] = P.nseg;
                    for (int lo = 0; lo < L.h; lo += P.gy) {
                        P.seg_axis.push_back(0);
                        P.seg_line.push_back(L.i0 + L.w);
                        P.seg_lo.push_back(L.j0 + lo);
                        P.seg_len.push_back(std::min(P.gy, L.h - lo));
                        P.seg_a.push_back(id);
                        P.seg_b.push_back(id + 1);
                        P.seg_grid.push_back(gi);
                        ++P.nseg;
                    }
                }
                if (J + 1 < Nly) {
                    yplus_first[id] = P.nseg;
                    for (int lo = 0; lo < L.w; lo += P.gx) {
                        P.seg_axis.push_back(1);
                        P.seg_line.push_back(L.j0 + L.h);
                        P.seg_lo.push_back(L.i0 + lo);
                        P.seg_len.push_back(std::min(P.gx, L.w - lo));
                        P.seg_a.push_back(id);
                        P.seg_b.push_back(id + Nlx);
                        P.seg_grid.push_back(gi);
                        ++P.nseg;
                    }
                }
            }
    }
    P.seg_face_off.resize(P.nseg + 1);
    P.seg_face_off[0] = 0;
    for (int t = 0; t < P.nseg; ++t) P.seg_face_off[t + 1] = P.seg_face_off[t] + P.seg_len[t];
    P.nskel_faces = P.seg_face_off[P.nseg];
    P.xface_seg.assign((size_t)P.nxface, -1);
    P.yface_seg.assign((size_t)P.nyface, -1);
    for (int t = 0; t < P.nseg; ++t) {
        const GridDesc& G = P.grids[P.seg_grid[t]];
        for (int e = 0; e < P.seg_len[t]; ++e) {
            const int k = P.seg_lo[t] + e;
            if (P.seg_axis[t] == 0)
                P.xface_seg[(size_t)G.fx0 + (size_t)P.seg_line[t] + (size_t)(G.nx + 1) * k] = t;
            else
                P.yface_seg[(size_t)G.fy0 + (size_t)k + (size_t)G.nx * P.seg_line[t]] = t;
        }
    }
    // leaf segment lists: x-, x+, y-, y+ sides
    for (int id = 0; id < P.nleaf; ++id) {
        const int gi = leaf_grid[id], Nlx = P.grid_Nlx[gi], local = id - P.grid_leaf0[gi];
        const int I = local % Nlx, J = local / Nlx;
        LeafDesc& L = P.leaves[id];
        L.seg_off = (int)P.leaf_segs.size();
        const int nx_side = ceil_div(L.h, P.gy), ny_side = ceil_div(L.w, P.gx);
        int cnt = 0;
        auto add_side = [&](int s, int first, int count) {
            if (first < 0) { L.side_off[s] = -1; return; }
            L.side_off[s] = cnt;
            for (int k = 0; k < count; ++k) P.leaf_segs.push_back(first + k);
            cnt += count;
        };
        add_side(0, I > 0 ? xplus_first[id - 1] : -1, nx_side);
        add_side(1, xplus_first[id], nx_side);
        add_side(2, J > 0 ? yplus_first[id - Nlx] : -1, ny_side);
        add_side(3, yplus_first[id], ny_side);
        L.m = cnt;
        P.max_m_leaf = std::max(P.max_m_leaf, cnt);
    }
    // one tree per grid, by recursive bisection of its leaf box
    P.nodes.resize(P.nleaf);
    for (int id = 0; id < P.nleaf; ++id) {
        Plan::Node& nd = P.nodes[id];
        const int gi = leaf_grid[id], Nlx = P.grid_Nlx[gi], local = id - P.grid_leaf0[gi];
        const int I = local % Nlx, J = local / Nlx;
        nd.box[0] = I; nd.box[1] = I + 1; nd.box[2] = J; nd.box[3] = J + 1;
        nd.leaf = id;
        const LeafDesc& L = P.leaves[id];
        nd.segs.assign(P.leaf_segs.begin() + L.seg_off, P.leaf_segs.begin() + L.seg_off + L.m);
    }
    struct Rec {
        Plan& P;
        int l0, Nlx;
        int build(int I0, int I1, int J0, int J1) {
            const int nxl = I1 - I0, nyl = J1 - J0;
            if (nxl == 1 && nyl == 1) return l0 + I0 + Nlx * J0;
            int c1, c2;
            if (nxl >= nyl) {
                const int mid = I0 + (nxl + 1) / 2;
                c1 = build(I0, mid, J0, J1);
                c2 = build(mid, I1, J0, J1);
            } else {
                const int mid = J0 + (nyl + 1) / 2;
                c1 = build(I0, I1, J0, mid);
                c2 = build(I0, I1, mid, J1);
            }
            const int box[4] = {I0, I1, J0, J1};
            return add_merge_node(P, c1, c2, box);
        }
    };
    P.height = 0;
    P.roots.clear();
    for (int gi = 0; gi < ngrid; ++gi) {
        Rec rec{P, P.grid_leaf0[gi], P.grid_Nlx[gi]};
        const int root = rec.build(0, P.grid_Nlx[gi], 0, P.grid_Nly[gi]);
        P.roots.push_back(root);
        P.height = std::max(P.height, P.nodes[root].height);
    }
    finish_tree(P);
    for (int id = 0; id < P.nleaf; ++id) {
        LeafDesc& L = P.leaves[id];
        const long long n = (long long)L.w * L.h;
        L.L_off = P.nL;
        P.nL += n * (kLeafThreads + 1);
        L.Z_off = P.nZ;
        P.nZ += n * L.m;
        L.zb_off = P.nzb;
        P.nzb += n;
        L.R_off = P.node_R_off[id];
        L.r_off = P.node_r_off[id];
        // flop model of the leaf kernel: LDL^T band steps, forward solve of
        // the Robin columns from their first nonzero row on, SYRK of the
        // lower triangle of the active columns (FMA = 2 flops)
        std::vector<int> starts;
        for (int s = 0; s < L.m; ++s) {
            int st;
            if (L.side_off[3] >= 0 && s >= L.side_off[3]) st = (L.h - 1) * L.w + (s - L.side_off[3]) * P.gx;
            else if (L.side_off[2] >= 0 && s >= L.side_off[2]) st = (s - L.side_off[2]) * P.gx;
            else if (L.side_off[1] >= 0 && s >= L.side_off[1]) st = (s - L.side_off[1]) * P.gy * L.w + L.w - 1;
            else st = (s - L.side_off[0]) * P.gy * L.w;
            starts.push_back(st);
        }
        std::sort(starts.begin(), starts.end());
        long long f = 0;
        int ck = 0;
        for (long long k = 0; k < n; ++k) {
            while (ck < L.m && starts[ck] <= k) ++ck;
            const long long wk = std::min<long long>(L.w, n - 1 - k);
            f += wk + wk * (wk + 1);                  // multipliers + trailing update
            f += 2 * wk * ck;                         // Z update
            f += ck + (long long)ck * (ck + 1);       // scaling + R update
        }
        P.leaf_flops += f;
        {
            const double nn = (double)n, b = (double)L.w, mm = (double)L.m;
            P.model_build += nn * b * b + 2.0 * nn * b * mm + mm * (mm + 1.0) * nn + 4.0 * nn * b;
        }
        // solve phase per leaf: forward sweep, Z^T y, Z lambda, backward sweep
        P.solve_flops += 2 * n * L.w * 2 + 2 * n * L.m * 2 + 2 * n;
        P.phase_pass[MRCM_PHASE_LEAF_PART] += 2.0 * n * L.w + 2.0 * n * L.m + n;
        P.phase_pass[MRCM_PHASE_LEAF_PRESSURE] += 2.0 * n * L.m + 2.0 * n * L.w + 2.0 * n;
    }
    // offsets of each segment inside the Robin-data arrays of its two leaves
    P.seg_lam_a.assign(P.nseg, -1);
    P.seg_lam_b.assign(P.nseg, -1);
    for (int id = 0; id < P.nleaf; ++id) {
        const LeafDesc& L = P.leaves[id];
        for (int k = 0; k < L.m; ++k) {
            const int t = P.leaf_segs[L.seg_off + k];
            if (P.seg_a[t] == id) P.seg_lam_a[t] = L.r_off + k;
            else P.seg_lam_b[t] = L.r_off + k;
        }
    }
    finish_merges(P);
    const double ncell = (double)P.ncell, nface = (double)(P.nxface + P.nyface);
    P.residual_flops = 8.0 * ncell + 8.0 * (double)P.nskel_faces;
    P.finish_flops = 3.0 * nface + 2.0 * ncell;
    return MRCM_OK;
}

// The merge descriptors grouped by tree height, their storage, and the flop
// counts of the merges and of the solve's tree sweeps.
void finish_merges(Plan& P) {
    const int nnode = (int)P.nodes.size();
    // merges grouped by height
    std::vector<double> node_lu_flops, node_inv_flops, node_prod_flops;
    std::vector<std::vector<int>> by_h(P.height + 1);
    for (int v = P.nleaf; v < nnode; ++v) by_h[P.nodes[v].height].push_back(v);
    P.level_first.assign(P.height, 0);
    P.level_count.assign(P.height, 0);
    P.level_max_g2.assign(P.height, 0);
    P.level_max_m.assign(P.height, 0);
    for (int h = 1; h <= P.height; ++h) {
        P.level_first[h - 1] = (int)P.merges.size();
        P.level_count[h - 1] = (int)by_h[h].size();
        for (int v : by_h[h]) {
            Plan::Node& nd = P.nodes[v];
            MergeDesc D;
            std::memset(&D, 0, sizeof(D));
            D.node = v;
            D.c1 = nd.c1;
            D.c2 = nd.c2;
            D.g = (int)nd.gamma.size();
            D.m = (int)nd.segs.size();
            D.o1 = nd.o1;
            D.m1 = (int)P.nodes[nd.c1].segs.size();
            D.m2 = (int)P.nodes[nd.c2].segs.size();
            D.map_off = (int)P.node_map.size();
            P.node_map.insert(P.node_map.end(), nd.map.begin(), nd.map.end());
            D.gamma_off = (int)P.gamma_segs.size();
            P.gamma_segs.insert(P.gamma_segs.end(), nd.gamma.begin(), nd.gamma.end());
            D.pinned = P.root_pinned[v];
            D.R_off = P.node_R_off[v];
            D.R1_off = P.node_R_off[nd.c1];
            D.R2_off = P.node_R_off[nd.c2];
            D.r_off = P.node_r_off[v];
            D.r1_off = P.node_r_off[nd.c1];
            D.r2_off = P.node_r_off[nd.c2];
            const long long g2 = 2LL * D.g, m = D.m;
            D.W_off = P.nW;    P.nW += g2 * g2;
            D.X_off = P.nX;    P.nX += g2 * m;
            P.merges.push_back(D);
            P.level_max_g2[h - 1] = std::max(P.level_max_g2[h - 1], (int)g2);
            P.level_max_m[h - 1] = std::max(P.level_max_m[h - 1], (int)m);
            P.max_g2 = std::max(P.max_g2, (int)g2);
            // flop model: Gauss-Jordan inversion of the 2g x 2g form (N steps
            // of a rank-one update of the lower triangle: N^2 (N + 1)), X =
            // -W C over C's blocks (2 N g m), the lower triangle of
            // the symmetric R update (g m (m + 1)); solve passes: up 2 m N,
            // down 2 N (m + N).  The path of a level is known once all its
            // nodes are listed, so inv is set in the phase pass below.
            const double N = (double)g2, gd = (double)D.g, md = (double)m;
            const double lu = 0.0, inv = 2.0 * N * N * N, prod = 2.0 * N * gd * md + md * (md + 1.0) * gd;
            P.merge_flops += (long long)(lu + inv + prod);
            P.model_build += 2.0 / 3.0 * N * N * N + 2.0 * N * N * (md + 1.0) + 2.0 * md * gd * (md + 1.0);
            P.solve_flops += 2LL * g2 * m + 2LL * g2 * (m + g2);
            if (m > 0) P.phase_pass[MRCM_PHASE_TREE_UP] += 2.0 * md * N;
            P.phase_pass[MRCM_PHASE_TREE_DOWN] += 2.0 * N * (md + N);
            node_lu_flops.push_back(lu);
            node_inv_flops.push_back(inv);
            node_prod_flops.push_back(prod);
        }
    }
    // build phases: leaves, then per level the per-node register path or the
    // blocked Gauss-Jordan sweep
    P.phase_build[MRCM_PHASE_LEAF_BUILD] = (double)P.leaf_flops;
    for (int h = 1; h <= P.height; ++h) {
        const int f0 = P.level_first[h - 1], cnt = P.level_count[h - 1];
        const bool blocked = merge_level_blocked(cnt, P.level_max_g2[h - 1], P.level_max_m[h - 1]);
        for (int q = f0; q < f0 + cnt; ++q) {
            const MergeDesc& D = P.merges[q];
            const double N = 2.0 * D.g, gd = D.g, md = D.m;
            if (!blocked) {
                const double sym = N * N * (N + 1.0);
                P.merge_flops += (long long)(sym - node_inv_flops[q]);
                P.phase_build[MRCM_PHASE_MERGE_SMALL] += sym + node_prod_flops[q];
                continue;
            }
            const double sym = N * N * (N + 1.0);      // lower-triangle sweep
            P.merge_flops += (long long)(sym - node_inv_flops[q]);
            P.model_sweep += 2.0 / 3.0 * N * N * N;
            P.phase_build[MRCM_PHASE_GJ_SWEEP] += sym;
            if (P.level_max_m[h - 1] == 0) {
                // factor form of a root level: the rank-one count of the
                // trailing updates, N (N^2 - 1) / 3; solve passes: the
                // forward sweep (N^2), the inverse diagonal blocks (2 kGJ N)
                // and the backward sweep (N^2) instead of the product (2 N^2)
                const double fac = N * (N * N - 1.0) / 3.0;
                for (int a = 0; a < 2; ++a) {
                    if (a == 1 && P.level_max_g2[h - 1] < kRootFactorMinG2) continue;
                    P.root_build[a][MRCM_PHASE_GJ_SWEEP] -= sym;
                    P.root_build[a][MRCM_PHASE_ROOT_FACTOR] += fac;
                    P.root_merge[a] += fac - sym;
                    P.root_model_sweep[a] -= 2.0 / 3.0 * N * N * N;
                    P.root_pass[a][MRCM_PHASE_TREE_UP] += N * N;
                    P.root_pass[a][MRCM_PHASE_TREE_DOWN] += N * N + 2.0 * kMergeBlock * N - 2.0 * N * N;
                    P.root_solve[a] += 2.0 * kMergeBlock * N;
                }
            }
            P.phase_build[MRCM_PHASE_MERGE_X] += 2.0 * N * gd * md;
            P.phase_build[MRCM_PHASE_MERGE_R] += md * (md + 1.0) * gd;
        }
    }
}


// First row of each column of B of a 3D block (local cells x fastest; the
// local segment of a skeleton face as the leaf kernel numbers it).
void leaf3_starts(const LeafDesc3& B, std::vector<int>& start) {
    const int n = B.w[0] * B.w[1] * B.w[2];
    start.assign(B.m, n);
    for (int c = 0; c < n; ++c) {
        const int loc[3] = {c % B.w[0], (c / B.w[0]) % B.w[1], c / (B.w[0] * B.w[1])};
        for (int side = 0; side < 6; ++side) {
            const int d = side >> 1, up = side & 1;
            const int p = loc[d] + (up ? 1 : -1);
            if ((p >= 0 && p < B.w[d]) || B.side_off[side] < 0) continue;
            const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
            const int s = B.side_off[side] + (B.side_fine[side] ? loc[t2] * B.w[t1] + loc[t1] : 0);
            start[s] = std::min(start[s], c);
        }
    }
}

// The 3D plan.  Blocks of the patch shape (seg cells per axis) tile the grid;
// a face between two blocks of one subdomain (sub cells per axis) is a
// segment of its own, the side shared by blocks of two subdomains is one
// patch.  One tree by recursive bisection of the block box (the axis with
// the most blocks, ties x, y, z; the lower half takes ceil(count / 2)).
int make_plan3d(Plan& P) {
    const Grid3& G = P.g3;
    const int b[3] = {P.gx, P.gy, P.gz};
    const int sub[3] = {P.sx, P.sy, P.sz};
    const int n[3] = {G.nx, G.ny, G.nz};
    int Nb[3];
    for (int d = 0; d < 3; ++d) Nb[d] = n[d] / b[d];
    P.ncell = (long long)G.nx * G.ny * G.nz;
    P.nxface = (long long)(G.nx + 1) * G.ny * G.nz;
    P.nyface = (long long)G.nx * (G.ny + 1) * G.nz;
    P.nzface = (long long)G.nx * G.ny * (G.nz + 1);
    P.nbc = 2LL * ((long long)G.ny * G.nz + (long long)G.nx * G.nz + (long long)G.nx * G.ny);
    P.pure_neumann = !(G.bc[0] || G.bc[1] || G.bc[2] || G.bc[3] || G.bc[4] || G.bc[5]);
    P.nleaf = Nb[0] * Nb[1] * Nb[2];
    P.leaves3.assign(P.nleaf, LeafDesc3{});
    const int stride[3] = {1, Nb[0], Nb[0] * Nb[1]};
    auto tang = [](int d, int& t1, int& t2) { t1 = d == 0 ? 1 : 0; t2 = d == 2 ? 1 : 2; };
    std::vector<int> plus_first(3 * (size_t)P.nleaf, -1), plus_fine(3 * (size_t)P.nleaf, 0);
    for (int id = 0; id < P.nleaf; ++id) {
        const int idx[3] = {id % Nb[0], (id / Nb[0]) % Nb[1], id / (Nb[0] * Nb[1])};
        LeafDesc3& B = P.leaves3[id];
        std::memset(&B, 0, sizeof(B));
        B.i0 = idx[0] * b[0]; B.j0 = idx[1] * b[1]; B.k0 = idx[2] * b[2];
        for (int d = 0; d < 3; ++d) B.w[d] = b[d];
        for (int d = 0; d < 3; ++d) {
            if (idx[d] + 1 >= Nb[d]) continue;
            const bool fine = (idx[d] * b[d]) / sub[d] == ((idx[d] + 1) * b[d]) / sub[d];
            int t1, t2;
            tang(d, t1, t2);
            const int base[3] = {B.i0, B.j0, B.k0};
            plus_first[3 * (size_t)id + d] = P.nseg;
            plus_fine[3 * (size_t)id + d] = fine ? 1 : 0;
            auto add = [&](int lo1, int len1, int lo2, int len2) {
                P.seg_axis.push_back(d);
                P.seg_line.push_back(base[d] + b[d]);
                P.seg_lo.push_back(lo1);
                P.seg_len.push_back(len1);
                P.seg_lo2.push_back(lo2);
                P.seg_len2.push_back(len2);
                P.seg_a.push_back(id);
                P.seg_b.push_back(id + stride[d]);
                P.seg_grid.push_back(0);
                ++P.nseg;
            };
            if (fine) {
                for (int w = 0; w < b[t2]; ++w)
                    for (int u = 0; u < b[t1]; ++u) add(base[t1] + u, 1, base[t2] + w, 1);
            } else {
                add(base[t1], b[t1], base[t2], b[t2]);
            }
        }
    }
    P.seg_face_off.resize(P.nseg + 1);
    P.seg_face_off[0] = 0;
    for (int t = 0; t < P.nseg; ++t) P.seg_face_off[t + 1] = P.seg_face_off[t] + P.seg_len[t] * P.seg_len2[t];
    P.nskel_faces = P.seg_face_off[P.nseg];
    P.xface_seg.assign((size_t)P.nxface, -1);
    P.yface_seg.assign((size_t)P.nyface, -1);
    P.zface_seg.assign((size_t)P.nzface, -1);
    for (int t = 0; t < P.nseg; ++t) {
        const int d = P.seg_axis[t];
        int t1, t2;
        tang(d, t1, t2);
        for (int w = P.seg_lo2[t]; w < P.seg_lo2[t] + P.seg_len2[t]; ++w)
            for (int u = P.seg_lo[t]; u < P.seg_lo[t] + P.seg_len[t]; ++u) {
                int pos[3];
                pos[d] = P.seg_line[t]; pos[t1] = u; pos[t2] = w;
                const long long i = pos[0], j = pos[1], k = pos[2];
                if (d == 0) P.xface_seg[(size_t)((k * G.ny + j) * (G.nx + 1) + i)] = t;
                else if (d == 1) P.yface_seg[(size_t)((k * (G.ny + 1) + j) * G.nx + i)] = t;
                else P.zface_seg[(size_t)((k * G.ny + j) * G.nx + i)] = t;
            }
    }
    // block segment lists: sides x-, x+, y-, y+, z-, z+
    for (int id = 0; id < P.nleaf; ++id) {
        const int idx[3] = {id % Nb[0], (id / Nb[0]) % Nb[1], id / (Nb[0] * Nb[1])};
        LeafDesc3& B = P.leaves3[id];
        B.seg_off = (int)P.leaf_segs.size();
        int cnt = 0;
        for (int side = 0; side < 6; ++side) {
            const int d = side >> 1, up = side & 1;
            int t1, t2;
            tang(d, t1, t2);
            const int owner = up ? id : (idx[d] > 0 ? id - stride[d] : -1);
            const int first = owner >= 0 ? plus_first[3 * (size_t)owner + d] : -1;
            if (first < 0) { B.side_off[side] = -1; B.side_fine[side] = 0; continue; }
            const int fine = plus_fine[3 * (size_t)owner + d];
            const int count = fine ? b[t1] * b[t2] : 1;
            B.side_off[side] = cnt;
            B.side_fine[side] = fine;
            for (int k = 0; k < count; ++k) P.leaf_segs.push_back(first + k);
            cnt += count;
        }
        B.m = cnt;
        P.max_m_leaf = std::max(P.max_m_leaf, cnt);
    }
    // tree
    P.nodes.assign(P.nleaf, Plan::Node{});
    for (int id = 0; id < P.nleaf; ++id) {
        Plan::Node& nd = P.nodes[id];
        const int I = id % Nb[0], J = (id / Nb[0]) % Nb[1];
        nd.box[0] = I; nd.box[1] = I + 1; nd.box[2] = J; nd.box[3] = J + 1;
        nd.leaf = id;
        const LeafDesc3& B = P.leaves3[id];
        nd.segs.assign(P.leaf_segs.begin() + B.seg_off, P.leaf_segs.begin() + B.seg_off + B.m);
    }
    struct Rec3 {
        Plan& P;
        const int* stride;
        int build(const int lo[3], const int hi[3]) {
            int d = 0;
            for (int a = 1; a < 3; ++a)
                if (hi[a] - lo[a] > hi[d] - lo[d]) d = a;
            if (hi[d] - lo[d] == 1) return lo[0] * stride[0] + lo[1] * stride[1] + lo[2] * stride[2];
            const int mid = lo[d] + (hi[d] - lo[d] + 1) / 2;
            int h1[3] = {hi[0], hi[1], hi[2]}, l2[3] = {lo[0], lo[1], lo[2]};
            h1[d] = mid;
            l2[d] = mid;
            const int c1 = build(lo, h1);
            const int c2 = build(l2, hi);
            const int box[4] = {lo[0], hi[0], lo[1], hi[1]};
            return add_merge_node(P, c1, c2, box);
        }
    };
    {
        Rec3 rec{P, stride};
        const int lo[3] = {0, 0, 0};
        const int root = rec.build(lo, Nb);
        P.roots.assign(1, root);
        P.height = P.nodes[root].height;
    }
    finish_tree(P);
    // block storage and flop counts (banded Cholesky, Z from each column's
    // first nonzero row within the band, the lower triangle of Z^T Z from
    // each pair's later start)
    std::map<std::vector<int>, long long> flop_cache;
    std::vector<int> start;
    for (int id = 0; id < P.nleaf; ++id) {
        LeafDesc3& B = P.leaves3[id];
        const long long nn = (long long)B.w[0] * B.w[1] * B.w[2], m = B.m;
        B.L_off = P.nL; P.nL += nn * nn;
        B.Z_off = P.nZ; P.nZ += nn * m;
        B.zb_off = P.nzb; P.nzb += nn;
        B.R_off = P.node_R_off[id];
        B.r_off = P.node_r_off[id];
        std::vector<int> key(B.side_off, B.side_off + 6);
        key.insert(key.end(), B.side_fine, B.side_fine + 6);
        auto it = flop_cache.find(key);
        long long f;
        if (it != flop_cache.end()) {
            f = it->second;
        } else {
            leaf3_starts(B, start);
            f = 0;
            const long long bw = (long long)B.w[0] * B.w[1];
            for (long long k = 0; k < nn; ++k) {
                const long long len = std::min(bw, nn - 1 - k);
                f += 2 + len + len * (len + 1);                  // 1/sqrt, column scale, band triangle
                for (int s = 0; s < m; ++s)
                    if (start[s] <= k) f += 1 + 2 * len;         // row scale and band update of Z
            }
            for (int r = 0; r < m; ++r)
                for (int q = 0; q <= r; ++q) f += 2 * (nn - std::max(start[r], start[q]));
            flop_cache[key] = f;
        }
        P.leaf_flops += f;
        P.model_build += (double)f;
        const long long bwn = (long long)B.w[0] * B.w[1] * nn;
        P.solve_flops += 4 * bwn + 4 * nn * m;
        P.phase_pass[MRCM_PHASE_LEAF_PART] += (double)(2 * bwn + 2 * nn * m);
        P.phase_pass[MRCM_PHASE_LEAF_PRESSURE] += (double)(2 * bwn + 2 * nn * m);
    }
    P.seg_lam_a.assign(P.nseg, -1);
    P.seg_lam_b.assign(P.nseg, -1);
    for (int id = 0; id < P.nleaf; ++id) {
        const LeafDesc3& B = P.leaves3[id];
        for (int k = 0; k < B.m; ++k) {
            const int t = P.leaf_segs[B.seg_off + k];
            if (P.seg_a[t] == id) P.seg_lam_a[t] = B.r_off + k;
            else P.seg_lam_b[t] = B.r_off + k;
        }
    }
    finish_merges(P);
    P.finish_flops = 3.0 * (double)(P.nxface + P.nyface + P.nzface) + (double)P.ncell;
    return MRCM_OK;
}

}  // namespace

// The CUDA error behind the last MRCM_ERR_CUDA / MRCM_ERR_OOM of this thread.
static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

int mrcm::cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return MRCM_OK;
    g_last_cuda_error = e;
    if (e == cudaErrorMemoryAllocation) return MRCM_ERR_OOM;
    return MRCM_ERR_CUDA;
}

// Refinement steps of the mixed form by default: with FP64 leaf factors and
// FP32 merges each step contracts the residual ~60 times at 4096^2, so three
// reach ~1e-9 against the FP64 solution.
constexpr int kMixedRefineDefault = 3;
// In 3D (FP32 merges over 4^3-cell blocks, FP64 blocks) each step contracts
// the residual ~1000 times at 256 x 256 x 64: two steps reach 1.6e-9 against
// the FP64 solution (one: 1.6e-6, three: 1.7e-12).
constexpr int kMixedRefineDefault3D = 2;

// Largest interface system 2g merged in FP32 by default in the mixed form:
// every one (the FP32 merges' errors are small beside the contraction; FP32
// leaf factors are what slowed the refinement at 4096^2: 0.3 per step).
constexpr int kMixedSplitDefault = 1 << 30;

struct mrcm_ctx {
    Plan P;
    int precision = MRCM_FP64;
    int mixed_split = kMixedSplitDefault;
    int root_form = MRCM_ROOT_AUTO;       // mrcm_set_root_form
    std::vector<MergeTune> tune;          // per tree height (mrcm_autotune); empty: heuristics
    cudaStream_t stream = nullptr;
    int device = 0;
    bool built = false;
    bool solved = false;
    DevView v{};
    std::vector<void*> allocs;
    size_t bytes = 0;
    double* K = nullptr;
    int launches_build = 0, launches_solve = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;          // event pairs, handed out per launch group
    std::vector<int> ev_phase;            // phase of each used pair
    int ev_used = 0;
    double* gj_scratch = nullptr;
    unsigned long long* gj_barrier = nullptr;
    TreeLevels tree{};                    // merge levels for the fused solve sweeps
    int tree_grid = 1;
    double* tree_scratch = nullptr;
    int refine_steps = 1;
    int refine_check = 0;
    int hist_count = 0;
    // CUDA graphs of the build and solve launch sequences (captured on first
    // use, replayed after; the solve graph is keyed by its arguments)
    bool use_graphs = true;      // mrcm_use_graphs
    bool graphs_ok = true;       // false once a capture failed on this stream
    bool capturing = false;
    long long graph_replays = 0;
    cudaGraphExec_t build_exec = nullptr;
    bool build_timing = false;
    int build_ev_used = 0;
    cudaGraphExec_t solve_exec = nullptr;
    const void* solve_key[9] = {};
    int solve_ev_begin = 0, solve_ev_used = 0, solve_launches = 0;
};

namespace {

int cuda_err(cudaError_t e) { return mrcm::cuda_status(e); }

template <class T>
int dev_alloc(mrcm_ctx* c, T** p, long long count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) return cuda_err(e);
    c->allocs.push_back(ptr);
    c->bytes += sizeof(T) * (size_t)count;
    *p = static_cast<T*>(ptr);
    return MRCM_OK;
}

template <class T>
int upload(mrcm_ctx* c, const T** out, const std::vector<T>& h) {
    T* d = nullptr;
    int rc = dev_alloc(c, &d, (long long)h.size());
    if (rc) return rc;
    if (!h.empty()) {
        cudaError_t e = cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_err(e);
    }
    *out = d;
    return MRCM_OK;
}

int read_status(mrcm_ctx* c) {
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, c->v.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(e);
    if (st & kStatusBadK) return MRCM_ERR_BAD_K;
    if (st & kStatusSingular) return MRCM_ERR_SINGULAR;
    if (st & kStatusTimeout) return MRCM_ERR_TIMEOUT;
    if (st & (kStatusBadIndex | kStatusInconsistent)) return MRCM_ERR_INVALID_ARG;
    return MRCM_OK;
}

// Records a CUDA event pair around one launch group of a phase; the phase
// time of a call is the sum over its groups.  The external-record flag makes
// the records event-record nodes when the sequence is captured into a graph.
constexpr int kEventPairs = 4096;
void record_event(mrcm_ctx* c, cudaEvent_t e) {
    if (c->capturing)
        cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
    else
        cudaEventRecord(e, c->stream);
}
void phase_begin(void* vc, int phase) {
    mrcm_ctx* c = static_cast<mrcm_ctx*>(vc);
    if (!c->timing || c->ev_used >= kEventPairs) return;
    c->ev_phase[c->ev_used] = phase;
    record_event(c, c->ev[2 * c->ev_used]);
}
void phase_end(void* vc, int) {
    mrcm_ctx* c = static_cast<mrcm_ctx*>(vc);
    if (!c->timing || c->ev_used >= kEventPairs) return;
    record_event(c, c->ev[2 * c->ev_used + 1]);
    ++c->ev_used;
}
struct PhaseScope {
    mrcm_ctx* c;
    int phase;
    PhaseScope(mrcm_ctx* c_, int p) : c(c_), phase(p) { phase_begin(c, p); }
    ~PhaseScope() { phase_end(c, phase); }
};

}  // namespace

#define TRY(x) do { int rc_ = (x); if (rc_ != MRCM_OK) return rc_; } while (0)
#define TRYC(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_err(e_); } while (0)

// Captures the launches of fn into a graph executable on the context's
// stream (updating *exec in place when only launch arguments differ); false
// (nothing left captured) when the stream cannot be captured (the legacy
// default stream) or capture fails.
template <class F>
static bool capture_graph(mrcm_ctx* c, cudaGraphExec_t* exec, F&& fn) {
    if (!c->use_graphs || !c->graphs_ok || c->stream == nullptr) return false;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        c->graphs_ok = false;
        return false;
    }
    c->capturing = true;
    const int rc = fn();
    c->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (rc != MRCM_OK || e != cudaSuccess || graph == nullptr) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        c->graphs_ok = false;
        return false;
    }
    if (*exec) {
        // same launch sequence with other arguments: update in place
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(*exec, graph, &info) == cudaSuccess) {
            cudaGraphDestroy(graph);
            return true;
        }
        cudaGetLastError();
    }
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        c->graphs_ok = false;
        return false;
    }
    if (*exec) cudaGraphExecDestroy(*exec);
    *exec = ge;
    return true;
}

extern "C" {

int mrcm_last_cuda_error(char* name, int cap) {
    const cudaError_t e = g_last_cuda_error;
    if (name && cap > 0) {
        std::strncpy(name, cudaGetErrorName(e), (size_t)cap - 1);
        name[cap - 1] = 0;
    }
    return (int)e;
}

const char* mrcm_error_string(int code) {
    switch (code) {
        case MRCM_OK: return "ok";
        case MRCM_ERR_INVALID_ARG: return "invalid argument";
        case MRCM_ERR_SHAPE: return "segment length does not divide the leaf side, or leaf too large";
        case MRCM_ERR_BAD_K: return "permeability not positive and finite";
        case MRCM_ERR_NOT_BUILT: return "basis not built (call mrcm_build_basis first)";
        case MRCM_ERR_SINGULAR: return "singular local or interface system";
        case MRCM_ERR_CUDA: return "CUDA runtime error";
        case MRCM_ERR_OOM: return "device out of memory";
        case MRCM_ERR_TIMEOUT: return "bounded device wait timed out";
        case MRCM_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown error";
    }
}

// A 3D grid: blocks of the patch shape (at most kLeaf3Cells cells, at most
// 16 faces per side) that tile the subdomains, which tile the grid.
static int validate3(const mrcm_grid& G, const int sub[3], const int seg[3], const int* bc) {
    long long cells = 1;
    for (int d = 0; d < 3; ++d) {
        if (G.n[d] < 1 || !(G.L[d] > 0) || sub[d] < 1 || seg[d] < 1) return MRCM_ERR_INVALID_ARG;
        cells *= G.n[d];
    }
    for (int s = 0; s < 6; ++s)
        if (bc[s] != MRCM_BC_NEUMANN && bc[s] != MRCM_BC_DIRICHLET) return MRCM_ERR_INVALID_ARG;
    if (4 * cells + 3LL * G.n[0] * G.n[1] > (1LL << 31)) return MRCM_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (sub[d] % seg[d] != 0 || G.n[d] % sub[d] != 0) return MRCM_ERR_SHAPE;
    if (seg[0] * seg[1] * seg[2] > kLeaf3Cells) return MRCM_ERR_SHAPE;
    for (int d = 0; d < 3; ++d) {
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        if (seg[t1] * seg[t2] > kLeaf3Segs / 6) return MRCM_ERR_SHAPE;
    }
    return MRCM_OK;
}

static void fill_plan_inputs3(Plan& P, const mrcm_grid& g, const int sub[3], const int seg[3], double alpha,
                              const int* bc) {
    P.dim = 3;
    P.g3.nx = g.n[0]; P.g3.ny = g.n[1]; P.g3.nz = g.n[2];
    P.g3.hx = g.L[0] / g.n[0]; P.g3.hy = g.L[1] / g.n[1]; P.g3.hz = g.L[2] / g.n[2];
    for (int s = 0; s < 6; ++s) P.g3.bc[s] = bc[s];
    P.grids.assign(1, GridDesc{});
    std::memset(&P.grids[0], 0, sizeof(GridDesc));
    P.grids[0].nx = g.n[0];
    P.grids[0].ny = g.n[1];
    P.alpha = alpha;
    P.sx = sub[0]; P.sy = sub[1]; P.sz = sub[2];
    P.gx = seg[0]; P.gy = seg[1]; P.gz = seg[2];
}

// count grids g[k] with boundary types bc_type[6 k .. 6 k + 5]
static int validate(int count, const mrcm_grid* g, const int sub_cells[3], const int seg_cells[3],
                    const int* bc_type) {
    if (count < 1 || !g || !sub_cells || !seg_cells || !bc_type) return MRCM_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k)
        if (g[k].dim == 3) return count == 1 ? validate3(g[0], sub_cells, seg_cells, bc_type) : MRCM_ERR_UNSUPPORTED;
    long long cells = 0, faces = 0;
    bool all_neumann = false;
    for (int k = 0; k < count; ++k) {
        const mrcm_grid& G = g[k];
        if (G.dim != 2) return MRCM_ERR_INVALID_ARG;
        if (G.n[0] < 1 || G.n[1] < 1 || !(G.L[0] > 0) || !(G.L[1] > 0)) return MRCM_ERR_INVALID_ARG;
        cells += (long long)G.n[0] * G.n[1];
        faces += 2LL * G.n[0] * G.n[1] + G.n[0] + G.n[1];
        const int* bc = bc_type + 6 * k;
        for (int s = 0; s < 4; ++s)
            if (bc[s] != MRCM_BC_NEUMANN && bc[s] != MRCM_BC_DIRICHLET) return MRCM_ERR_INVALID_ARG;
        all_neumann |= !(bc[0] || bc[1] || bc[2] || bc[3]);
    }
    // every index of the workspace stays below 2^31 (32-bit index arithmetic)
    if (cells > (1LL << 31) || faces > (1LL << 31)) return MRCM_ERR_INVALID_ARG;
    for (int d = 0; d < 2; ++d) {
        if (sub_cells[d] < 1 || seg_cells[d] < 1) return MRCM_ERR_INVALID_ARG;
        if (sub_cells[d] > kMaxLeafSide) return MRCM_ERR_SHAPE;
        if (seg_cells[d] > sub_cells[d] || sub_cells[d] % seg_cells[d] != 0) return MRCM_ERR_SHAPE;
    }
    // all-Neumann problems (zero-mean pressure) only as a context of their own
    if (all_neumann && count > 1) return MRCM_ERR_UNSUPPORTED;
    return MRCM_OK;
}

static void fill_plan_inputs(Plan& P, int count, const mrcm_grid* g, const int sub[3], const int seg[3],
                             double alpha, const int* bc_type) {
    P.grids.assign(count, GridDesc{});
    for (int k = 0; k < count; ++k) {
        GridDesc& G = P.grids[k];
        std::memset(&G, 0, sizeof(G));
        G.nx = g[k].n[0];
        G.ny = g[k].n[1];
        G.hx = g[k].L[0] / g[k].n[0];
        G.hy = g[k].L[1] / g[k].n[1];
        for (int s = 0; s < 4; ++s) G.bc[s] = bc_type[6 * k + s];
    }
    P.alpha = alpha;
    P.sx = sub[0]; P.sy = sub[1];
    P.gx = seg[0]; P.gy = seg[1];
}

// which set of root-level flop differences applies to a root form: -1 none
static int root_set(int form) { return form == MRCM_ROOT_FACTOR ? 0 : (form == MRCM_ROOT_AUTO ? 1 : -1); }

static int plan_value(const Plan& P, int what, long long* value, int form = MRCM_ROOT_AUTO) {
    const int a = root_set(form);
    const double f = a >= 0 ? 1.0 : 0.0;
    const int ai = a >= 0 ? a : 0;
    switch (what) {
        case MRCM_Q_LEAVES: *value = P.nleaf; break;
        case MRCM_Q_SEGMENTS: *value = P.nseg; break;
        case MRCM_Q_LEVELS: *value = P.height; break;
        case MRCM_Q_NODES: *value = (long long)P.nodes.size(); break;
        case MRCM_Q_MAX_GAMMA: *value = P.max_g2; break;
        case MRCM_Q_BUILD_FLOPS: *value = P.leaf_flops + P.merge_flops + (long long)(f * P.root_merge[ai]); break;
        case MRCM_Q_SOLVE_FLOPS: *value = P.solve_flops + (long long)(f * P.root_solve[ai]); break;  // one pass
        case MRCM_Q_LEAF_FLOPS: *value = P.leaf_flops; break;
        case MRCM_Q_MODEL_BUILD_FLOPS: *value = (long long)P.model_build; break;
        case MRCM_Q_MODEL_SWEEP_FLOPS: *value = (long long)(P.model_sweep + f * P.root_model_sweep[ai]); break;
        case MRCM_Q_GRIDS: *value = (long long)P.grids.size(); break;
        case MRCM_Q_CELLS: *value = P.ncell; break;
        default: return MRCM_ERR_INVALID_ARG;
    }
    return MRCM_OK;
}

int mrcm_plan_query(const mrcm_grid* g, const int sub_cells[3], const int seg_cells[3],
                    const int bc_type[6], int what, long long* value) {
    if (!value) return MRCM_ERR_INVALID_ARG;
    TRY(validate(1, g, sub_cells, seg_cells, bc_type));
    if (what == MRCM_Q_WORKSPACE_BYTES) { *value = 0; return MRCM_OK; }
    Plan P;
    if (g->dim == 3) {
        fill_plan_inputs3(P, *g, sub_cells, seg_cells, 1.0, bc_type);
        TRY(make_plan3d(P));
    } else {
        fill_plan_inputs(P, 1, g, sub_cells, seg_cells, 1.0, bc_type);
        TRY(make_plan(P));
    }
    return plan_value(P, what, value);
}

// Whether height h (1-based) keeps the factor of its interface systems: a
// blocked level whose nodes have no outer segments (roots), in the factor
// form of the context.
static bool level_factor(const mrcm_ctx* c, int h) {
    const Plan& P = c->P;
    if (c->root_form == MRCM_ROOT_INVERSE || P.level_max_m[h - 1] != 0 ||
        !merge_level_blocked(P.level_count[h - 1], P.level_max_g2[h - 1], P.level_max_m[h - 1]))
        return false;
    return c->root_form == MRCM_ROOT_FACTOR || P.level_max_g2[h - 1] >= kRootFactorMinG2;
}
static void set_tree_forms(mrcm_ctx* c) {
    for (int h = 1; h <= c->P.height; ++h) c->tree.form[h - 1] = level_factor(c, h) ? 1 : 0;
}

// Workspace of the merges and of the fused solve sweeps (both forms, 2D and
// 3D): Gauss-Jordan scratch and barrier words, the sweep levels, the factor
// form's flags and the sweep plan.
static int setup_tree(mrcm_ctx* c) {
    const Plan& P = c->P;
    DevView& v = c->v;
    {
        size_t nscr = 1;
        for (int h = 1; h <= P.height; ++h)
            nscr = std::max(nscr, merge_scratch_doubles(P.level_count[h - 1], P.level_max_g2[h - 1],
                                                        P.level_max_m[h - 1]));
        TRY(dev_alloc(c, &c->gj_scratch, (long long)nscr));
        TRY(dev_alloc(c, &c->gj_barrier, (long long)(kMergeBarrierBytes / sizeof(unsigned long long))));
    }
    {
        if (P.height > kMaxTreeLevels) return MRCM_ERR_UNSUPPORTED;
        TreeLevels& T = c->tree;
        T.height = P.height;
        T.x_len = P.nX;
        T.w_len = P.nW;
        T.n_merges = (long long)P.merges.size();
        T.map_len = (long long)P.node_map.size();
        for (int h = 1; h <= P.height; ++h) {
            T.first[h - 1] = P.level_first[h - 1];
            T.count[h - 1] = P.level_count[h - 1];
            T.g2[h - 1] = P.level_max_g2[h - 1];
            T.m[h - 1] = P.level_max_m[h - 1];
        }
        TRY(dev_alloc(c, &v.rgam, std::max<long long>(2 * (long long)P.gamma_segs.size(), 1)));
        TRY(dev_alloc(c, &v.fwd, std::max<long long>(2 * (long long)P.gamma_segs.size(), 1)));
        // flags of the triangular sweeps: per node of a level that may take
        // the factor form, one per solve block
        long long nflag = 1;
        for (int h = 1; h <= P.height; ++h)
            if (P.level_max_m[h - 1] == 0)
                nflag = std::max(nflag, (long long)P.level_count[h - 1] *
                                            ((P.level_max_g2[h - 1] + kTriBlock - 1) / kTriBlock));
        v.tri_flag_n = nflag;
        TRY(dev_alloc(c, &v.tri_flags, 2 * nflag));
        set_tree_forms(c);
        TRYC(tree_grid(&c->tree_grid));
        const long long need = tree_plan_chunks(T, c->tree_grid);
        TRY(dev_alloc(c, &c->tree_scratch, std::max(need, 1LL)));
    }
    return MRCM_OK;
}

static int setup3_impl(mrcm_ctx* c, const mrcm_grid* g, const double* K_dev, const int sub[3], const int seg[3],
                       double alpha, const int* bc_type, int precision, void* stream) {
    if (precision != MRCM_FP64 && precision != MRCM_MIXED) return MRCM_ERR_UNSUPPORTED;
    Plan& P = c->P;
    fill_plan_inputs3(P, *g, sub, seg, alpha, bc_type);
    c->stream = static_cast<cudaStream_t>(stream);
    TRYC(cudaGetDevice(&c->device));
    TRY(make_plan3d(P));
    if (P.pure_neumann && P.nleaf == 1) return MRCM_ERR_UNSUPPORTED;
    DevView& v = c->v;
    v.dim = 3;
    v.g3 = P.g3;
    v.mixed = precision == MRCM_MIXED ? 1 : 0;
    v.leaf32 = 0;                  // 3D blocks are factored in FP64
    v.res_dd = 0;                  // 3D refinement residuals in FP64
    c->precision = precision;
    c->refine_steps = v.mixed ? kMixedRefineDefault3D : 0;
    v.alpha = P.alpha;
    v.ncell = P.ncell; v.nxface = P.nxface; v.nyface = P.nyface; v.nzface = P.nzface; v.nbc = P.nbc;
    v.ngrid = 1;
    TRY(upload(c, &v.grids, P.grids));
    v.nleaf = P.nleaf; v.nseg = P.nseg;
    v.sx = P.sx; v.sy = P.sy; v.gx = P.gx; v.gy = P.gy;
    TRY(dev_alloc(c, &c->K, P.ncell));
    v.K = c->K;
    TRY(dev_alloc(c, &v.rx, 1));
    TRY(dev_alloc(c, &v.ry, 1));
    TRY(dev_alloc(c, &v.seg_beta, std::max(P.nseg, 1)));
    TRY(dev_alloc(c, &v.seg_D, std::max(P.nseg, 1)));
    TRY(dev_alloc(c, &v.cxL, P.nxface));
    TRY(dev_alloc(c, &v.cxU, P.nxface));
    TRY(dev_alloc(c, &v.cyL, P.nyface));
    TRY(dev_alloc(c, &v.cyU, P.nyface));
    TRY(dev_alloc(c, &v.czL, P.nzface));
    TRY(dev_alloc(c, &v.czU, P.nzface));
    TRY(upload(c, &v.seg_axis, P.seg_axis));
    TRY(upload(c, &v.seg_line, P.seg_line));
    TRY(upload(c, &v.seg_lo, P.seg_lo));
    TRY(upload(c, &v.seg_len, P.seg_len));
    TRY(upload(c, &v.seg_lo2, P.seg_lo2));
    TRY(upload(c, &v.seg_len2, P.seg_len2));
    TRY(upload(c, &v.seg_a, P.seg_a));
    TRY(upload(c, &v.seg_b, P.seg_b));
    TRY(upload(c, &v.seg_face_off, P.seg_face_off));
    TRY(upload(c, &v.seg_grid, P.seg_grid));
    TRY(upload(c, &v.xface_seg, P.xface_seg));
    TRY(upload(c, &v.yface_seg, P.yface_seg));
    TRY(upload(c, &v.zface_seg, P.zface_seg));
    TRY(dev_alloc(c, &v.seg_lam_dd, 2LL * std::max(P.nseg, 1)));
    TRY(upload(c, &v.seg_lam_a, P.seg_lam_a));
    TRY(upload(c, &v.seg_lam_b, P.seg_lam_b));
    TRY(upload(c, &v.leaves3, P.leaves3));
    TRY(upload(c, &v.leaf_segs, P.leaf_segs));
    TRY(upload(c, &v.merges, P.merges));
    TRY(upload(c, &v.node_map, P.node_map));
    TRY(upload(c, &v.gamma_segs, P.gamma_segs));
    TRY(dev_alloc(c, &v.leafL, P.nL));
    TRY(dev_alloc(c, &v.leafZ, std::max(P.nZ, 1LL)));
    TRY(dev_alloc(c, &v.leafL32, 1));
    TRY(dev_alloc(c, &v.leafZ32, 1));
    TRY(dev_alloc(c, &v.leafzb, P.nzb));
    TRY(dev_alloc(c, &v.R, std::max(P.nR, 1LL)));
    TRY(dev_alloc(c, &v.rbar, std::max(P.nr, 1LL)));
    TRY(dev_alloc(c, &v.lam, std::max(P.nr, 1LL)));
    TRY(dev_alloc(c, &v.X, std::max(P.nX, 1LL)));
    TRY(dev_alloc(c, &v.W, std::max(P.nW, 1LL)));
    TRY(dev_alloc(c, &v.W32, v.mixed ? std::max(P.nW, 1LL) : 1));
    TRY(dev_alloc(c, &v.segP, std::max(P.nseg, 1)));
    TRY(dev_alloc(c, &v.segU, std::max(P.nseg, 1)));
    TRY(dev_alloc(c, &v.segP_lo, std::max(P.nseg, 1)));
    TRY(dev_alloc(c, &v.segU_lo, std::max(P.nseg, 1)));
    TRY(dev_alloc(c, &v.p_hi, P.ncell));
    TRY(dev_alloc(c, &v.p_lo, P.ncell));
    TRY(dev_alloc(c, &v.rcell, P.ncell));
    TRY(dev_alloc(c, &v.sadj, std::max(P.nr, 1LL)));
    TRY(dev_alloc(c, &v.res_max, kMaxRefine + 1));
    TRY(dev_alloc(c, &v.red, 1024));
    TRY(setup_tree(c));
    TRY(dev_alloc(c, &v.status, 4));
    v.spin_limit = kDefaultSpinLimit;
    TRYC(cudaMemcpyAsync(c->K, K_dev, sizeof(double) * P.ncell, cudaMemcpyDefault, c->stream));
    TRYC(cudaMemsetAsync(v.status, 0, sizeof(int), c->stream));
    TRYC(cudaStreamSynchronize(c->stream));
    return MRCM_OK;
}

static int setup_impl(mrcm_ctx* c, int count, const mrcm_grid* g, const double* K_dev, const int sub[3],
                      const int seg[3], double alpha, const int* bc_type, int precision, void* stream) {
    Plan& P = c->P;
    fill_plan_inputs(P, count, g, sub, seg, alpha, bc_type);
    c->stream = static_cast<cudaStream_t>(stream);
    TRYC(cudaGetDevice(&c->device));
    TRY(make_plan(P));
    if (P.pure_neumann && P.nleaf == 1) return MRCM_ERR_UNSUPPORTED;
    DevView& v = c->v;
    v.mixed = precision == MRCM_MIXED ? 1 : 0;
    v.leaf32 = 0;                  // the mixed form's leaves in FP64 unless mrcm_set_mixed_leaves(1)
    v.res_dd = v.mixed ? 0 : 1;    // FP64 residuals suffice for the mixed form's tolerance
    c->precision = precision;
    if (v.mixed) c->refine_steps = kMixedRefineDefault;
    v.alpha = P.alpha;
    v.ncell = P.ncell; v.nxface = P.nxface; v.nyface = P.nyface; v.nbc = P.nbc;
    v.ngrid = (int)P.grids.size();
    TRY(upload(c, &v.grids, P.grids));
    v.nleaf = P.nleaf; v.nseg = P.nseg;
    v.sx = P.sx; v.sy = P.sy; v.gx = P.gx; v.gy = P.gy;
    const long long ncell = P.ncell;
    const long long nxf = P.nxface, nyf = P.nyface;
    TRY(dev_alloc(c, &c->K, ncell));
    v.K = c->K;
    TRY(dev_alloc(c, &v.rx, ncell));
    TRY(dev_alloc(c, &v.ry, ncell));
    TRY(dev_alloc(c, &v.seg_beta, P.nseg));
    TRY(dev_alloc(c, &v.seg_D, P.nseg));
    TRY(dev_alloc(c, &v.cxL, nxf));
    TRY(dev_alloc(c, &v.cxU, nxf));
    TRY(dev_alloc(c, &v.cyL, nyf));
    TRY(dev_alloc(c, &v.cyU, nyf));
    TRY(upload(c, &v.seg_axis, P.seg_axis));
    TRY(upload(c, &v.seg_line, P.seg_line));
    TRY(upload(c, &v.seg_lo, P.seg_lo));
    TRY(upload(c, &v.seg_len, P.seg_len));
    TRY(upload(c, &v.seg_a, P.seg_a));
    TRY(upload(c, &v.seg_b, P.seg_b));
    TRY(upload(c, &v.seg_face_off, P.seg_face_off));
    TRY(upload(c, &v.seg_grid, P.seg_grid));
    TRY(upload(c, &v.xface_seg, P.xface_seg));
    TRY(upload(c, &v.yface_seg, P.yface_seg));
    TRY(dev_alloc(c, &v.seg_lam_dd, 2LL * P.nseg));
    TRY(upload(c, &v.seg_lam_a, P.seg_lam_a));
    TRY(upload(c, &v.seg_lam_b, P.seg_lam_b));
    TRY(upload(c, &v.leaves, P.leaves));
    TRY(upload(c, &v.leaf_segs, P.leaf_segs));
    TRY(upload(c, &v.merges, P.merges));
    TRY(upload(c, &v.node_map, P.node_map));
    TRY(upload(c, &v.gamma_segs, P.gamma_segs));
    // leaf factors in the precision of the form (FP32 in the mixed form)
    // (the mixed form holds both precisions: mrcm_set_mixed_leaves switches)
    TRY(dev_alloc(c, &v.leafL, P.nL));
    TRY(dev_alloc(c, &v.leafZ, P.nZ));
    TRY(dev_alloc(c, &v.leafL32, v.mixed ? P.nL : 1));
    TRY(dev_alloc(c, &v.leafZ32, v.mixed ? P.nZ : 1));
    TRY(dev_alloc(c, &v.leafzb, P.nzb));
    TRY(dev_alloc(c, &v.R, P.nR));
    TRY(dev_alloc(c, &v.rbar, P.nr));
    TRY(dev_alloc(c, &v.lam, P.nr));
    TRY(dev_alloc(c, &v.X, P.nX));
    TRY(dev_alloc(c, &v.W, P.nW));
    TRY(dev_alloc(c, &v.W32, v.mixed ? P.nW : 1));
    TRY(dev_alloc(c, &v.segP, P.nseg));
    TRY(dev_alloc(c, &v.segU, P.nseg));
    TRY(dev_alloc(c, &v.segP_lo, P.nseg));
    TRY(dev_alloc(c, &v.segU_lo, P.nseg));
    TRY(dev_alloc(c, &v.p_hi, ncell));
    TRY(dev_alloc(c, &v.p_lo, ncell));
    TRY(dev_alloc(c, &v.rcell, ncell));
    TRY(dev_alloc(c, &v.sadj, P.nr));
    TRY(dev_alloc(c, &v.res_max, kMaxRefine + 1));
    TRY(dev_alloc(c, &v.red, 1024));
    TRY(setup_tree(c));
    TRY(dev_alloc(c, &v.status, 4));
    v.spin_limit = kDefaultSpinLimit;
    TRYC(cudaMemcpyAsync(c->K, K_dev, sizeof(double) * ncell, cudaMemcpyDefault, c->stream));
    // the root's lambda has no entries; lambda of every other node is written
    // top-down before it is read
    TRYC(cudaMemsetAsync(v.status, 0, sizeof(int), c->stream));
    TRYC(cudaStreamSynchronize(c->stream));
    return MRCM_OK;
}

int mrcm_setup(mrcm_ctx** out, const mrcm_grid* g, const double* K_dev, const int sub_cells[3],
               const int seg_cells[3], double alpha, const int bc_type[6], int precision,
               void* cuda_stream) {
    return mrcm_setup_batch(out, 1, g, bc_type, K_dev, sub_cells, seg_cells, alpha, precision, cuda_stream);
}

int mrcm_setup_batch(mrcm_ctx** out, int count, const mrcm_grid* grids, const int* bc_types, const double* K_dev,
                     const int sub_cells[3], const int seg_cells[3], double alpha, int precision,
                     void* cuda_stream) {
    if (!out) return MRCM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!K_dev) return MRCM_ERR_INVALID_ARG;
    const mrcm_grid* g = grids;
    const int* bc_type = bc_types;
    TRY(validate(count, g, sub_cells, seg_cells, bc_type));
    if (precision != MRCM_FP64 && precision != MRCM_MIXED && precision != MRCM_SURROGATE)
        return MRCM_ERR_INVALID_ARG;
    if (precision == MRCM_SURROGATE) return MRCM_ERR_UNSUPPORTED;
    if (!(alpha > 0) || !std::isfinite(alpha)) return MRCM_ERR_INVALID_ARG;
    mrcm_ctx* c = new (std::nothrow) mrcm_ctx();
    if (!c) return MRCM_ERR_OOM;
    int rc = g[0].dim == 3
                 ? setup3_impl(c, g, K_dev, sub_cells, seg_cells, alpha, bc_type, precision, cuda_stream)
                 : setup_impl(c, count, g, K_dev, sub_cells, seg_cells, alpha, bc_type, precision, cuda_stream);
    if (rc != MRCM_OK) {
        mrcm_destroy(c);
        return rc;
    }
    *out = c;
    return MRCM_OK;
}

int mrcm_set_permeability(mrcm_ctx* c, const double* K_dev) {
    if (!c || !K_dev) return MRCM_ERR_INVALID_ARG;
    TRYC(cudaMemcpyAsync(c->K, K_dev, sizeof(double) * (size_t)c->P.ncell, cudaMemcpyDefault,
                         c->stream));
    c->built = false;
    c->solved = false;
    TRYC(cudaStreamSynchronize(c->stream));
    return MRCM_OK;
}

// The launch sequence of mrcm_build_basis (no synchronisation); with
// merges_only the leaf maps already in place are merged again.
static int enqueue_build(mrcm_ctx* c, int& launches, bool merges_only = false) {
    const Plan& P = c->P;
    const DevView& v = c->v;
    cudaStream_t s = c->stream;
    launches = 0;
    TRYC(cudaMemsetAsync(v.status, 0, sizeof(int), s));
    if (!merges_only && P.dim == 3) {
        {
            PhaseScope ps(c, MRCM_PHASE_COEF);
            TRYC(launch_check_K(v, s)); ++launches;
            TRYC(launch_coef3(v, s)); launches += 1 + (P.nseg > 0);
        }
        PhaseScope ps(c, MRCM_PHASE_LEAF_BUILD);
        TRYC(launch_leaf3_build(v, s)); ++launches;
    } else if (!merges_only) {
        PhaseScope ps(c, MRCM_PHASE_COEF);
        TRYC(launch_check_K(v, s)); ++launches;
        TRYC(launch_cell_resist(v, s)); ++launches;
        TRYC(launch_seg_beta(v, s)); launches += P.nseg > 0;
        TRYC(launch_face_coef(v, s)); ++launches;
    }
    if (!merges_only && P.dim != 3) {
        PhaseScope ps(c, MRCM_PHASE_LEAF_BUILD);
        TRYC(launch_leaf_build(v, P.max_m_leaf, s)); ++launches;
    }
    {
        const PhaseHook hook{c, phase_begin, phase_end};
        for (int h = 1; h <= P.height; ++h) {
            const bool fp32 = v.mixed && P.level_max_g2[h - 1] <= c->mixed_split;
            const MergeTune tune = c->tune.empty() ? MergeTune{} : c->tune[h - 1];
            TRYC(launch_merge_build(v, P.level_first[h - 1], P.level_count[h - 1], P.level_max_g2[h - 1],
                                    P.level_max_m[h - 1], fp32, level_factor(c, h), tune, c->gj_scratch,
                                    c->gj_barrier, s, &launches, hook));
        }
    }
    return MRCM_OK;
}

int mrcm_build_basis(mrcm_ctx* c) {
    if (!c) return MRCM_ERR_INVALID_ARG;
    c->built = false;
    c->solved = false;
    int launches = 0;
    if (c->build_exec == nullptr || c->build_timing != c->timing) {
        c->ev_used = 0;
        if (capture_graph(c, &c->build_exec, [&] { return enqueue_build(c, launches); })) {
            c->build_timing = c->timing;
            c->build_ev_used = c->ev_used;
            c->launches_build = launches;
            c->solve_key[0] = nullptr;          // the solve graph's event pairs follow these
        }
    }
    if (c->use_graphs && c->build_exec != nullptr && c->build_timing == c->timing) {
        c->ev_used = c->build_ev_used;
        TRYC(cudaGraphLaunch(c->build_exec, c->stream));
        ++c->graph_replays;
    } else {
        c->ev_used = 0;
        TRY(enqueue_build(c, launches));
        c->launches_build = launches;
    }
    TRY(read_status(c));
    c->built = true;
    return MRCM_OK;
}

// One pass of the solve phase for the data (q, bc) -- or, with bc == nullptr
// and with_sadj, for a refinement residual: leaf particular solutions,
// up-sweep and root, down-sweep, leaf pressures, interface unknowns.
static int solve_pass(mrcm_ctx* c, const double* q, const double* bc, bool with_sadj, bool accumulate,
                      int& launches) {
    const Plan& P = c->P;
    const DevView& v = c->v;
    cudaStream_t s = c->stream;
    {
        PhaseScope ps(c, MRCM_PHASE_LEAF_PART);
        if (P.dim == 3) TRYC(launch_leaf3_particular(v, q, bc, with_sadj, s));
        else TRYC(launch_leaf_particular(v, q, bc, with_sadj, s));
        ++launches;
    }
    if (P.height > 0) {
        {
            PhaseScope ps(c, MRCM_PHASE_TREE_UP);
            TRYC(launch_tree_up(v, c->tree, c->tree_grid, c->gj_barrier, s));
            ++launches;
        }
        PhaseScope ps(c, MRCM_PHASE_TREE_DOWN);
        TRYC(launch_tree_down(v, c->tree, c->tree_grid, c->tree_scratch, c->gj_barrier, s));
        ++launches;
    }
    {
        PhaseScope ps(c, MRCM_PHASE_LEAF_PRESSURE);
        if (P.dim == 3) {
            TRYC(launch_leaf3_pressure(v, accumulate, s)); ++launches;
            TRYC(launch_lam_to_PU(v, accumulate, s)); launches += P.nseg > 0;
        } else {
            TRYC(launch_leaf_pressure(v, accumulate, s)); ++launches;
            TRYC(launch_lam_to_PU(v, accumulate, s)); launches += P.nseg > 0;
        }
    }
    return MRCM_OK;
}

// The launch sequence of mrcm_solve (no synchronisation).
static int enqueue_solve(mrcm_ctx* c, const double* q_dev, const double* bc_val_dev, double* p_dev, double* Fx_dev,
                         double* Fy_dev, double* Fz_dev, double* iface_dev, int& launches) {
    const Plan& P = c->P;
    const DevView& v = c->v;
    cudaStream_t s = c->stream;
    launches = 0;
    TRYC(cudaMemsetAsync(v.status, 0, sizeof(int), s));
    const int steps = c->refine_steps, nres = steps + (c->refine_check ? 1 : 0);
    if (nres > 0) TRYC(cudaMemsetAsync(v.res_max, 0, sizeof(unsigned long long) * nres, s));
    if (P.pure_neumann) {
        // all-Neumann data must balance (Section 2: no solution otherwise)
        PhaseScope ps(c, MRCM_PHASE_FINISH);
        TRYC(launch_compat_check(v, q_dev, bc_val_dev, s));
        launches += 2;
    }
    TRY(solve_pass(c, q_dev, bc_val_dev, false, false, launches));
    for (int it = 0; it < steps; ++it) {
        {
            PhaseScope ps(c, MRCM_PHASE_RESIDUAL);
            if (P.dim == 3) TRYC(launch_residual3(v, q_dev, bc_val_dev, it, s));
            else TRYC(launch_residual(v, q_dev, bc_val_dev, it, s));
            launches += 1 + (P.nseg > 0);
        }
        TRY(solve_pass(c, v.rcell, nullptr, true, true, launches));
    }
    if (c->refine_check) {
        if (P.dim == 3) TRYC(launch_residual3(v, q_dev, bc_val_dev, steps, s));
        else TRYC(launch_residual(v, q_dev, bc_val_dev, steps, s));
        launches += 1 + (P.nseg > 0);
    }
    {
        PhaseScope ps(c, MRCM_PHASE_FINISH);
        if (P.pure_neumann) {
            TRYC(launch_mean_shift(v, steps == 0 || !v.res_dd, s));
            launches += 2;
        }
        if (P.dim == 3) TRYC(launch_face_fluxes3(v, bc_val_dev, p_dev, Fx_dev, Fy_dev, Fz_dev, iface_dev, s));
        else TRYC(launch_face_fluxes(v, bc_val_dev, p_dev, Fx_dev, Fy_dev, iface_dev, steps == 0, s));
        ++launches;
    }
    return MRCM_OK;
}

int mrcm_solve(mrcm_ctx* c, const double* q_dev, const double* bc_val_dev, double* p_dev, double* Fx_dev,
               double* Fy_dev, double* Fz_dev, double* iface_dev) {
    if (!c) return MRCM_ERR_INVALID_ARG;
    if (!c->built) return MRCM_ERR_NOT_BUILT;
    if (!q_dev || !bc_val_dev || !p_dev || !Fx_dev || !Fy_dev) return MRCM_ERR_INVALID_ARG;
    // Fz in 3D only
    if (c->P.dim == 3 ? !Fz_dev : (Fz_dev != nullptr)) return MRCM_ERR_INVALID_ARG;
    // keep the build's event pairs, reuse the solve's
    while (c->ev_used > 0 && c->ev_phase[c->ev_used - 1] >= MRCM_PHASE_LEAF_PART &&
           c->ev_phase[c->ev_used - 1] <= MRCM_PHASE_FINISH)
        --c->ev_used;
    const int ev_begin = c->ev_used;
    const void* key[9] = {q_dev, bc_val_dev, p_dev, Fx_dev, Fy_dev, iface_dev, Fz_dev,
                          reinterpret_cast<const void*>(
                              (long long)((c->refine_steps * 2 + c->refine_check) * 2 + c->v.res_dd) + 1),
                          reinterpret_cast<const void*>((long long)(c->timing ? 2 : 1) + 4 * (long long)ev_begin)};
    int launches = 0;
    if (c->solve_exec == nullptr || std::memcmp(key, c->solve_key, sizeof(key)) != 0) {
        if (capture_graph(c, &c->solve_exec, [&] {
                return enqueue_solve(c, q_dev, bc_val_dev, p_dev, Fx_dev, Fy_dev, Fz_dev, iface_dev, launches);
            })) {
            std::memcpy(c->solve_key, key, sizeof(key));
            c->solve_ev_begin = ev_begin;
            c->solve_ev_used = c->ev_used;
            c->solve_launches = launches;
        } else {
            c->solve_key[0] = nullptr;
        }
    }
    if (c->use_graphs && c->solve_exec != nullptr && std::memcmp(key, c->solve_key, sizeof(key)) == 0) {
        c->ev_used = c->solve_ev_used;
        c->launches_solve = c->solve_launches;
        TRYC(cudaGraphLaunch(c->solve_exec, c->stream));
        ++c->graph_replays;
    } else {
        c->ev_used = ev_begin;
        TRY(enqueue_solve(c, q_dev, bc_val_dev, p_dev, Fx_dev, Fy_dev, Fz_dev, iface_dev, launches));
        c->launches_solve = launches;
    }
    c->hist_count = c->refine_steps + (c->refine_check ? 1 : 0);
    TRY(read_status(c));
    c->solved = true;
    return MRCM_OK;
}

int mrcm_autotune(mrcm_ctx* c, int reps) {
    if (!c || reps < 1 || reps > 100) return MRCM_ERR_INVALID_ARG;
    if (!c->built) return MRCM_ERR_NOT_BUILT;
    const Plan& P = c->P;
    std::vector<MergeTune> tune(P.height);
    for (int h = 1; h <= P.height; ++h) {
        const bool fp32 = c->v.mixed && P.level_max_g2[h - 1] <= c->mixed_split;
        TRYC(tune_merge_level(c->v, P.level_first[h - 1], P.level_count[h - 1], P.level_max_g2[h - 1],
                              P.level_max_m[h - 1], fp32, level_factor(c, h), c->gj_scratch, c->gj_barrier,
                              c->stream, reps, &tune[h - 1]));
    }
    TRY(read_status(c));
    c->tune = tune;
    // the captured build graph holds the previous launch shapes
    if (c->build_exec) cudaGraphExecDestroy(c->build_exec);
    c->build_exec = nullptr;
    return MRCM_OK;
}

int mrcm_tune_info(const mrcm_ctx* c, int height, int out[3]) {
    if (!c || !out || height < 1 || height > c->P.height) return MRCM_ERR_INVALID_ARG;
    const MergeTune t = c->tune.empty() ? MergeTune{} : c->tune[height - 1];
    out[0] = t.sweep_per_sm;
    out[1] = t.x_rows;
    out[2] = t.r_tile;
    return MRCM_OK;
}

int mrcm_set_mixed_split(mrcm_ctx* c, int max_g2_fp32) {
    if (!c || max_g2_fp32 < 0) return MRCM_ERR_INVALID_ARG;
    if (!c->v.mixed) return MRCM_ERR_UNSUPPORTED;
    if (max_g2_fp32 == c->mixed_split) return MRCM_OK;
    c->mixed_split = max_g2_fp32;
    c->built = false;
    c->solved = false;
    // the captured build graph holds the old per-level choice
    TRYC(cudaStreamSynchronize(c->stream));
    if (c->build_exec) cudaGraphExecDestroy(c->build_exec);
    c->build_exec = nullptr;
    return MRCM_OK;
}

int mrcm_set_mixed_leaves(mrcm_ctx* c, int fp32) {
    if (!c || (fp32 != 0 && fp32 != 1)) return MRCM_ERR_INVALID_ARG;
    if (!c->v.mixed || (c->P.dim == 3 && fp32)) return MRCM_ERR_UNSUPPORTED;
    if (fp32 == c->v.leaf32) return MRCM_OK;
    TRYC(cudaStreamSynchronize(c->stream));
    c->v.leaf32 = fp32;
    c->built = false;
    c->solved = false;
    // both captured graphs launch the leaf kernels of the old precision
    if (c->build_exec) cudaGraphExecDestroy(c->build_exec);
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    c->build_exec = c->solve_exec = nullptr;
    c->solve_key[0] = nullptr;
    return MRCM_OK;
}

int mrcm_set_root_form(mrcm_ctx* c, int form) {
    if (!c || (form != MRCM_ROOT_FACTOR && form != MRCM_ROOT_INVERSE && form != MRCM_ROOT_AUTO))
        return MRCM_ERR_INVALID_ARG;
    if (form == c->root_form) return MRCM_OK;
    TRYC(cudaStreamSynchronize(c->stream));
    c->root_form = form;
    c->built = false;
    c->solved = false;
    set_tree_forms(c);
    // both captured graphs hold the old form (the build's launches, the
    // solve sweeps' level table)
    if (c->build_exec) cudaGraphExecDestroy(c->build_exec);
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    c->build_exec = c->solve_exec = nullptr;
    c->solve_key[0] = nullptr;
    return MRCM_OK;
}

int mrcm_set_wait_limit(mrcm_ctx* c, long long polls) {
    if (!c) return MRCM_ERR_INVALID_ARG;
    const long long lim = polls >= 0 ? polls : kDefaultSpinLimit;
    if (lim == c->v.spin_limit) return MRCM_OK;
    c->v.spin_limit = lim;
    // the captured graphs hold the old limit in their launch arguments
    TRYC(cudaStreamSynchronize(c->stream));
    if (c->build_exec) cudaGraphExecDestroy(c->build_exec);
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    c->build_exec = c->solve_exec = nullptr;
    c->solve_key[0] = nullptr;
    return MRCM_OK;
}

// ---- learned basis surrogate ----------------------------------------------
int mrcm_interior_leaves(const mrcm_ctx* c, int* ids, int cap) {
    if (!c || cap < 0 || (cap > 0 && !ids)) return MRCM_ERR_INVALID_ARG;
    if (c->P.dim == 3) return MRCM_ERR_UNSUPPORTED;
    int n = 0;
    for (int id = 0; id < c->P.nleaf; ++id) {
        const LeafDesc& L = c->P.leaves[id];
        if (L.w != kMaxLeafSide || L.h != kMaxLeafSide || L.m != 16) continue;
        if (L.side_off[0] < 0 || L.side_off[1] < 0 || L.side_off[2] < 0 || L.side_off[3] < 0) continue;
        if (n < cap) ids[n] = id;
        ++n;
    }
    return n;
}

static int surrogate_ready(mrcm_ctx* c, const int* ids, int count) {
    if (!c || !ids || count < 0) return MRCM_ERR_INVALID_ARG;
    if (c->P.dim == 3 || c->P.max_m_leaf > 16) return MRCM_ERR_UNSUPPORTED;
    return MRCM_OK;
}

int mrcm_leaf_fields(mrcm_ctx* c, const int* ids, int count, float* psi) {
    TRY(surrogate_ready(c, ids, count));
    if (!psi) return MRCM_ERR_INVALID_ARG;
    if (!c->built) return MRCM_ERR_NOT_BUILT;
    TRYC(cudaMemsetAsync(c->v.status, 0, sizeof(int), c->stream));
    TRYC(launch_leaf_fields(c->v, ids, count, psi, c->stream));
    return read_status(c);
}

int mrcm_leaf_patches(mrcm_ctx* c, const int* ids, int count, void* x) {
    TRY(surrogate_ready(c, ids, count));
    if (!x) return MRCM_ERR_INVALID_ARG;
    TRYC(cudaMemsetAsync(c->v.status, 0, sizeof(int), c->stream));
    TRYC(launch_leaf_patches(c->v, ids, count, x, c->stream));
    return read_status(c);
}

int mrcm_leaf_gate(mrcm_ctx* c, const int* ids, int count, const float* psi, double* res) {
    TRY(surrogate_ready(c, ids, count));
    if (!psi || !res) return MRCM_ERR_INVALID_ARG;
    TRYC(cudaMemsetAsync(c->v.status, 0, sizeof(int), c->stream));
    TRYC(launch_leaf_gate(c->v, ids, count, psi, res, c->stream));
    return read_status(c);
}

int mrcm_leaf_apply(mrcm_ctx* c, const int* ids, int count, const float* psi, const double* res, double tau,
                    int* accepted) {
    TRY(surrogate_ready(c, ids, count));
    if (!psi || !res || !accepted) return MRCM_ERR_INVALID_ARG;
    if (!c->built) return MRCM_ERR_NOT_BUILT;
    TRYC(cudaMemsetAsync(c->v.status, 0, sizeof(int), c->stream));
    TRYC(launch_leaf_apply(c->v, ids, count, psi, res, tau, accepted, c->stream));
    TRY(read_status(c));
    // the merged maps above the changed leaves
    c->built = false;
    c->solved = false;
    int launches = 0;
    TRY(enqueue_build(c, launches, true));
    TRY(read_status(c));
    c->built = true;
    return MRCM_OK;
}

int mrcm_cnn_conv_forward(const void* x, int count, int cin, int cout, int pad, int relu, const void* w,
                          const float* b, void* y_bf16, float* y_f32, void* stream) {
    if (!x || !w || count < 0 || (!y_bf16 && !y_f32)) return MRCM_ERR_INVALID_ARG;
    if (count == 0) return MRCM_OK;
    const cudaError_t e = launch_conv_fwd(x, count, cin, cout, pad, relu, w, b, y_bf16, y_f32,
                                          static_cast<cudaStream_t>(stream));
    return e == cudaErrorInvalidValue ? MRCM_ERR_UNSUPPORTED : cuda_err(e);
}

int mrcm_cnn_conv_wgrad(const void* x, const void* dy, int count, int cin, int cout, int pad, float* dw, float* db,
                        void* stream) {
    if (!x || !dy || !dw || count < 0) return MRCM_ERR_INVALID_ARG;
    if (count == 0) return MRCM_OK;
    const cudaError_t e = launch_conv_wgrad(x, dy, count, cin, cout, pad, dw, db, static_cast<cudaStream_t>(stream));
    return e == cudaErrorInvalidValue ? MRCM_ERR_UNSUPPORTED : cuda_err(e);
}

int mrcm_cnn_flip_weights(const void* w, int cout, int cin, void* w2, void* stream) {
    if (!w || !w2 || cout < 1 || cin < 1) return MRCM_ERR_INVALID_ARG;
    return cuda_err(launch_flip_weights(w, cout, cin, w2, static_cast<cudaStream_t>(stream)));
}

int mrcm_cnn_relu_grad(const float* dpost, const void* y, long long n, int mask, void* dpre, void* stream) {
    if (!dpost || !dpre || n < 0 || (mask && !y)) return MRCM_ERR_INVALID_ARG;
    if (n == 0) return MRCM_OK;
    return cuda_err(launch_relu_grad(dpost, y, n, mask, dpre, static_cast<cudaStream_t>(stream)));
}

int mrcm_cnn_mse_grad(const float* pred, const float* target, int count, float* dpred, float* loss, void* stream) {
    if (!pred || !target || !dpred || !loss || count < 1) return MRCM_ERR_INVALID_ARG;
    return cuda_err(launch_mse_grad(pred, target, count, dpred, loss, static_cast<cudaStream_t>(stream)));
}

int mrcm_cnn_adam(float* p, const float* g, float* m1, float* m2, void* p_bf16, long long n, float lr, float beta1,
                  float beta2, float eps, int step, void* stream) {
    if (!p || !g || !m1 || !m2 || n < 0 || step < 1) return MRCM_ERR_INVALID_ARG;
    if (n == 0) return MRCM_OK;
    return cuda_err(launch_adam(p, g, m1, m2, p_bf16, n, lr, beta1, beta2, eps, step,
                                static_cast<cudaStream_t>(stream)));
}

int mrcm_set_refinement(mrcm_ctx* c, int steps, int check) {
    if (!c || steps < 0 || steps > kMaxRefine) return MRCM_ERR_INVALID_ARG;
    c->refine_steps = steps;
    c->refine_check = check ? 1 : 0;
    return MRCM_OK;
}

int mrcm_set_residual(mrcm_ctx* c, int dd) {
    if (!c || (dd != 0 && dd != 1)) return MRCM_ERR_INVALID_ARG;
    if (c->P.dim == 3 && dd) return MRCM_ERR_UNSUPPORTED;   // 3D residuals are FP64 only
    c->v.res_dd = dd;              // the solve graph is keyed by it
    return MRCM_OK;
}

int mrcm_residual_history(mrcm_ctx* c, double* out, int cap) {
    if (!c || !out || cap < 0) return MRCM_ERR_INVALID_ARG;
    if (!c->solved) return MRCM_ERR_NOT_BUILT;
    const int n = std::min(cap, c->hist_count);
    unsigned long long bits[kMaxRefine + 1];
    if (n > 0) {
        TRYC(cudaMemcpyAsync(bits, c->v.res_max, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost,
                             c->stream));
        TRYC(cudaStreamSynchronize(c->stream));
    }
    for (int k = 0; k < n; ++k) std::memcpy(&out[k], &bits[k], sizeof(double));
    return c->hist_count;
}

int mrcm_query(const mrcm_ctx* c, int what, long long* value) {
    if (!c || !value) return MRCM_ERR_INVALID_ARG;
    switch (what) {
        case MRCM_Q_WORKSPACE_BYTES: *value = (long long)c->bytes; return MRCM_OK;
        case MRCM_Q_KERNEL_LAUNCHES_BUILD: *value = c->launches_build; return MRCM_OK;
        case MRCM_Q_KERNEL_LAUNCHES_SOLVE: *value = c->launches_solve; return MRCM_OK;
        case MRCM_Q_GRAPH_REPLAYS: *value = c->graph_replays; return MRCM_OK;
        default: return plan_value(c->P, what, value, c->root_form);
    }
}

int mrcm_node_info(const mrcm_ctx* c, int node, int info[11]) {
    if (!c || !info || node < 0 || node >= (int)c->P.nodes.size()) return MRCM_ERR_INVALID_ARG;
    const Plan::Node& nd = c->P.nodes[node];
    info[0] = nd.height;
    info[1] = (int)nd.segs.size();
    info[2] = (int)nd.gamma.size();
    info[3] = nd.c1;
    info[4] = nd.c2;
    info[5] = nd.parent;
    info[6] = nd.leaf;
    for (int k = 0; k < 4; ++k) info[7 + k] = nd.box[k];
    return MRCM_OK;
}

int mrcm_node_segments(const mrcm_ctx* c, int node, int* seg_ids) {
    if (!c || !seg_ids || node < 0 || node >= (int)c->P.nodes.size()) return MRCM_ERR_INVALID_ARG;
    const std::vector<int>& s = c->P.nodes[node].segs;
    std::copy(s.begin(), s.end(), seg_ids);
    return MRCM_OK;
}

int mrcm_segment_info(const mrcm_ctx* c, int seg, int info[6]) {
    if (!c || !info || seg < 0 || seg >= c->P.nseg) return MRCM_ERR_INVALID_ARG;
    const Plan& P = c->P;
    info[0] = P.seg_axis[seg];
    info[1] = P.seg_line[seg];
    info[2] = P.seg_lo[seg];
    info[3] = P.seg_len[seg];
    info[4] = P.seg_a[seg];
    info[5] = P.seg_b[seg];
    return MRCM_OK;
}

int mrcm_node_operator(mrcm_ctx* c, int node, double* R_host, double* rbar_host) {
    if (!c || !R_host || node < 0 || node >= (int)c->P.nodes.size()) return MRCM_ERR_INVALID_ARG;
    if (!c->built) return MRCM_ERR_NOT_BUILT;
    if (rbar_host && !c->solved) return MRCM_ERR_NOT_BUILT;
    const long long m = (long long)c->P.nodes[node].segs.size();
    if (m > 0) {
        TRYC(cudaMemcpyAsync(R_host, c->v.R + c->P.node_R_off[node], sizeof(double) * m * m,
                             cudaMemcpyDeviceToHost, c->stream));
        if (rbar_host)
            TRYC(cudaMemcpyAsync(rbar_host, c->v.rbar + c->P.node_r_off[node], sizeof(double) * m,
                                 cudaMemcpyDeviceToHost, c->stream));
    }
    TRYC(cudaStreamSynchronize(c->stream));
    return MRCM_OK;
}

int mrcm_enable_timing(mrcm_ctx* c, int on) {
    if (!c) return MRCM_ERR_INVALID_ARG;
    if (on && c->ev.empty()) {
        c->ev.assign(2 * kEventPairs, nullptr);
        c->ev_phase.assign(kEventPairs, 0);
        for (auto& e : c->ev) TRYC(cudaEventCreate(&e));
    }
    c->timing = on != 0;
    return MRCM_OK;
}

int mrcm_use_graphs(mrcm_ctx* c, int on) {
    if (!c) return MRCM_ERR_INVALID_ARG;
    c->use_graphs = on != 0;
    if (!c->use_graphs) {
        TRYC(cudaStreamSynchronize(c->stream));
        if (c->build_exec) cudaGraphExecDestroy(c->build_exec);
        if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
        c->build_exec = c->solve_exec = nullptr;
        c->solve_key[0] = nullptr;
    }
    return MRCM_OK;
}

int mrcm_phase_times(mrcm_ctx* c, double* ms) {
    if (!c || !ms) return MRCM_ERR_INVALID_ARG;
    TRYC(cudaStreamSynchronize(c->stream));
    for (int p = 0; p < MRCM_PHASE_COUNT; ++p) ms[p] = 0.0;
    for (int k = 0; k < c->ev_used; ++k) {
        float t = 0.f;
        TRYC(cudaEventElapsedTime(&t, c->ev[2 * k], c->ev[2 * k + 1]));
        ms[c->ev_phase[k]] += t;
    }
    return MRCM_OK;
}

int mrcm_check_reciprocal(const double* x_dev, double* r_dev, long long n, void* cuda_stream) {
    if (!x_dev || !r_dev || n < 0) return MRCM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = launch_reciprocal(x_dev, r_dev, n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MRCM_OK : MRCM_ERR_CUDA;
}

int mrcm_group_times(mrcm_ctx* c, int* phase, double* ms, int cap) {
    if (!c || cap < 0 || (cap > 0 && (!phase || !ms))) return MRCM_ERR_INVALID_ARG;
    TRYC(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < c->ev_used && k < cap; ++k) {
        float t = 0.f;
        TRYC(cudaEventElapsedTime(&t, c->ev[2 * k], c->ev[2 * k + 1]));
        phase[k] = c->ev_phase[k];
        ms[k] = t;
    }
    return c->ev_used;
}

int mrcm_phase_flops(const mrcm_ctx* c, double* flops) {
    if (!c || !flops) return MRCM_ERR_INVALID_ARG;
    const Plan& P = c->P;
    const int a = root_set(c->root_form);
    const double passes = 1.0 + c->refine_steps, f = a >= 0 ? 1.0 : 0.0;
    const int ai = a >= 0 ? a : 0;
    for (int p = 0; p < MRCM_PHASE_COUNT; ++p)
        flops[p] = P.phase_build[p] + f * P.root_build[ai][p] +
                   passes * (P.phase_pass[p] + f * P.root_pass[ai][p]);
    flops[MRCM_PHASE_RESIDUAL] = (c->refine_steps + (c->refine_check ? 1 : 0)) * P.residual_flops;
    flops[MRCM_PHASE_FINISH] = P.finish_flops;
    return MRCM_OK;
}

void mrcm_destroy(mrcm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->build_exec) cudaGraphExecDestroy(c->build_exec);
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

}  // extern "C"
