// Iterative refinement of the discrete MRCM solution and the final fluxes.
//
// The discrete solution is defined by Eqs. (11.2)-(14.2) of arXiv 2009.07965
// with lumped RT0.  With the skeleton face fluxes eliminated by the lumped
// Robin relation of Eq. (11.2),
//     F^a_e = rho^a_e (p_a - P_t + beta_t U_t),   F^b_e = rho^b_e (p_b - P_t - beta_t U_t),
// the unknowns are the cell pressures p and the interface pair (P_t, U_t),
// and the equations are
//     E_c   = sum of the outward fluxes of cell c - q_c          (Eq. 12.2)
//     E13_t = F^a_t + F^b_t                                        (Eq. 13.2)
//     E14_t = F^a_t - F^b_t - 2 |t| U_t                            (Eq. 14.2)
// A direct FP64 solve meets these only to the conditioning of the problem
// times the rounding unit.  The residual below is evaluated in double-double
// arithmetic (error-free TwoSum of Knuth and FMA-based TwoProd); the
// Recursive MRCM then solves for the correction with -E as data (cell source
// -E_c, interface rows sigma^a = -(E13 + E14)/2, sigma^b = -(E13 - E14)/2 in
// the lambda form), which is Wilkinson's iterative refinement.  Coefficients
// are those of the face-coefficient kernel, evaluated in a fixed order.
#include "mrcm_internal.h"

namespace mrcm {
namespace {

// Unnormalised double-double pairs (hi + lo): the high parts are combined
// with the error-free TwoSum / FMA TwoProd, the low parts are summed in FP64;
// the represented value is exact to O(u^2) of the magnitudes involved, which
// is all a residual needs, at a third of the operations of normalised
// double-double arithmetic.
__device__ __forceinline__ DD dd_sub_u(DD x, DD y) {
    DD s = dd_two_sum(x.h, -y.h);
    s.l += x.l - y.l;
    return s;
}
__device__ __forceinline__ DD dd_scale_u(DD d, double c) {
    const double p = c * d.h;
    return {p, fma(c, d.l, fma(c, d.h, -p))};
}
__device__ __forceinline__ DD dd_acc_u(DD sum, DD x) {
    DD s = dd_two_sum(sum.h, x.h);
    s.l += sum.l + x.l;
    return s;
}

__device__ __forceinline__ DD state_p(const DevView& v, long long c) { return {v.p_hi[c], v.p_lo[c]}; }
__device__ __forceinline__ DD seg_lam(const DevView& v, int t, int side_b) {
    const double2 x = v.seg_lam_dd[2 * t + side_b];
    return {x.x, x.y};
}

// Largest |x| over the CTA, one atomic per CTA (|x| >= 0: the IEEE bit
// pattern orders like the value).
__device__ __forceinline__ void block_record_max(unsigned long long* slot, double x) {
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
        if (threadIdx.x == 0 && b > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(b));
    }
}

// Outward flux of a cell through one face: coef (pc - pn) for an interior
// face (pn the neighbour), coef (pc - lambda) for a skeleton face (lambda
// the Robin datum of the cell's side), coef (pc - g) for a Dirichlet face.
__device__ __forceinline__ DD face_out_u(DD pc, DD pn, double coef) { return dd_scale_u(dd_sub_u(pc, pn), coef); }

// One face of cell c: its outward flux in the residual sum.  lower: the cell
// lies below / left of the face (side a of a skeleton segment).
__device__ __forceinline__ DD cell_face(const DevView& v, const double* bc_val, int dirichlet, bool boundary,
                                        int seg, bool lower, double coef, double area, DD pc, long long nb,
                                        long long bc_index) {
    if (boundary) {
        const double g = bc_val[bc_index];
        if (dirichlet) return face_out_u(pc, DD{g, 0.0}, coef);
        return dd_two_prod(area, g);                 // Neumann: |e| g_N outward
    }
    if (seg >= 0) return face_out_u(pc, seg_lam(v, seg, lower ? 0 : 1), coef);
    return face_out_u(pc, state_p(v, nb), coef);
}

__global__ void __launch_bounds__(256) residual_cells_kernel(DevView v, const double* __restrict__ q,
                                                             const double* __restrict__ bc_val, int step) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (c < v.ncell) {
        const GridDesc& G = v.grids[grid_of<0>(v, c)];
        int i, j;
        udivmod(c - G.c0, G.nx, j, i);
        const DD pc = state_p(v, c);
        const long long fx = G.fx0 + i + (long long)(G.nx + 1) * j;
        const long long fy = G.fy0 + i + (long long)G.nx * j;
        const long long b0 = G.b0;
        DD E = dd_two_sum(0.0, -q[c]);
        E = dd_acc_u(E, cell_face(v, bc_val, G.bc[0], i == 0, i > 0 ? v.xface_seg[fx] : -1, false, v.cxU[fx], G.hy,
                                  pc, c - 1, b0 + j));
        E = dd_acc_u(E, cell_face(v, bc_val, G.bc[1], i == G.nx - 1, i < G.nx - 1 ? v.xface_seg[fx + 1] : -1, true,
                                  v.cxL[fx + 1], G.hy, pc, c + 1, b0 + G.ny + j));
        E = dd_acc_u(E, cell_face(v, bc_val, G.bc[2], j == 0, j > 0 ? v.yface_seg[fy] : -1, false, v.cyU[fy], G.hx,
                                  pc, c - G.nx, b0 + 2 * G.ny + i));
        E = dd_acc_u(E, cell_face(v, bc_val, G.bc[3], j == G.ny - 1, j < G.ny - 1 ? v.yface_seg[fy + G.nx] : -1,
                                  true, v.cyL[fy + G.nx], G.hx, pc, c + G.nx, b0 + 2 * G.ny + G.nx + i));
        e = E.h + E.l;
        v.rcell[c] = -e;
    }
    block_record_max(v.res_max + step, e);
}

__global__ void __launch_bounds__(128) residual_segments_kernel(DevView v, int step) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double E13 = 0.0, E14 = 0.0;
    if (t < v.nseg) {
        const int axis = v.seg_axis[t], line = v.seg_line[t], lo = v.seg_lo[t], len = v.seg_len[t];
        const GridDesc& G = v.grids[v.seg_grid[t]];
        const DD la = seg_lam(v, t, 0), lb = seg_lam(v, t, 1);
        DD Fa = {0.0, 0.0}, Fb = {0.0, 0.0};
        for (int e = 0; e < len; ++e) {
            long long ca, cb, f;
            double ra, rb;
            if (axis == 0) {
                const int j = lo + e;
                ca = G.c0 + (long long)j * G.nx + line - 1;
                cb = ca + 1;
                f = G.fx0 + line + (long long)(G.nx + 1) * j;
                ra = v.cxL[f];
                rb = v.cxU[f];
            } else {
                const int i = lo + e;
                ca = G.c0 + (long long)(line - 1) * G.nx + i;
                cb = ca + G.nx;
                f = G.fy0 + i + (long long)G.nx * line;
                ra = v.cyL[f];
                rb = v.cyU[f];
            }
            Fa = dd_acc_u(Fa, face_out_u(state_p(v, ca), la, ra));
            Fb = dd_acc_u(Fb, face_out_u(state_p(v, cb), lb, rb));
        }
        const double length = len * (axis == 0 ? G.hy : G.hx);
        const DD two_u = dd_scale_u(DD{v.segU[t], v.segU_lo[t]}, 2.0 * length);
        const DD e13 = dd_acc_u(Fa, Fb);
        const DD e14 = dd_sub_u(dd_sub_u(Fa, Fb), two_u);
        E13 = e13.h + e13.l;
        E14 = e14.h + e14.l;
        // lambda-form rows: row_a + row_b = Eq. 13.2, row_a - row_b = Eq. 14.2
        v.sadj[v.seg_lam_a[t]] = -0.5 * (E13 + E14);
        v.sadj[v.seg_lam_b[t]] = -0.5 * (E13 - E14);
    }
    block_record_max(v.res_max + step, fmax(fabs(E13), fabs(E14)));
}

// The same residuals in plain FP64 (the state's pairs rounded to double):
// three operations per face instead of nineteen.  Enough for refinement to
// a tolerance well above the FP64 rounding level (the mixed form's 1e-8);
// refinement to the rounding level itself needs the double-double kernels.
__global__ void __launch_bounds__(256) residual_cells_fp64_kernel(DevView v, const double* __restrict__ q,
                                                                  const double* __restrict__ bc_val, int step) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (c < v.ncell) {
        const GridDesc& G = v.grids[grid_of<0>(v, c)];
        int i, j;
        udivmod(c - G.c0, G.nx, j, i);
        const double pc = v.p_hi[c] + v.p_lo[c];
        const long long fx = G.fx0 + i + (long long)(G.nx + 1) * j;
        const long long fy = G.fy0 + i + (long long)G.nx * j;
        const long long b0 = G.b0;
        // outward flux of the cell through one face
        auto face = [&](int dirichlet, bool boundary, int seg, bool lower, double coef, double area, long long nb,
                        long long bc_index) -> double {
            if (boundary) {
                const double g = bc_val[bc_index];
                return dirichlet ? coef * (pc - g) : area * g;
            }
            if (seg >= 0) {
                const double2 l = v.seg_lam_dd[2 * seg + (lower ? 0 : 1)];
                return coef * (pc - (l.x + l.y));
            }
            return coef * (pc - (v.p_hi[nb] + v.p_lo[nb]));
        };
        double E = -q[c];
        E += face(G.bc[0], i == 0, i > 0 ? v.xface_seg[fx] : -1, false, v.cxU[fx], G.hy, c - 1, b0 + j);
        E += face(G.bc[1], i == G.nx - 1, i < G.nx - 1 ? v.xface_seg[fx + 1] : -1, true, v.cxL[fx + 1], G.hy, c + 1,
                  b0 + G.ny + j);
        E += face(G.bc[2], j == 0, j > 0 ? v.yface_seg[fy] : -1, false, v.cyU[fy], G.hx, c - G.nx,
                  b0 + 2 * G.ny + i);
        E += face(G.bc[3], j == G.ny - 1, j < G.ny - 1 ? v.yface_seg[fy + G.nx] : -1, true, v.cyL[fy + G.nx], G.hx,
                  c + G.nx, b0 + 2 * G.ny + G.nx + i);
        e = E;
        v.rcell[c] = -e;
    }
    block_record_max(v.res_max + step, e);
}

__global__ void __launch_bounds__(128) residual_segments_fp64_kernel(DevView v, int step) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double E13 = 0.0, E14 = 0.0;
    if (t < v.nseg) {
        const int axis = v.seg_axis[t], line = v.seg_line[t], lo = v.seg_lo[t], len = v.seg_len[t];
        const GridDesc& G = v.grids[v.seg_grid[t]];
        const double2 l2a = v.seg_lam_dd[2 * t], l2b = v.seg_lam_dd[2 * t + 1];
        const double la = l2a.x + l2a.y, lb = l2b.x + l2b.y;
        double Fa = 0.0, Fb = 0.0;
        for (int e = 0; e < len; ++e) {
            long long ca, cb, f;
            double ra, rb;
            if (axis == 0) {
                const int j = lo + e;
                ca = G.c0 + (long long)j * G.nx + line - 1;
                cb = ca + 1;
                f = G.fx0 + line + (long long)(G.nx + 1) * j;
                ra = v.cxL[f];
                rb = v.cxU[f];
            } else {
                const int i = lo + e;
                ca = G.c0 + (long long)(line - 1) * G.nx + i;
                cb = ca + G.nx;
                f = G.fy0 + i + (long long)G.nx * line;
                ra = v.cyL[f];
                rb = v.cyU[f];
            }
            Fa += ra * ((v.p_hi[ca] + v.p_lo[ca]) - la);
            Fb += rb * ((v.p_hi[cb] + v.p_lo[cb]) - lb);
        }
        const double length = len * (axis == 0 ? G.hy : G.hx);
        const double two_u = 2.0 * length * (v.segU[t] + v.segU_lo[t]);
        E13 = Fa + Fb;
        E14 = (Fa - Fb) - two_u;
        v.sadj[v.seg_lam_a[t]] = -0.5 * (E13 + E14);
        v.sadj[v.seg_lam_b[t]] = -0.5 * (E13 - E14);
    }
    block_record_max(v.res_max + step, fmax(fabs(E13), fabs(E14)));
}

// P = (lambda^a + lambda^b) / 2, U = (lambda^b - lambda^a) / (2 beta) into the
// refined state (set, or added in double-double), then the state's Robin
// data lambda^a = P - beta U, lambda^b = P + beta U in double-double.
__global__ void lam_to_PU_kernel(DevView v, bool accumulate) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.nseg) return;
    const double la = v.lam[v.seg_lam_a[t]], lb = v.lam[v.seg_lam_b[t]];
    const double beta = v.seg_beta[t];
    const double P = 0.5 * (la + lb);
    const double U = (lb - la) / (2.0 * beta);
    DD xp = {P, 0.0}, xu = {U, 0.0};
    if (accumulate) {
        xp = dd_add(DD{v.segP[t], v.segP_lo[t]}, xp);
        xu = dd_add(DD{v.segU[t], v.segU_lo[t]}, xu);
    }
    v.segP[t] = xp.h;
    v.segP_lo[t] = xp.l;
    v.segU[t] = xu.h;
    v.segU_lo[t] = xu.l;
    const DD bu = dd_mul_d(xu, beta);
    const DD lam_a = dd_add(xp, dd_neg(bu)), lam_b = dd_add(xp, bu);
    v.seg_lam_dd[2 * t] = make_double2(lam_a.h, lam_a.l);
    v.seg_lam_dd[2 * t + 1] = make_double2(lam_b.h, lam_b.l);
}

// Cell pressures and face fluxes (+axis direction) from the double-double
// state, each formed in double-double and rounded once.  Skeleton faces: the
// one-sided F^a = rho^a (p_a - lambda^a), F^b = -(rho^b (p_b - lambda^b))
// and their mean.
template <int kMode>
__global__ void face_flux_kernel(DevView v, const double* __restrict__ bc_val, double* __restrict__ p,
                                 double* __restrict__ Fx, double* __restrict__ Fy, double* __restrict__ iface) {
    const long long nxf = v.nxface, nyf = v.nyface;
    long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (f < v.ncell) p[f] = v.p_hi[f] + v.p_lo[f];
    if (f >= nxf + nyf) return;
    const bool xface = f < nxf;
    const long long fl = xface ? f : f - nxf;        // index in Fx or Fy (all grids)
    const GridDesc& G = v.grids[xface ? grid_of<1>(v, fl) : grid_of<2>(v, fl)];
    double F, fa = 0.0, fb = 0.0;
    bool skel = false;
    int axis, line, k;
    if (xface) { axis = 0; udivmod(fl - G.fx0, G.nx + 1, k, line); }
    else { axis = 1; udivmod(fl - G.fy0, G.nx, line, k); }
    const int nline = axis == 0 ? G.nx : G.ny;
    const double* cL = axis == 0 ? v.cxL : v.cyL;
    const double* cU = axis == 0 ? v.cxU : v.cyU;
    // cells below / above the face
    const long long cb = G.c0 + (axis == 0 ? (long long)k * G.nx + line : (long long)line * G.nx + k);
    const long long ca = axis == 0 ? cb - 1 : cb - G.nx;
    const double area = axis == 0 ? G.hy : G.hx;
    const double* bv = bc_val + G.b0;
    // kMode 1: a state without low parts (no refinement step), plain FP64;
    // 2: a refined state rounded to FP64, plain FP64 (refinement to a
    // tolerance above the rounding level: FP64 residuals); 0: the state's
    // double-double pairs in double-double arithmetic
    auto pres = [&](long long c) -> double { return kMode == 2 ? v.p_hi[c] + v.p_lo[c] : v.p_hi[c]; };
    if (kMode != 0) {
        if (line == 0) {
            const double g = bv[axis == 0 ? k : 2 * G.ny + k];
            F = G.bc[2 * axis] ? -(cU[fl] * (pres(cb) - g)) : -(area * g);
        } else if (line == nline) {
            const double g = bv[axis == 0 ? G.ny + k : 2 * G.ny + G.nx + k];
            F = G.bc[2 * axis + 1] ? cL[fl] * (pres(ca) - g) : area * g;
        } else {
            const int t = axis == 0 ? v.xface_seg[fl] : v.yface_seg[fl];
            if (t >= 0) {
                const double2 la = v.seg_lam_dd[2 * t], lb = v.seg_lam_dd[2 * t + 1];
                const double da = cL[fl] * (pres(ca) - (la.x + la.y));
                const double db = cU[fl] * (pres(cb) - (lb.x + lb.y));
                fa = da;
                fb = -db;
                F = 0.5 * (da - db);
                skel = true;
            } else {
                F = cL[fl] * (pres(ca) - pres(cb));
            }
        }
    } else if (line == 0) {
        const double g = bv[axis == 0 ? k : 2 * G.ny + k];
        DD out = G.bc[2 * axis] ? face_out_u(state_p(v, cb), DD{g, 0.0}, cU[fl]) : DD{__dmul_rn(area, g), 0.0};
        F = -(out.h + out.l);
    } else if (line == nline) {
        const double g = bv[axis == 0 ? G.ny + k : 2 * G.ny + G.nx + k];
        DD out = G.bc[2 * axis + 1] ? face_out_u(state_p(v, ca), DD{g, 0.0}, cL[fl]) : DD{__dmul_rn(area, g), 0.0};
        F = out.h + out.l;
    } else {
        const int t = axis == 0 ? v.xface_seg[fl] : v.yface_seg[fl];
        if (t >= 0) {
            const DD da = face_out_u(state_p(v, ca), seg_lam(v, t, 0), cL[fl]);
            const DD db = face_out_u(state_p(v, cb), seg_lam(v, t, 1), cU[fl]);
            fa = da.h + da.l;
            fb = -(db.h + db.l);
            const DD dm = dd_sub_u(da, db);
            F = 0.5 * (dm.h + dm.l);
            skel = true;
        } else {
            const DD d = face_out_u(state_p(v, ca), state_p(v, cb), cL[fl]);
            F = d.h + d.l;
        }
    }
    if (xface) {
        Fx[fl] = F;
        if (iface) {
            iface[fl] = skel ? fa : F;
            iface[nxf + fl] = skel ? fb : F;
        }
    } else {
        Fy[fl] = F;
        if (iface) {
            iface[2 * nxf + fl] = skel ? fa : F;
            iface[2 * nxf + nyf + fl] = skel ? fb : F;
        }
    }
}

// Compatibility of all-Neumann data: the sources must balance the boundary
// outflow, sum_c q_c = sum_e |e| g_N (otherwise the problem has no
// solution).  Each of kCompatBlocks CTAs sums its share of
// q_c - (outflow of the boundary faces) in double-double (error-free
// TwoSum / TwoProd) and of the magnitudes in FP64; one CTA then adds the
// partials in a fixed order and sets kStatusInconsistent when
// |sum| > kCompatTol * (sum of magnitudes).  Partials in v.red[256, 1024).
constexpr int kCompatBlocks = 256;
__global__ void __launch_bounds__(256) compat_partial_kernel(DevView v, const double* __restrict__ q,
                                                             const double* __restrict__ bc_val) {
    __shared__ double sh_h[256], sh_l[256], sh_a[256];
    // all-Neumann problems: single-grid contexts only
    const GridDesc& G = v.grids[0];
    const long long n = v.ncell, nb = v.nbc;
    DD acc = {0.0, 0.0};
    double mag = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n + nb; i += stride) {
        const double val = i < n ? q[i] : bc_val[i - n];
        // zeros (most cells of a point-source problem) are skipped on the
        // bit pattern: an FP64 compare would cost a full FP64 instruction
        if (((unsigned long long)__double_as_longlong(val) << 1) == 0ull) continue;
        DD x;
        if (i < n) {
            x = {val, 0.0};
        } else {
            // face area of the boundary value's side (2D: x sides, then y
            // sides; 3D: x, y, z sides of ny nz, nx nz, nx ny faces each)
            double area;
            const long long b = i - n;
            if (v.dim == 3) {
                const Grid3& H = v.g3;
                const long long sx = (long long)H.ny * H.nz, sy = (long long)H.nx * H.nz;
                area = b < 2 * sx ? H.hy * H.hz : (b < 2 * sx + 2 * sy ? H.hx * H.hz : H.hx * H.hy);
            } else {
                area = b < 2LL * G.ny ? G.hy : G.hx;
            }
            x = dd_neg(dd_two_prod(area, val));
        }
        acc = dd_add(acc, x);
        mag += fabs(x.h);
    }
    sh_h[threadIdx.x] = acc.h;
    sh_l[threadIdx.x] = acc.l;
    sh_a[threadIdx.x] = mag;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const DD y = dd_add(DD{sh_h[threadIdx.x], sh_l[threadIdx.x]},
                                DD{sh_h[threadIdx.x + w], sh_l[threadIdx.x + w]});
            sh_h[threadIdx.x] = y.h;
            sh_l[threadIdx.x] = y.l;
            sh_a[threadIdx.x] += sh_a[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        v.red[256 + 2 * blockIdx.x] = sh_h[0];
        v.red[256 + 2 * blockIdx.x + 1] = sh_l[0];
        v.red[768 + blockIdx.x] = sh_a[0];
    }
}
__global__ void __launch_bounds__(kCompatBlocks) compat_final_kernel(DevView v) {
    __shared__ double sh_h[kCompatBlocks], sh_l[kCompatBlocks], sh_a[kCompatBlocks];
    const int b = threadIdx.x;
    sh_h[b] = v.red[256 + 2 * b];
    sh_l[b] = v.red[256 + 2 * b + 1];
    sh_a[b] = v.red[768 + b];
    __syncthreads();
    for (int w = kCompatBlocks / 2; w > 0; w >>= 1) {
        if (b < w) {
            const DD y = dd_add(DD{sh_h[b], sh_l[b]}, DD{sh_h[b + w], sh_l[b + w]});
            sh_h[b] = y.h;
            sh_l[b] = y.l;
            sh_a[b] += sh_a[b + w];
        }
        __syncthreads();
    }
    if (b == 0 && !(fabs(sh_h[0] + sh_l[0]) <= kCompatTol * sh_a[0])) atomicOr(v.status, kStatusInconsistent);
}

}  // namespace

cudaError_t launch_compat_check(const DevView& v, const double* q, const double* bc_val, cudaStream_t s) {
    compat_partial_kernel<<<kCompatBlocks, 256, 0, s>>>(v, q, bc_val);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    compat_final_kernel<<<1, kCompatBlocks, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_residual(const DevView& v, const double* q, const double* bc_val, int step,
                            cudaStream_t s) {
    const long long n = v.ncell;
    if (v.res_dd)
        residual_cells_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, q, bc_val, step);
    else
        residual_cells_fp64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, q, bc_val, step);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || v.nseg == 0) return e;
    if (v.res_dd)
        residual_segments_kernel<<<(v.nseg + 127) / 128, 128, 0, s>>>(v, step);
    else
        residual_segments_fp64_kernel<<<(v.nseg + 127) / 128, 128, 0, s>>>(v, step);
    return cudaGetLastError();
}

cudaError_t launch_lam_to_PU(const DevView& v, bool accumulate, cudaStream_t s) {
    if (v.nseg == 0) return cudaSuccess;
    lam_to_PU_kernel<<<(v.nseg + 127) / 128, 128, 0, s>>>(v, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_face_fluxes(const DevView& v, const double* bc_val, double* p, double* Fx,
                               double* Fy, double* iface, bool plain, cudaStream_t s) {
    const long long nf = v.nxface + v.nyface;
    if (plain)
        face_flux_kernel<1><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(v, bc_val, p, Fx, Fy, iface);
    else if (!v.res_dd)
        face_flux_kernel<2><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(v, bc_val, p, Fx, Fy, iface);
    else
        face_flux_kernel<0><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(v, bc_val, p, Fx, Fy, iface);
    return cudaGetLastError();
}

}  // namespace mrcm
