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

// p_c - P + s * beta U  (s = +1: side a, s = -1: side b), as a double-double
__device__ __forceinline__ DD robin_gap(DD pc, DD P, DD bu, double sgn) {
    const DD x = dd_add(pc, dd_neg(P));
    return dd_add(x, sgn > 0 ? bu : dd_neg(bu));
}

__device__ __forceinline__ DD state_p(const DevView& v, long long c) { return {v.p_hi[c], v.p_lo[c]}; }
__device__ __forceinline__ DD state_P(const DevView& v, int t) { return {v.segP[t], v.segP_lo[t]}; }
__device__ __forceinline__ DD state_bu(const DevView& v, int t) {
    return dd_mul_d(DD{v.segU[t], v.segU_lo[t]}, v.seg_beta[t]);
}

__device__ __forceinline__ void record_max(unsigned long long* slot, double a) {
    // |a| >= 0: the IEEE bit pattern orders like the value
    atomicMax(slot, (unsigned long long)__double_as_longlong(fabs(a)));
}

// Outward flux of cell c through one face, double-double.
// kind: 0 interior (coef T, neighbour cell n), 1 skeleton (coef rho, segment
// t, sgn = +1 when the cell is side a), 2 Dirichlet (coef tau, value g),
// 3 Neumann (|e| g).
__device__ __forceinline__ DD face_out(const DevView& v, int kind, double coef, DD pc, long long n, int t,
                                       double sgn, double g) {
    if (kind == 0) return dd_mul_d(dd_add(pc, dd_neg(state_p(v, n))), coef);
    if (kind == 1) return dd_mul_d(robin_gap(pc, state_P(v, t), state_bu(v, t), sgn), coef);
    if (kind == 2) return dd_mul_d(dd_add(pc, DD{-g, 0.0}), coef);
    return dd_two_prod(coef, g);
}

__global__ void residual_cells_kernel(DevView v, const double* __restrict__ q, const double* __restrict__ bc_val,
                                      int step) {
    const long long n = (long long)v.nx * v.ny;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = (int)(c % v.nx), j = (int)(c / v.nx);
    const DD pc = state_p(v, c);
    const long long fx = i + (long long)(v.nx + 1) * j;
    const long long fy = i + (long long)v.nx * j;
    DD E = {0.0, 0.0};
    // west
    if (i == 0) {
        E = dd_add(E, v.bc[0] ? face_out(v, 2, v.cxU[fx], pc, 0, 0, 0, bc_val[j])
                              : face_out(v, 3, v.hy, pc, 0, 0, 0, bc_val[j]));
    } else if (x_skeleton(v, i)) {
        E = dd_add(E, face_out(v, 1, v.cxU[fx], pc, 0, skeleton_segment(v, 0, i, j), -1.0, 0));
    } else {
        E = dd_add(E, face_out(v, 0, v.cxU[fx], pc, c - 1, 0, 0, 0));
    }
    // east
    if (i == v.nx - 1) {
        const double g = bc_val[v.ny + j];
        E = dd_add(E, v.bc[1] ? face_out(v, 2, v.cxL[fx + 1], pc, 0, 0, 0, g)
                              : face_out(v, 3, v.hy, pc, 0, 0, 0, g));
    } else if (x_skeleton(v, i + 1)) {
        E = dd_add(E, face_out(v, 1, v.cxL[fx + 1], pc, 0, skeleton_segment(v, 0, i + 1, j), 1.0, 0));
    } else {
        E = dd_add(E, face_out(v, 0, v.cxL[fx + 1], pc, c + 1, 0, 0, 0));
    }
    // south
    if (j == 0) {
        const double g = bc_val[2 * v.ny + i];
        E = dd_add(E, v.bc[2] ? face_out(v, 2, v.cyU[fy], pc, 0, 0, 0, g)
                              : face_out(v, 3, v.hx, pc, 0, 0, 0, g));
    } else if (y_skeleton(v, j)) {
        E = dd_add(E, face_out(v, 1, v.cyU[fy], pc, 0, skeleton_segment(v, 1, j, i), -1.0, 0));
    } else {
        E = dd_add(E, face_out(v, 0, v.cyU[fy], pc, c - v.nx, 0, 0, 0));
    }
    // north
    if (j == v.ny - 1) {
        const double g = bc_val[2 * v.ny + v.nx + i];
        E = dd_add(E, v.bc[3] ? face_out(v, 2, v.cyL[fy + v.nx], pc, 0, 0, 0, g)
                              : face_out(v, 3, v.hx, pc, 0, 0, 0, g));
    } else if (y_skeleton(v, j + 1)) {
        E = dd_add(E, face_out(v, 1, v.cyL[fy + v.nx], pc, 0, skeleton_segment(v, 1, j + 1, i), 1.0, 0));
    } else {
        E = dd_add(E, face_out(v, 0, v.cyL[fy + v.nx], pc, c + v.nx, 0, 0, 0));
    }
    E = dd_add(E, DD{-q[c], 0.0});
    const double e = dd_round(E);
    v.rcell[c] = -e;
    record_max(v.res_max + step, e);
}

__global__ void residual_segments_kernel(DevView v, int step) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.nseg) return;
    const int axis = v.seg_axis[t], line = v.seg_line[t], lo = v.seg_lo[t], len = v.seg_len[t];
    const DD P = state_P(v, t);
    const DD bu = state_bu(v, t);
    DD Fa = {0.0, 0.0}, Fb = {0.0, 0.0};
    for (int e = 0; e < len; ++e) {
        long long ca, cb, f;
        double ra, rb;
        if (axis == 0) {
            const int j = lo + e;
            ca = (long long)j * v.nx + line - 1;
            cb = ca + 1;
            f = line + (long long)(v.nx + 1) * j;
            ra = v.cxL[f];
            rb = v.cxU[f];
        } else {
            const int i = lo + e;
            ca = (long long)(line - 1) * v.nx + i;
            cb = ca + v.nx;
            f = i + (long long)v.nx * line;
            ra = v.cyL[f];
            rb = v.cyU[f];
        }
        Fa = dd_add(Fa, dd_mul_d(robin_gap(state_p(v, ca), P, bu, 1.0), ra));
        Fb = dd_add(Fb, dd_mul_d(robin_gap(state_p(v, cb), P, bu, -1.0), rb));
    }
    const double length = len * (axis == 0 ? v.hy : v.hx);
    const DD e13 = dd_add(Fa, Fb);
    DD e14 = dd_add(Fa, dd_neg(Fb));
    e14 = dd_add(e14, dd_neg(dd_mul_d(DD{v.segU[t], v.segU_lo[t]}, 2.0 * length)));
    const double E13 = dd_round(e13), E14 = dd_round(e14);
    // lambda-form rows: row_a + row_b = Eq. 13.2, row_a - row_b = Eq. 14.2
    v.sadj[v.seg_lam_a[t]] = -0.5 * (E13 + E14);
    v.sadj[v.seg_lam_b[t]] = -0.5 * (E13 - E14);
    record_max(v.res_max + step, E13);
    record_max(v.res_max + step, E14);
}

// P = (lambda^a + lambda^b) / 2, U = (lambda^b - lambda^a) / (2 beta)
__global__ void lam_to_PU_kernel(DevView v, bool accumulate) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.nseg) return;
    const double la = v.lam[v.seg_lam_a[t]], lb = v.lam[v.seg_lam_b[t]];
    const double P = 0.5 * (la + lb);
    const double U = (lb - la) / (2.0 * v.seg_beta[t]);
    if (accumulate) {
        const DD xp = dd_add(DD{v.segP[t], v.segP_lo[t]}, DD{P, 0.0});
        const DD xu = dd_add(DD{v.segU[t], v.segU_lo[t]}, DD{U, 0.0});
        v.segP[t] = xp.h;
        v.segP_lo[t] = xp.l;
        v.segU[t] = xu.h;
        v.segU_lo[t] = xu.l;
    } else {
        v.segP[t] = P;
        v.segP_lo[t] = 0.0;
        v.segU[t] = U;
        v.segU_lo[t] = 0.0;
    }
}

// Cell pressures and face fluxes (+axis direction) from the double-double
// state, each formed in double-double and rounded once.  Skeleton faces: the
// one-sided F^a = rho^a (p_a - P + beta U), F^b = -(rho^b (p_b - P - beta U))
// and their mean.
__global__ void face_flux_kernel(DevView v, const double* __restrict__ bc_val, double* __restrict__ p,
                                 double* __restrict__ Fx, double* __restrict__ Fy, double* __restrict__ iface) {
    const long long nxf = (long long)(v.nx + 1) * v.ny;
    const long long nyf = (long long)v.nx * (v.ny + 1);
    const long long ncell = (long long)v.nx * v.ny;
    long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (f < ncell) p[f] = dd_round(state_p(v, f));
    if (f >= nxf + nyf) return;
    const bool xface = f < nxf;
    const long long fl = xface ? f : f - nxf;
    double F, fa = 0.0, fb = 0.0;
    bool skel = false;
    int axis, line, k;
    if (xface) { axis = 0; line = (int)(fl % (v.nx + 1)); k = (int)(fl / (v.nx + 1)); }
    else { axis = 1; k = (int)(fl % v.nx); line = (int)(fl / v.nx); }
    const int nline = axis == 0 ? v.nx : v.ny;
    const double* cL = axis == 0 ? v.cxL : v.cyL;
    const double* cU = axis == 0 ? v.cxU : v.cyU;
    // cells below / above the face
    const long long cb = axis == 0 ? (long long)k * v.nx + line : (long long)line * v.nx + k;
    const long long ca = axis == 0 ? cb - 1 : cb - v.nx;
    const double area = axis == 0 ? v.hy : v.hx;
    if (line == 0) {
        const double g = bc_val[axis == 0 ? k : 2 * v.ny + k];
        const double out = v.bc[2 * axis] ? dd_round(dd_mul_d(dd_add(state_p(v, cb), DD{-g, 0.0}), cU[fl]))
                                          : __dmul_rn(area, g);
        F = -out;
    } else if (line == nline) {
        const double g = bc_val[axis == 0 ? v.ny + k : 2 * v.ny + v.nx + k];
        const double out = v.bc[2 * axis + 1]
                               ? dd_round(dd_mul_d(dd_add(state_p(v, ca), DD{-g, 0.0}), cL[fl]))
                               : __dmul_rn(area, g);
        F = out;
    } else if (axis == 0 ? x_skeleton(v, line) : y_skeleton(v, line)) {
        const int t = skeleton_segment(v, axis, line, k);
        const DD P = state_P(v, t), bu = state_bu(v, t);
        const DD da = dd_mul_d(robin_gap(state_p(v, ca), P, bu, 1.0), cL[fl]);
        const DD db = dd_mul_d(robin_gap(state_p(v, cb), P, bu, -1.0), cU[fl]);
        fa = dd_round(da);
        fb = -dd_round(db);
        F = __dmul_rn(0.5, dd_round(dd_add(da, dd_neg(db))));
        skel = true;
    } else {
        F = dd_round(dd_mul_d(dd_add(state_p(v, ca), dd_neg(state_p(v, cb))), cL[fl]));
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

}  // namespace

cudaError_t launch_residual(const DevView& v, const double* q, const double* bc_val, int step,
                            cudaStream_t s) {
    const long long n = (long long)v.nx * v.ny;
    residual_cells_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, q, bc_val, step);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || v.nseg == 0) return e;
    residual_segments_kernel<<<(v.nseg + 127) / 128, 128, 0, s>>>(v, step);
    return cudaGetLastError();
}

cudaError_t launch_lam_to_PU(const DevView& v, bool accumulate, cudaStream_t s) {
    if (v.nseg == 0) return cudaSuccess;
    lam_to_PU_kernel<<<(v.nseg + 127) / 128, 128, 0, s>>>(v, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_face_fluxes(const DevView& v, const double* bc_val, double* p, double* Fx,
                               double* Fy, double* iface, cudaStream_t s) {
    const long long nf = (long long)(v.nx + 1) * v.ny + (long long)v.nx * (v.ny + 1);
    face_flux_kernel<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(v, bc_val, p, Fx, Fy, iface);
    return cudaGetLastError();
}

}  // namespace mrcm
