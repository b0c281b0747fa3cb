// Learned basis surrogate (the grown form with a learned part).
//
// A leaf's basis responses (Eqs. 11Hhatbasisa / 11Hhatbasisb: one Robin
// response per interface segment, Section 3.1) are the fields
//     psi_s = A^-1 B e_s     (cell pressures for a unit Robin datum on s),
// and its Robin-to-flux map follows from them exactly: R = B^T psi - W.  A
// small convolutional network maps a leaf's permeability patch (with a
// one-cell halo, which fixes the Robin coefficients of its segments) and
// alpha to the 16 fields of a full interior leaf.  This file holds
//   - the training targets from the plain method (psi from the stored leaf
//     factors) and the network inputs (normalised log K patches);
//   - the network's hand-written BF16 kernels: 3 x 3 convolutions as
//     implicit GEMMs on the tensor cores (mma.sync m16n8k16, BF16 operands,
//     FP32 accumulation), their weight gradients, the input gradient (the
//     forward kernel on flipped weights), ReLU masks, the loss gradient and
//     Adam updates on FP32 master weights;
//   - the residual gate: ||A psi_s - B e_s|| / ||B e_s|| per leaf in FP64,
//     and the maps of the accepted leaves, R = B^T psi - W (symmetrised).
// Layouts: activations NHWC, [item][y][x][c]; weights [cout][ky][kx][cin]
// (so that row cout is contiguous in k = (ky 3 + kx) cin + ci); every
// output is 16 x 16 pixels (a full leaf).
#include <cuda_bf16.h>

#include "mrcm_internal.h"

namespace mrcm {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kS = 16;          // output side (a full leaf)
constexpr int kIn = kS + 2;     // input side with the halo

// ---------------------------------------------------------------------------
// Training targets and inputs from the plain method.
//
// psi[item][k][s] (float; cell k = i + 16 j, segment s fastest: the
// network's NHWC output layout) for the leaves ids[item]: column s of
// Z = L^-1 B scaled by D^-1, then the backward sweep L^T psi = y.
template <class TS>
__global__ void __launch_bounds__(128) leaf_fields_kernel(DevView v, const int* __restrict__ ids, int count,
                                                          float* __restrict__ psi) {
    __shared__ double ys[8][kS * kS];
    const int t = threadIdx.x & 15, slot = threadIdx.x >> 4;
    const int item = blockIdx.x * 8 + slot;
    if (item >= count) return;                        // uniform over the leaf's 16 lanes
    const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
    const int id = ids[item];
    if ((unsigned)id >= (unsigned)v.nleaf || v.leaves[id].m > 16) {
        if (t == 0) atomicOr(v.status, kStatusBadIndex);
        return;
    }
    const LeafDesc L = v.leaves[id];
    const int w = L.w, n = L.w * L.h, m = L.m;
    const TS* Lg = leaf_L<TS>(v) + L.L_off;
    const TS* Dg = Lg + (long long)n * kLeafThreads;
    const TS* Zg = leaf_Z<TS>(v) + L.Z_off;
    double* y = ys[slot];
    for (int s = 0; s < m; ++s) {
        for (int k = t; k < n; k += kLeafThreads) y[k] = (double)Zg[(long long)s * n + k] * (double)Dg[k];
        __syncwarp(mask);
        for (int k = n - 1; k >= 1; --k) {
            const double pk = y[k];
            if (t < min(w, k)) y[k - 1 - t] = fma(-(double)Lg[(long long)(k - 1 - t) * kLeafThreads + t], pk, y[k - 1 - t]);
            __syncwarp(mask);
        }
        for (int k = t; k < n; k += kLeafThreads) psi[((long long)item * (kS * kS) + k) * 16 + s] = (float)y[k];
        __syncwarp(mask);
    }
}

// x[item][18][18][16] (bf16): channel 0 = (log K - its mean over the leaf)
// / 2 on the leaf and its one-cell halo (0 outside the domain), channel 1 =
// log10(alpha) / 3, the others 0.  The basis fields do not change when K is
// scaled (A and B scale with it), hence the shift by the mean.
__global__ void __launch_bounds__(kIn * kIn) leaf_patches_kernel(DevView v, const int* __restrict__ ids,
                                                                 bf16* __restrict__ x) {
    __shared__ float red[kIn * kIn];
    const int item = blockIdx.x;
    const int id = ids[item];
    if ((unsigned)id >= (unsigned)v.nleaf) {              // uniform per CTA
        if (threadIdx.x == 0) atomicOr(v.status, kStatusBadIndex);
        return;
    }
    const LeafDesc L = v.leaves[id];
    const GridDesc& G = v.grids[L.grid];
    const int p = threadIdx.x, iy = p / kIn, ix = p % kIn;
    const int gi = L.i0 + ix - 1, gj = L.j0 + iy - 1;
    const bool in = gi >= 0 && gi < G.nx && gj >= 0 && gj < G.ny;
    const float lk = in ? (float)log(v.K[G.c0 + (long long)gj * G.nx + gi]) : 0.f;
    const bool inleaf = ix >= 1 && ix <= L.w && iy >= 1 && iy <= L.h;
    red[p] = inleaf ? lk : 0.f;
    __syncthreads();
    for (int s = 256; s > 0; s >>= 1) {
        if (p < s && p + s < kIn * kIn) red[p] += red[p + s];
        __syncthreads();
    }
    const float mean = red[0] / (float)(L.w * L.h);
    bf16* o = x + ((long long)item * kIn * kIn + p) * 16;
    o[0] = __float2bfloat16(in ? 0.5f * (lk - mean) : 0.f);
    o[1] = __float2bfloat16((float)log10(v.alpha) / 3.f);
    for (int c = 2; c < 16; ++c) o[c] = __float2bfloat16(0.f);
}

// ---------------------------------------------------------------------------
// 3 x 3 convolution, forward, as an implicit GEMM on the tensor cores: one
// CTA per item (256 output pixels x COUT channels), 8 warps of 2 output rows
// each; k = (ky 3 + kx) CIN + ci in chunks of 16 (one tap, 16 channels).
// PAD = 1: 16 x 16 input, zero border ('same'); PAD = 0: 18 x 18 input.
// y = act(conv(x, w) + b), written as bf16 (ybf) and / or float (yf).
__device__ __forceinline__ unsigned ld_u32(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }
__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int CIN, int COUT, int PAD, bool RELU>
__global__ void __launch_bounds__(256) conv_fwd_kernel(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                       const float* __restrict__ bias, bf16* __restrict__ ybf,
                                                       float* __restrict__ yf) {
    constexpr int CP = CIN + 8;                 // padded channel stride (bank spread)
    constexpr int K = 9 * CIN, KP = K + 8;
    constexpr int NT = COUT / 8;
    constexpr int HIN = PAD ? kS : kIn;
    __shared__ __align__(16) bf16 sx[kIn][kIn][CP];
    __shared__ __align__(16) bf16 sw[COUT][KP];
    const int item = blockIdx.x, tid = threadIdx.x;
    const bf16* xi = x + (long long)item * HIN * HIN * CIN;
    for (int idx = tid; idx < kIn * kIn * CIN; idx += 256) {
        const int c = idx % CIN, pix = idx / CIN, iy = pix / kIn, ix = pix % kIn;
        const int sy = iy - PAD, sxx = ix - PAD;
        sx[iy][ix][c] = (sy >= 0 && sy < HIN && sxx >= 0 && sxx < HIN) ? xi[(sy * HIN + sxx) * CIN + c]
                                                                      : __float2bfloat16(0.f);
    }
    for (int idx = tid; idx < COUT * K; idx += 256) sw[idx / K][idx % K] = w[idx];
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0.f;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
#pragma unroll
        for (int c0 = 0; c0 < CIN; c0 += 16) {
            const int kb = tap * CIN + c0;
            unsigned b[NT][2];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                b[nt][0] = ld_u32(&sw[nt * 8 + g][kb + 2 * t4]);
                b[nt][1] = ld_u32(&sw[nt * 8 + g][kb + 2 * t4 + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int oy = 2 * warp + mt;          // the m16 tile is output row oy
                const bf16* r0 = &sx[oy + ky][g + kx][c0 + 2 * t4];
                const bf16* r1 = &sx[oy + ky][g + 8 + kx][c0 + 2 * t4];
                const unsigned a0 = ld_u32(r0), a1 = ld_u32(r1), a2 = ld_u32(r0 + 8), a3 = ld_u32(r1 + 8);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], a0, a1, a2, a3, b[nt][0], b[nt][1]);
            }
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int oy = 2 * warp + mt;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int ox = g + (r >= 2 ? 8 : 0), co = nt * 8 + 2 * t4 + (r & 1);
                float val = acc[mt][nt][r] + (bias ? bias[co] : 0.f);
                if (RELU) val = fmaxf(val, 0.f);
                const long long o = (((long long)item * kS + oy) * kS + ox) * COUT + co;
                if (ybf) ybf[o] = __float2bfloat16(val);
                if (yf) yf[o] = val;
            }
    }
}

// Weight gradient of one 3 x 3 convolution: dw[co][k] += sum over the item's
// 256 output pixels of dy[pix][co] xcol[pix][k] (an M = COUT, N = 9 CIN,
// K = 256 GEMM per item on the tensor cores, added into FP32 dw with
// atomics), and db[co] += sum dy[pix][co].
template <int CIN, int COUT, int PAD>
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const bf16* __restrict__ x, const bf16* __restrict__ dy,
                                                         float* __restrict__ dw, float* __restrict__ db) {
    constexpr int HIN = PAD ? kS : kIn;
    constexpr int XP = kIn + 2;                  // padded row of the transposed input
    constexpr int NTILE = 9 * CIN / 8;           // n8 tiles of k
    constexpr int MTILE = COUT / 16;
    __shared__ __align__(16) bf16 sxt[CIN][kIn][XP];      // input, channel-major (pixels of a row contiguous)
    __shared__ __align__(16) bf16 sdy[COUT][kS * kS + 8]; // dy, channel-major
    const int item = blockIdx.x, tid = threadIdx.x;
    const bf16* xi = x + (long long)item * HIN * HIN * CIN;
    for (int idx = tid; idx < kIn * kIn * CIN; idx += 256) {
        const int c = idx % CIN, pix = idx / CIN, iy = pix / kIn, ix = pix % kIn;
        const int sy = iy - PAD, sxx = ix - PAD;
        sxt[c][iy][ix] = (sy >= 0 && sy < HIN && sxx >= 0 && sxx < HIN) ? xi[(sy * HIN + sxx) * CIN + c]
                                                                       : __float2bfloat16(0.f);
    }
    const bf16* dyi = dy + (long long)item * kS * kS * COUT;
    for (int idx = tid; idx < kS * kS * COUT; idx += 256) sdy[idx % COUT][idx / COUT] = dyi[idx];
    __syncthreads();
    if (db && tid < COUT) {
        float s = 0.f;
        for (int pix = 0; pix < kS * kS; ++pix) s += __bfloat162float(sdy[tid][pix]);
        atomicAdd(db + tid, s);
    }
    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
    // (m tile, n tile) pairs spread over the 8 warps
    for (int pair = warp; pair < MTILE * NTILE; pair += 8) {
        const int mt = pair / NTILE, nt = pair % NTILE;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        // this n tile's 8 values of k = (tap, ci): lane column g
        const int kcol = nt * 8 + g, tap = kcol / CIN, ci = kcol % CIN, ky = tap / 3, kx = tap % 3;
#pragma unroll 4
        for (int p0 = 0; p0 < kS * kS; p0 += 16) {
            // A: dy^T (co x pix), rows co = mt 16 + g (+8), cols pix = p0 + 2 t4 (+8)
            const bf16* d0 = &sdy[mt * 16 + g][p0 + 2 * t4];
            const bf16* d1 = &sdy[mt * 16 + g + 8][p0 + 2 * t4];
            const unsigned a0 = ld_u32(d0), a1 = ld_u32(d1), a2 = ld_u32(d0 + 8), a3 = ld_u32(d1 + 8);
            // B: xcol (pix x k), column k = kcol, rows pix = p0 + 2 t4 (+1) and + 8; the 16 pixels of a
            // chunk are one output row (oy = p0 / 16), so consecutive pixels are consecutive input columns
            const int oy = p0 / kS, ox = 2 * t4;
            const bf16* xr = &sxt[ci][oy + ky][ox + kx];
            const unsigned b0 = (unsigned)__bfloat16_as_ushort(xr[0]) | ((unsigned)__bfloat16_as_ushort(xr[1]) << 16);
            const unsigned b1 = (unsigned)__bfloat16_as_ushort(xr[8]) | ((unsigned)__bfloat16_as_ushort(xr[9]) << 16);
            mma_bf16(acc, a0, a1, a2, a3, b0, b1);
        }
        // C: rows co = mt 16 + g (+8), cols k = nt 8 + 2 t4 (+1)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int co = mt * 16 + g + (r >= 2 ? 8 : 0), k = nt * 8 + 2 * t4 + (r & 1);
            atomicAdd(dw + (long long)co * 9 * CIN + k, acc[r]);
        }
    }
}

// w2[ci][ky][kx][co] = w[co][2 - ky][2 - kx][ci]: the forward kernel on w2
// computes the input gradient of a 'same' convolution.
__global__ void flip_weights_kernel(const bf16* __restrict__ w, int cout, int cin, bf16* __restrict__ w2) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= cout * 9 * cin) return;
    const int ci = idx % cin, tap = (idx / cin) % 9, co = idx / (9 * cin);
    const int ky = tap / 3, kx = tap % 3;
    w2[((long long)ci * 9 + (2 - ky) * 3 + (2 - kx)) * cout + co] = w[idx];
}

// dpre = dpost * (y > 0) in bf16 (the ReLU's backward; y the layer's
// post-activation output); mask = 0: no activation.
__global__ void relu_grad_kernel(const float* __restrict__ dpost, const bf16* __restrict__ y, long long n, int mask,
                                 bf16* __restrict__ dpre) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d = dpost[i];
    if (mask && !(__bfloat162float(y[i]) > 0.f)) d = 0.f;
    dpre[i] = __float2bfloat16(d);
}

// Loss 0.5 sum (pred - target)^2 / count (both [item][16 x 16][16]);
// writes dpred = (pred - target) / count and adds the loss into *loss.
__global__ void mse_grad_kernel(const float* __restrict__ pred, const float* __restrict__ target, int count,
                                float* __restrict__ dpred, float* __restrict__ loss) {
    __shared__ float red[256];
    const long long n = (long long)count * kS * kS * 16;
    float acc = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        dpred[i] = d / (float)count;
        acc += 0.5f * d * d / (float)count;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// Adam on FP32 master weights, the BF16 copy refreshed: step t (from 1).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, bf16* __restrict__ pbf, long long n, float lr, float b1,
                            float b2, float eps, int t) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi, b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float ah = a / (1.f - powf(b1, (float)t)), bh = b / (1.f - powf(b2, (float)t));
    const float v = p[i] - lr * ah / (sqrtf(bh) + eps);
    p[i] = v;
    if (pbf) pbf[i] = __float2bfloat16(v);
}

// ---------------------------------------------------------------------------
// The residual gate and the maps of accepted leaves.
//
// res[item] = max over the segments s of ||A psi_s - B e_s|| / ||B e_s||
// (FP64, psi given as float [item][k][s]); one CTA of 256 threads per leaf,
// a thread per cell.
__device__ __forceinline__ void leaf_cell_coefs(const DevView& v, const LeafDesc& L, int i, int j, double c[6]) {
    const GridDesc& G = v.grids[L.grid];
    const int gi = L.i0 + i, gj = L.j0 + j;
    const long long fx = G.fx0 + gi + (long long)(G.nx + 1) * gj;
    const long long fy = G.fy0 + gi + (long long)G.nx * gj;
    c[0] = v.cxU[fx];            // west face, seen from the cell
    c[1] = v.cxL[fx + 1];        // east
    c[2] = v.cyU[fy];            // south
    c[3] = v.cyL[fy + G.nx];     // north
}
__device__ __forceinline__ int robin_segment(const DevView& v, const LeafDesc& L, int side, int i, int j) {
    if (L.side_off[side] < 0) return -1;
    if (side == 0 && i != 0) return -1;
    if (side == 1 && i != L.w - 1) return -1;
    if (side == 2 && j != 0) return -1;
    if (side == 3 && j != L.h - 1) return -1;
    return L.side_off[side] + (side < 2 ? j / v.gy : i / v.gx);
}

__global__ void __launch_bounds__(kS * kS) leaf_gate_kernel(DevView v, const int* __restrict__ ids,
                                                            const float* __restrict__ psi, double* __restrict__ res) {
    __shared__ double sp[kS * kS];
    __shared__ double red[2][kS * kS / 32];
    const int item = blockIdx.x, tid = threadIdx.x;
    const int id = ids[item];
    if ((unsigned)id >= (unsigned)v.nleaf || v.leaves[id].m > 16) {   // uniform per CTA
        if (tid == 0) {
            atomicOr(v.status, kStatusBadIndex);
            res[item] = 1e300;
        }
        return;
    }
    const LeafDesc L = v.leaves[id];
    const int w = L.w, h = L.h, n = w * h;
    const int i = tid % w, j = tid / w;
    double cf[4] = {0, 0, 0, 0};
    int seg[4] = {-1, -1, -1, -1};
    if (tid < n) {
        double c[6];
        leaf_cell_coefs(v, L, i, j, c);
        for (int d = 0; d < 4; ++d) {
            cf[d] = c[d];
            seg[d] = robin_segment(v, L, d, i, j);
        }
    }
    double worst = 0.0;
    for (int s = 0; s < L.m; ++s) {
        __syncthreads();
        if (tid < n) sp[tid] = (double)psi[((long long)item * (kS * kS) + tid) * 16 + s];
        __syncthreads();
        double r = 0.0, b = 0.0;
        if (tid < n) {
            // (A psi)_c = (sum of the cell's face coefficients) psi_c - sum over
            // its neighbours inside the leaf of T psi_neighbour
            const double pc = sp[tid];
            double ap = (cf[0] + cf[1] + cf[2] + cf[3]) * pc;
            if (i > 0) ap -= cf[0] * sp[tid - 1];
            if (i < w - 1) ap -= cf[1] * sp[tid + 1];
            if (j > 0) ap -= cf[2] * sp[tid - w];
            if (j < h - 1) ap -= cf[3] * sp[tid + w];
            for (int d = 0; d < 4; ++d)
                if (seg[d] == s) b += cf[d];
            r = ap - b;
        }
        double rr = r * r, bb = b * b;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rr += __shfl_xor_sync(0xffffffffu, rr, o);
            bb += __shfl_xor_sync(0xffffffffu, bb, o);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = rr;
            red[1][tid >> 5] = bb;
        }
        __syncthreads();
        if (tid == 0) {
            double R = 0.0, Bn = 0.0;
            for (int k = 0; k < kS * kS / 32; ++k) {
                R += red[0][k];
                Bn += red[1][k];
            }
            worst = fmax(worst, sqrt(R / Bn));
        }
    }
    if (tid == 0) res[item] = worst;
}

// For the leaves with res[item] <= tau: R = B^T psi - W from the predicted
// fields, symmetrised, written over the leaf's map (then the merges are
// rebuilt); accepted[item] = 1 for them.
__global__ void __launch_bounds__(kS * kS) leaf_apply_kernel(DevView v, const int* __restrict__ ids,
                                                             const float* __restrict__ psi,
                                                             const double* __restrict__ res, double tau,
                                                             int* __restrict__ accepted) {
    __shared__ double F[16][16];
    const int item = blockIdx.x, tid = threadIdx.x;
    const int id = ids[item];
    if (!(res[item] <= tau) || (unsigned)id >= (unsigned)v.nleaf || v.leaves[id].m > 16) {   // uniform per CTA
        if (tid == 0) accepted[item] = 0;
        return;
    }
    const LeafDesc L = v.leaves[id];
    const int w = L.w, n = w * L.h, m = L.m;
    if (tid < m * m) F[tid / m][tid % m] = 0.0;
    __syncthreads();
    if (tid < n) {
        const int i = tid % w, j = tid / w;
        double c[6];
        leaf_cell_coefs(v, L, i, j, c);
        for (int d = 0; d < 4; ++d) {
            const int s = robin_segment(v, L, d, i, j);
            if (s < 0) continue;
            // flux out through face d of segment s for a unit datum on t:
            // rho (psi_t(c) - delta_st)
            for (int t = 0; t < m; ++t) {
                const double pt = (double)psi[((long long)item * (kS * kS) + tid) * 16 + t];
                atomicAdd(&F[s][t], c[d] * (pt - (s == t ? 1.0 : 0.0)));
            }
        }
    }
    __syncthreads();
    double* Rg = v.R + L.R_off;
    if (tid < m * m) {
        const int s = tid / m, t = tid % m;
        Rg[tid] = 0.5 * (F[s][t] + F[t][s]);
    }
    if (tid == 0) accepted[item] = 1;
}

}  // namespace

cudaError_t launch_leaf_fields(const DevView& v, const int* ids, int count, float* psi, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (v.leaf32)
        leaf_fields_kernel<float><<<(count + 7) / 8, 128, 0, s>>>(v, ids, count, psi);
    else
        leaf_fields_kernel<double><<<(count + 7) / 8, 128, 0, s>>>(v, ids, count, psi);
    return cudaGetLastError();
}
cudaError_t launch_leaf_patches(const DevView& v, const int* ids, int count, void* x, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    leaf_patches_kernel<<<count, kIn * kIn, 0, s>>>(v, ids, static_cast<bf16*>(x));
    return cudaGetLastError();
}
cudaError_t launch_leaf_gate(const DevView& v, const int* ids, int count, const float* psi, double* res,
                             cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    leaf_gate_kernel<<<count, kS * kS, 0, s>>>(v, ids, psi, res);
    return cudaGetLastError();
}
cudaError_t launch_leaf_apply(const DevView& v, const int* ids, int count, const float* psi, const double* res,
                              double tau, int* accepted, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    leaf_apply_kernel<<<count, kS * kS, 0, s>>>(v, ids, psi, res, tau, accepted);
    return cudaGetLastError();
}

// Network kernels (no context): shapes as in include/mrcm.h.
cudaError_t launch_conv_fwd(const void* x, int count, int cin, int cout, int pad, int relu, const void* w,
                            const float* b, void* ybf, float* yf, cudaStream_t s) {
    const bf16* X = static_cast<const bf16*>(x);
    const bf16* Wt = static_cast<const bf16*>(w);
    bf16* Y = static_cast<bf16*>(ybf);
#define MRCM_CONV(CI, CO, PD, RL)                                                                   \
    if (cin == CI && cout == CO && pad == PD && (relu != 0) == RL) {                                \
        conv_fwd_kernel<CI, CO, PD, RL><<<count, 256, 0, s>>>(X, Wt, b, Y, yf);                     \
        return cudaGetLastError();                                                                  \
    }
    MRCM_CONV(16, 32, 0, true)
    MRCM_CONV(16, 32, 0, false)
    MRCM_CONV(32, 32, 1, true)
    MRCM_CONV(32, 32, 1, false)
    MRCM_CONV(32, 16, 1, false)
    MRCM_CONV(32, 16, 1, true)
    MRCM_CONV(16, 32, 1, false)
    MRCM_CONV(16, 32, 1, true)
#undef MRCM_CONV
    return cudaErrorInvalidValue;
}
cudaError_t launch_conv_wgrad(const void* x, const void* dy, int count, int cin, int cout, int pad, float* dw,
                              float* db, cudaStream_t s) {
    const bf16* X = static_cast<const bf16*>(x);
    const bf16* D = static_cast<const bf16*>(dy);
#define MRCM_WG(CI, CO, PD)                                                                         \
    if (cin == CI && cout == CO && pad == PD) {                                                     \
        conv_wgrad_kernel<CI, CO, PD><<<count, 256, 0, s>>>(X, D, dw, db);                          \
        return cudaGetLastError();                                                                  \
    }
    MRCM_WG(16, 32, 0)
    MRCM_WG(32, 32, 1)
    MRCM_WG(32, 16, 1)
#undef MRCM_WG
    return cudaErrorInvalidValue;
}
cudaError_t launch_flip_weights(const void* w, int cout, int cin, void* w2, cudaStream_t s) {
    const int n = cout * 9 * cin;
    flip_weights_kernel<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const bf16*>(w), cout, cin,
                                                         static_cast<bf16*>(w2));
    return cudaGetLastError();
}
cudaError_t launch_relu_grad(const float* dpost, const void* y, long long n, int mask, void* dpre, cudaStream_t s) {
    relu_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dpost, static_cast<const bf16*>(y), n, mask,
                                                                  static_cast<bf16*>(dpre));
    return cudaGetLastError();
}
cudaError_t launch_mse_grad(const float* pred, const float* target, int count, float* dpred, float* loss,
                            cudaStream_t s) {
    mse_grad_kernel<<<304, 256, 0, s>>>(pred, target, count, dpred, loss);
    return cudaGetLastError();
}
cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, void* pbf, long long n, float lr, float b1,
                        float b2, float eps, int t, cudaStream_t s) {
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, g, m1, m2, static_cast<bf16*>(pbf), n, lr, b1, b2,
                                                            eps, t);
    return cudaGetLastError();
}

}  // namespace mrcm
