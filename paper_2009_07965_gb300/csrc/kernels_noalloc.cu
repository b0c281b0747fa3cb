// Allocation-free merge of two Robin-to-flux maps (mrcm_merge_pair_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// merge: code that runs inside another framework's execution step (an
// inference-engine plugin's enqueue, a solver callback) where that framework
// owns all device memory, or latency-bound loops that cannot afford the
// implicit device synchronisation of cudaMalloc.  This entry point takes
// every input and output from the caller and keeps its only workspace -- the
// LU factors and pivots of the interface matrix and a status word -- in a
// file-scope device array of fixed size, which each GPU that loads the
// library holds until the process exits.
//
// It gives the merged map of one merge step of the build, but by its own
// route: one CTA factors the interface matrix by LU with partial pivoting
// (the build inverts the quasi-definite form instead), then
//     M = [[R1_gg + D, -D], [-D, R2_gg + D]],  X = -M^-1 C,
//     R = blockdiag(R1_oo, R2_oo) + blockdiag(R1_og, R2_og) X.
// Its singularity test looks at pivot magnitudes only (|pivot| <= 1e-14
// max |M|); the build's pivot-sign test of the quasi-definite form has no
// counterpart in a partial-pivot LU.
#include "mrcm_internal.h"
#include "../../include/mrcm.h"

namespace mrcm {
namespace {

constexpr int kNoAllocMaxG2 = MRCM_NOALLOC_MAX_G2;
constexpr int kNoAllocThreads = 256;

// LU factors (row-major), pivot rows and one status word.
struct NoAllocScratch {
    double lu[kNoAllocMaxG2 * kNoAllocMaxG2];
    int piv[kNoAllocMaxG2];
    int status;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__global__ void __launch_bounds__(kNoAllocThreads)
merge_pair_noalloc_kernel(NoAllocScratch* S, const double* __restrict__ R1, int m1,
                          const double* __restrict__ R2, int m2, const int* __restrict__ map, int g,
                          const double* __restrict__ D, double* __restrict__ Rp,
                          double* __restrict__ X) {
    constexpr int NT = kNoAllocThreads;
    __shared__ double red_v[NT / 32];
    __shared__ int red_i[NT / 32];
    __shared__ double s_thresh;
    const int tid = threadIdx.x;
    const int g2 = 2 * g, m = m1 + m2 - 2 * g, o1 = m1 - g;
    const int *gpos1 = map, *gpos2 = map + g, *opos1 = map + 2 * g, *opos2 = map + 2 * g + o1;
    double* M = S->lu;
    __shared__ int s_bad;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // the index map comes from the caller: check it before any indexed access
    for (int k = tid; k < g2 + m; k += NT) {
        const int lim = (k < g || (k >= g2 && k < g2 + o1)) ? m1 : m2;
        if (map[k] < 0 || map[k] >= lim) s_bad = 1;
    }
    if (tid == 0) S->status = 0;   // the array keeps the previous call's contents
    __syncthreads();
    if (s_bad) {
        if (tid == 0) S->status = kStatusBadIndex;
        return;
    }
    double amax = 0.0;
    for (int idx = tid; idx < g2 * g2; idx += NT) {
        const int r = idx / g2, c = idx % g2;
        double val = 0.0;
        if (r < g && c < g) val = R1[gpos1[r] * m1 + gpos1[c]] + (r == c ? D[r] : 0.0);
        else if (r >= g && c >= g) val = R2[gpos2[r - g] * m2 + gpos2[c - g]] + (r == c ? D[r - g] : 0.0);
        else if (r < g && c - g == r) val = -D[r];
        else if (r >= g && r - g == c) val = -D[c];
        M[idx] = val;
        amax = fmax(amax, fabs(val));
    }
    for (int idx = tid; idx < g2 * m; idx += NT) {
        const int r = idx / m, c = idx % m;
        double val = 0.0;
        if (r < g && c < o1) val = R1[gpos1[r] * m1 + opos1[c]];
        else if (r >= g && c >= o1) val = R2[gpos2[r - g] * m2 + opos2[c - o1]];
        X[idx] = val;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_down_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) red_v[tid >> 5] = amax;
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int w = 0; w < NT / 32; ++w) mx = fmax(mx, red_v[w]);
        s_thresh = 1e-14 * mx;
    }
    __syncthreads();
    const double thresh = s_thresh;
    bool singular = false;
    for (int k = 0; k < g2; ++k) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < g2; i += NT) {
            const double a = fabs(M[i * g2 + k]);
            if (a > best) { best = a; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            double bv = red_v[0];
            int b = red_i[0];
            for (int w = 1; w < NT / 32; ++w)
                if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < b)) { bv = red_v[w]; b = red_i[w]; }
            S->piv[k] = b;
        }
        __syncthreads();
        const int p = S->piv[k];
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
    if (singular && tid == 0) S->status = kStatusSingular;
    for (int j = tid; j < m; j += NT) {
        for (int k = 0; k < g2; ++k) {
            const int p = S->piv[k];
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
    for (int idx = tid; idx < m * m; idx += NT) {
        const int i = idx / m, j = idx % m;
        double acc = 0.0;
        if (i < o1) {
            const double* row = R1 + opos1[i] * m1;
            if (j < o1) acc = row[opos1[j]];
            for (int k = 0; k < g; ++k) acc += row[gpos1[k]] * X[k * m + j];
        } else {
            const double* row = R2 + opos2[i - o1] * m2;
            if (j >= o1) acc = row[opos2[j - o1]];
            for (int k = 0; k < g; ++k) acc += row[gpos2[k]] * X[(g + k) * m + j];
        }
        Rp[idx] = acc;
    }
}

}  // namespace
}  // namespace mrcm

using namespace mrcm;

extern "C" int mrcm_merge_pair_noalloc(const double* R1_dev, int m1, const double* R2_dev, int m2,
                                       const int* map_dev, int g, const double* D_dev,
                                       double* R_dev, double* X_dev, void* cuda_stream) {
    if (!R1_dev || !R2_dev || !map_dev || !D_dev || !R_dev || !X_dev) return MRCM_ERR_INVALID_ARG;
    if (g < 1 || 2 * g > kNoAllocMaxG2) return MRCM_ERR_INVALID_ARG;
    if (m1 < g || m2 < g) return MRCM_ERR_INVALID_ARG;
    // The array's device address, looked up on every call with the
    // caller's device and context current (the host name of the array is
    // only a host-side stand-in).  The lookup is a host-side query: it
    // allocates nothing and does not synchronise, and a fresh lookup stays
    // right when the module is loaded again (after cudaDeviceReset, or in
    // another context of the same device).
    void* addr = nullptr;
    int rc = cuda_status(cudaGetSymbolAddress(&addr, g_noalloc_scratch));
    if (rc != MRCM_OK) return rc;
    NoAllocScratch* scratch = static_cast<NoAllocScratch*>(addr);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // an error left pending by earlier work is not this call's failure
    cudaGetLastError();
    merge_pair_noalloc_kernel<<<1, kNoAllocThreads, 0, s>>>(scratch, R1_dev, m1, R2_dev, m2, map_dev, g,
                                                            D_dev, R_dev, X_dev);
    if ((rc = cuda_status(cudaGetLastError())) != MRCM_OK) return rc;
    int status = 0;
    if ((rc = cuda_status(cudaMemcpyAsync(&status, &scratch->status, sizeof(int), cudaMemcpyDeviceToHost, s))) !=
        MRCM_OK)
        return rc;
    if ((rc = cuda_status(cudaStreamSynchronize(s))) != MRCM_OK) return rc;
    if (status & kStatusBadIndex) return MRCM_ERR_INVALID_ARG;
    return (status & kStatusSingular) ? MRCM_ERR_SINGULAR : MRCM_OK;
}
