// ali.cu -- operator splitting with the diagonal Lambda* (Hauschildt & Baron
// IV, Sect. 3.2.1; the OS step of Papers I-II read as R10), Ng acceleration
// (R11) and the FP64 residual / FP32 correction pieces of the mixed-precision
// iterative refinement.  All in FP64.  Reductions (max, Ng dot products) use
// a fixed grid and a fixed tree order, so they are deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.h"

namespace rtk {
namespace {

constexpr int NG_BLOCKS = 304;  // 2 x 152 SMs
constexpr int NG_THREADS = 256;

__device__ __forceinline__ void block_max_to(double v, unsigned long long *dst)
{
    __shared__ double red[32];
    const unsigned FULL = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(FULL, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(FULL, v, o));
        // non-negative doubles order like their bit patterns (NaN sorts above +inf)
        if (threadIdx.x == 0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
    }
}

__global__ void k_pack64(int n, const double *chi, const double *S, double2 *cs)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) cs[v] = make_double2(chi[v], S[v]);
}

__global__ void k_pack32(int n, const double *chi, const double *S, const double *B, float2 *cs, float *B32,
                         float *S32)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        const float s = (float)S[v];
        cs[v] = make_float2((float)chi[v], s);
        B32[v] = (float)B[v];
        if (S32) S32[v] = s;
    }
}

__global__ void k_ali(int n, double *S, const double *J, const double *L, const double *eps, const double *B,
                      int use_lstar, double *slot, unsigned long long *maxrel)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double rel = 0.0;
    if (v < n) {
        double e = eps[v];
        double lst = use_lstar ? L[v] : 0.0;
        double s = S[v];
        double sn = s + ((1.0 - e) * J[v] + e * B[v] - s) / (1.0 - (1.0 - e) * lst);
        rel = fabs(sn - s) / fabs(sn);
        S[v] = sn;
        if (slot) slot[v] = sn;
    }
    block_max_to(rel, maxrel);
}

__global__ void k_residual(int n, const double *S, const double *J, const double *L, const double *eps,
                           const double *B, int use_lstar, double *r, unsigned long long *maxrel)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double rel = 0.0;
    if (v < n) {
        double e = eps[v];
        double lst = use_lstar ? L[v] : 0.0;
        double rv = (1.0 - e) * J[v] + e * B[v] - S[v];
        double step = rv / (1.0 - (1.0 - e) * lst);
        rel = fabs(step) / fabs(S[v] + step);
        r[v] = rv;
    }
    block_max_to(rel, maxrel);
}

// One ALI sweep on the correction equation delta = (1-eps) Lambda delta + r.
__global__ void k_ali_corr(int n, double *delta, const double *Jd, const double *r, const double *L,
                           const double *eps, const double *S, int use_lstar, double *slot,
                           unsigned long long *maxrel)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double rel = 0.0;
    if (v < n) {
        double e = eps[v];
        double lst = use_lstar ? L[v] : 0.0;
        double d = delta[v];
        double dn = d + ((1.0 - e) * Jd[v] + r[v] - d) / (1.0 - (1.0 - e) * lst);
        rel = fabs(dn - d) / fabs(S[v] + dn);
        delta[v] = dn;
        if (slot) slot[v] = dn;
    }
    block_max_to(rel, maxrel);
}

__global__ void k_add(int n, double *S, const double *d)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) S[v] += d[v];
}

__global__ void k_fill(int n, double *x, double val)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) x[v] = val;
}

// Ng normal-equation sums over voxels with weights 1/wref^2 (wref = y0 if null).
__global__ void __launch_bounds__(NG_THREADS) k_ng_dots(int n, const double *y0, const double *y1, const double *y2,
                                                        const double *y3, const double *wref, double *partial)
{
    __shared__ double sh[5][NG_THREADS];
    double a11 = 0, a12 = 0, a22 = 0, b1 = 0, b2 = 0;
    for (int v = blockIdx.x * NG_THREADS + threadIdx.x; v < n; v += NG_BLOCKS * NG_THREADS) {
        double ref = wref ? wref[v] : y0[v];
        double W = 1.0 / (ref * ref);
        double r1 = y0[v] - y1[v], r2 = y1[v] - y2[v], r3 = y2[v] - y3[v];
        double d1 = r1 - r2, d2 = r1 - r3;
        a11 += W * d1 * d1;
        a12 += W * d1 * d2;
        a22 += W * d2 * d2;
        b1 += W * d1 * r1;
        b2 += W * d2 * r1;
    }
    sh[0][threadIdx.x] = a11; sh[1][threadIdx.x] = a12; sh[2][threadIdx.x] = a22;
    sh[3][threadIdx.x] = b1; sh[4][threadIdx.x] = b2;
    __syncthreads();
    for (int s = NG_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(NG_THREADS) k_ng_solve(const double *partial, double *coef)
{
    __shared__ double sh[5][NG_THREADS];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < NG_BLOCKS; b += NG_THREADS)
        for (int c = 0; c < 5; ++c) acc[c] += partial[b * 5 + c];
    for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = NG_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double A11 = sh[0][0], A12 = sh[1][0], A22 = sh[2][0], b1 = sh[3][0], b2 = sh[4][0];
        double det = A11 * A22 - A12 * A12;
        bool ok = (fabs(det) > 1e-14 * (A11 * A22)) && (det == det);
        coef[0] = ok ? (b1 * A22 - b2 * A12) / det : 0.0;
        coef[1] = ok ? (A11 * b2 - A12 * b1) / det : 0.0;
        coef[2] = ok ? 1.0 : 0.0;
    }
}

__global__ void k_ng_apply(int n, const double *y0, const double *y1, const double *y2, const double *coef, double *out)
{
    if (coef[2] == 0.0) return;
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        double a = coef[0], b = coef[1];
        out[v] = (1.0 - a - b) * y0[v] + a * y1[v] + b * y2[v];
    }
}

inline unsigned nb(int n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int ng_partial_elems(int) { return NG_BLOCKS * 5; }

cudaError_t pack_chiS64(int nvox, const double *chi, const double *S, double2 *cs, cudaStream_t st)
{
    k_pack64<<<nb(nvox), 256, 0, st>>>(nvox, chi, S, cs);
    return cudaGetLastError();
}

cudaError_t pack_chiS32(int nvox, const double *chi, const double *S, const double *B, float2 *cs, float *B32, float *S32,
                        cudaStream_t st)
{
    k_pack32<<<nb(nvox), 256, 0, st>>>(nvox, chi, S, B, cs, B32, S32);
    return cudaGetLastError();
}

// Input check of rt_set_opacity for device arrays: the smallest 4 v + c over
// voxels v whose chi (c = 0), eps (c = 1) or B (c = 2) is out of range.
__global__ void k_check_opacity(int n, const double *chi, const double *eps, const double *B,
                                unsigned long long *first_bad)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double c = chi[v], e = eps[v], b = B[v];
        int code = -1;
        if (!(c > 0.0) || !isfinite(c)) code = 0;
        else if (!(e > 0.0 && e <= 1.0)) code = 1;
        else if (!(b >= 0.0) || !isfinite(b)) code = 2;
        if (code >= 0) atomicMin(first_bad, 4ull * (unsigned long long)v + (unsigned long long)code);
    }
}

cudaError_t check_opacity(int nvox, const double *chi, const double *eps, const double *B,
                          unsigned long long *first_bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(first_bad, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int blocks = nb(nvox);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_check_opacity<<<blocks, 256, 0, st>>>(nvox, chi, eps, B, first_bad);
    return cudaGetLastError();
}

cudaError_t pack_preload()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_pack64);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_pack32);
    return e;
}

cudaError_t ali_update(int nvox, double *S, const double *J, const double *Lst, const double *eps, const double *B,
                       int use_lstar, double *hist_slot, unsigned long long *maxrel, cudaStream_t st)
{
    k_ali<<<nb(nvox), 256, 0, st>>>(nvox, S, J, Lst, eps, B, use_lstar, hist_slot, maxrel);
    return cudaGetLastError();
}

cudaError_t ng_extrapolate(int nvox, const double *y0, const double *y1, const double *y2, const double *y3,
                           const double *wref, double *partial, double *coef, double *out, cudaStream_t st)
{
    k_ng_dots<<<NG_BLOCKS, NG_THREADS, 0, st>>>(nvox, y0, y1, y2, y3, wref, partial);
    k_ng_solve<<<1, NG_THREADS, 0, st>>>(partial, coef);
    k_ng_apply<<<nb(nvox), 256, 0, st>>>(nvox, y0, y1, y2, coef, out);
    return cudaGetLastError();
}

cudaError_t residual(int nvox, const double *S, const double *J, const double *Lst, const double *eps,
                     const double *B, int use_lstar, double *r, unsigned long long *maxrel, cudaStream_t st)
{
    k_residual<<<nb(nvox), 256, 0, st>>>(nvox, S, J, Lst, eps, B, use_lstar, r, maxrel);
    return cudaGetLastError();
}

cudaError_t ali_correction(int nvox, double *delta, const double *Jd, const double *r, const double *Lst,
                           const double *eps, const double *S, int use_lstar, double *hist_slot,
                           unsigned long long *maxrel, cudaStream_t st)
{
    k_ali_corr<<<nb(nvox), 256, 0, st>>>(nvox, delta, Jd, r, Lst, eps, S, use_lstar, hist_slot, maxrel);
    return cudaGetLastError();
}

cudaError_t add_inplace(int nvox, double *S, const double *delta, cudaStream_t st)
{
    k_add<<<nb(nvox), 256, 0, st>>>(nvox, S, delta);
    return cudaGetLastError();
}

cudaError_t fill_const(int n, double *x, double v, cudaStream_t st)
{
    k_fill<<<nb(n), 256, 0, st>>>(n, x, v);
    return cudaGetLastError();
}

}  // namespace rtk
