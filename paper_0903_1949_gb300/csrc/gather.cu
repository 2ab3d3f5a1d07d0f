// gather.cu -- per-voxel ownership of the formal-solution results.
//
// For every solid-angle block the segments that cross voxel v are listed in
// a CSR structure (sorted by segment index, hence by angle and ray order).
// One thread owns one voxel and sums, in that fixed order, the path-length
// weighted intensities l*I and Lambda* terms l*lambda that the ray march
// wrote per segment; the per-angle path-length average (Ibar = sum l I /
// sum l, R8) is then folded into J, Lambda* and the flux vector with the
// quadrature weights (Sect. 3.2: J, flux vectors of voxels).  No float atomics
// are used, so every result is bit-reproducible from run to run.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.h"

namespace rtk {
namespace {

constexpr double FOUR_PI = 12.566370614359172953850573533118;
constexpr int MAX_BLOCK_ANGLES = 256;
constexpr int UNIT_LEN = 512;  // ownership-list entries per gather work unit

__global__ void k_count_vox(const uint32_t *vox, int64_t n, int32_t *counts)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + (vox[s] & RTK_VOXMASK), 1);
}

__global__ void k_off32(const int64_t *off64, int32_t *off32, int n1)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) off32[i] = (int32_t)off64[i];
}

__global__ void k_fill(const uint32_t *vox, int64_t n, int32_t *cursor, int32_t *perm)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        int v = vox[s] & RTK_VOXMASK;
        int pos = atomicAdd(cursor + v, 1);
        perm[pos] = (int32_t)s;
    }
}

// The fill order above is arbitrary: sort every voxel's list so the
// summation order is the segment order.
__global__ void k_sort_lists(int nvox, const int32_t *off, int32_t *perm)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    int lo = off[v], hi = off[v + 1];
    for (int a = lo + 1; a < hi; ++a) {
        int32_t x = perm[a];
        int b = a - 1;
        while (b >= lo && perm[b] > x) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = x;
    }
}

__global__ void k_invL(int nvox, const int32_t *off, const int32_t *perm, const double *len, const int64_t *ang_seg_off,
                       int w0, int nw, int64_t seg_lo, double *invL)
{
    __shared__ int64_t soff[MAX_BLOCK_ANGLES + 1];
    for (int q = threadIdx.x; q <= nw; q += blockDim.x) soff[q] = ang_seg_off[w0 + q] - seg_lo;
    __syncthreads();
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    int lo = off[v], hi = off[v + 1];
    int q = 0;
    int64_t next = soff[1];
    double acc = 0.0;
    for (int e = lo; e < hi; ++e) {
        int s = perm[e];
        while (s >= next && q < nw) {
            invL[(int64_t)(w0 + q) * nvox + v] = (acc > 0.0) ? 1.0 / acc : 0.0;
            acc = 0.0;
            ++q;
            next = (q < nw) ? soff[q + 1] : INT64_MAX;
        }
        acc += len[s];
    }
    while (q < nw) {
        invL[(int64_t)(w0 + q) * nvox + v] = (acc > 0.0) ? 1.0 / acc : 0.0;
        acc = 0.0;
        ++q;
    }
}

template <typename P>
__global__ void k_gather_angle(int nvox, const int32_t *off, const int32_t *perm, const P *buf, int64_t s_lo,
                               int64_t s_hi, const double *invL_w, double *Ibar, double *Lbar)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    double aI = 0.0, aL = 0.0;
    for (int e = off[v]; e < off[v + 1]; ++e) {
        int s = perm[e];
        if (s < s_lo || s >= s_hi) continue;
        P val = buf[s];
        aI += (double)val.x;
        aL += (double)val.y;
    }
    Ibar[v] = aI * invL_w[v];
    Lbar[v] = aL * invL_w[v];
}

__global__ void k_flux_local(GeomDev G, const double *Fc, double *F)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G.nvox) return;
    int k = v % G.n3, j = (v / G.n3) % G.n2;
    double x = FOUR_PI * Fc[3 * (int64_t)v], y = FOUR_PI * Fc[3 * (int64_t)v + 1], z = FOUR_PI * Fc[3 * (int64_t)v + 2];
    double e0x, e0y, e0z, e1x, e1y, e1z, e2x, e2y, e2z;
    if (G.coord == RT_SPHERICAL) {
        double st = G.stm[j], ct = G.ctm[j], c = G.cpm[k], s = G.spm[k];
        e0x = st * c; e0y = st * s; e0z = ct;
        e1x = ct * c; e1y = ct * s; e1z = -st;
        e2x = -s; e2y = c; e2z = 0.0;
    } else {
        double c = G.cpm[j], s = G.spm[j];
        e0x = c; e0y = s; e0z = 0.0;
        e1x = -s; e1y = c; e1z = 0.0;
        e2x = 0.0; e2y = 0.0; e2z = 1.0;
    }
    F[3 * (int64_t)v] = e0x * x + e0y * y + e0z * z;
    F[3 * (int64_t)v + 1] = e1x * x + e1y * y + e1z * z;
    F[3 * (int64_t)v + 2] = e2x * x + e2y * y + e2z * z;
}

// Work units: every ownership list is cut into pieces of at most UNIT_LEN
// entries so one warp never walks more than UNIT_LEN / 32 steps, whatever
// the visit count of the voxel (outer voxels on the line of sight through the
// core collect thousands of visits per solid angle).
__global__ void k_unit_count(int nvox, const int32_t *off, int32_t *nu)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    int len = off[v + 1] - off[v];
    nu[v] = len <= UNIT_LEN ? 1 : (len + UNIT_LEN - 1) / UNIT_LEN;
}

__global__ void k_unit_fill(int nvox, const int32_t *off, const int64_t *ufirst, int32_t *urow, int32_t *ubeg)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    int64_t u0 = ufirst[v], u1 = ufirst[v + 1];
    for (int64_t u = u0; u < u1; ++u) {
        urow[u] = v;
        ubeg[u] = off[v] + (int32_t)((u - u0) * UNIT_LEN);
    }
}

// One warp per work unit: weighted sums of the unit's entries,
//   J += wt_q / L_qv * (l I),  Lambda* += wt_q / L_qv * (l lambda),  F += n_q * (J term),
// reduced across the warp in a fixed shuffle order.
template <typename P>
__global__ void __launch_bounds__(256) k_gather_units(int nvox, int64_t nunits, const int32_t *__restrict__ urow,
                                                      const int32_t *__restrict__ ubeg, const int32_t *__restrict__ off,
                                                      const int32_t *__restrict__ perm, const P *__restrict__ buf,
                                                      const int64_t *__restrict__ ang_seg_off, int w0, int nw,
                                                      int64_t seg_lo, const double *__restrict__ invL,
                                                      const double *__restrict__ wt, const double *__restrict__ dirs,
                                                      double *__restrict__ part)
{
    __shared__ int32_t soff[MAX_BLOCK_ANGLES + 1];
    __shared__ double swt[MAX_BLOCK_ANGLES], sdir[3 * MAX_BLOCK_ANGLES];
    for (int q = threadIdx.x; q <= nw; q += blockDim.x) soff[q] = (int32_t)(ang_seg_off[w0 + q] - seg_lo);
    for (int q = threadIdx.x; q < nw; q += blockDim.x) {
        swt[q] = wt[w0 + q];
        sdir[3 * q] = dirs[3 * (w0 + q)];
        sdir[3 * q + 1] = dirs[3 * (w0 + q) + 1];
        sdir[3 * q + 2] = dirs[3 * (w0 + q) + 2];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (u >= nunits) return;
    const int v = urow[u];
    const int e0 = ubeg[u];
    const int e1 = (u + 1 < nunits && urow[u + 1] == v) ? ubeg[u + 1] : off[v + 1];
    double aj = 0.0, al = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    for (int e = e0 + lane; e < e1; e += 32) {
        int s = perm[e];
        int lo = 0, hi = nw;  // angle of segment s: soff[q] <= s < soff[q+1]
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (soff[mid] <= s) lo = mid;
            else hi = mid;
        }
        double f = swt[lo] * invL[(int64_t)(w0 + lo) * nvox + v];
        P val = buf[s];
        double cj = f * (double)val.x;
        aj += cj;
        al += f * (double)val.y;
        fx += sdir[3 * lo] * cj;
        fy += sdir[3 * lo + 1] * cj;
        fz += sdir[3 * lo + 2] * cj;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        aj += __shfl_xor_sync(0xffffffffu, aj, o);
        al += __shfl_xor_sync(0xffffffffu, al, o);
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (lane == 0) {
        double *o = part + 5 * u;
        o[0] = aj; o[1] = al; o[2] = fx; o[3] = fy; o[4] = fz;
    }
}

// Thread per voxel: add the voxel's unit sums in unit order to J, Lambda*, F.
__global__ void k_gather_rows(int nvox, const int64_t *__restrict__ ufirst, const double *__restrict__ part, double *J,
                              double *Lst, double *Fc, int first)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    double j = 0.0, l = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    for (int64_t u = ufirst[v]; u < ufirst[v + 1]; ++u) {
        const double *o = part + 5 * u;
        j += o[0]; l += o[1]; fx += o[2]; fy += o[3]; fz += o[4];
    }
    if (!first) {
        j += J[v];
        l += Lst[v];
        fx += Fc[3 * (int64_t)v];
        fy += Fc[3 * (int64_t)v + 1];
        fz += Fc[3 * (int64_t)v + 2];
    }
    J[v] = j;
    Lst[v] = l;
    Fc[3 * (int64_t)v] = fx;
    Fc[3 * (int64_t)v + 1] = fy;
    Fc[3 * (int64_t)v + 2] = fz;
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t csr_build(int nvox, const uint32_t *vox_blk, int64_t nseg_blk, int32_t *counts, int32_t *csr_off,
                      int32_t *cursor, int32_t *perm_blk, int64_t *tmp, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * nvox, st);
    if (e != cudaSuccess) return e;
    k_count_vox<<<grid_for(nseg_blk, 256), 256, 0, st>>>(vox_blk, nseg_blk, counts);
    // offsets in int64 scratch, then narrowed (a block holds < 2^31 segments)
    int64_t *off64 = tmp;
    int64_t *stmp = tmp + (nvox + 1);
    if ((e = scan_i32(counts, off64, nvox, stmp, st)) != cudaSuccess) return e;
    k_off32<<<(nvox + 256) / 256, 256, 0, st>>>(off64, csr_off, nvox + 1);
    if ((e = cudaMemcpyAsync(cursor, csr_off, sizeof(int32_t) * nvox, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    k_fill<<<grid_for(nseg_blk, 256), 256, 0, st>>>(vox_blk, nseg_blk, cursor, perm_blk);
    k_sort_lists<<<(nvox + 127) / 128, 128, 0, st>>>(nvox, csr_off, perm_blk);
    return cudaGetLastError();
}

cudaError_t csr_invL(int nvox, const int32_t *csr_off, const int32_t *perm_blk, const double *len64_blk,
                     const int64_t *ang_seg_off, int w0, int nw, int64_t seg_lo, double *invL, cudaStream_t st)
{
    if (nw > MAX_BLOCK_ANGLES) return cudaErrorInvalidValue;
    k_invL<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, perm_blk, len64_blk, ang_seg_off, w0, nw, seg_lo, invL);
    return cudaGetLastError();
}

cudaError_t gather_units_build(int nvox, const int32_t *csr_off, int32_t *nu, int64_t *ufirst, int64_t *tmp,
                               cudaStream_t st)
{
    k_unit_count<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, nu);
    return scan_i32(nu, ufirst, nvox, tmp, st);
}

cudaError_t gather_units_fill(int nvox, const int32_t *csr_off, const int64_t *ufirst, int32_t *urow, int32_t *ubeg,
                              cudaStream_t st)
{
    k_unit_fill<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, ufirst, urow, ubeg);
    return cudaGetLastError();
}

template <typename P>
cudaError_t gather_block(int nvox, const int32_t *csr_off, const int32_t *perm_blk, const P *buf,
                         const int64_t *ang_seg_off, int w0, int nw, int64_t seg_lo, const double *invL,
                         const double *wt, const double *dirs, const int32_t *urow, const int32_t *ubeg,
                         const int64_t *ufirst, int64_t nunits, double *part, double *J, double *Lst, double *Fc,
                         int first, cudaStream_t st)
{
    if (nw > MAX_BLOCK_ANGLES) return cudaErrorInvalidValue;
    int64_t blocks = (nunits * 32 + 255) / 256;
    k_gather_units<P><<<(unsigned)blocks, 256, 0, st>>>(nvox, nunits, urow, ubeg, csr_off, perm_blk, buf, ang_seg_off,
                                                        w0, nw, seg_lo, invL, wt, dirs, part);
    k_gather_rows<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, ufirst, part, J, Lst, Fc, first);
    return cudaGetLastError();
}

cudaError_t gather_angle_range(int nvox, const int32_t *csr_off, const int32_t *perm_blk, const void *buf, int fp32,
                               int64_t s_lo, int64_t s_hi, const double *invL_w, double *Ibar, double *Lbar,
                               cudaStream_t st)
{
    if (fp32)
        k_gather_angle<float2><<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, perm_blk, (const float2 *)buf, s_lo,
                                                                   s_hi, invL_w, Ibar, Lbar);
    else
        k_gather_angle<double2><<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, perm_blk, (const double2 *)buf, s_lo,
                                                                    s_hi, invL_w, Ibar, Lbar);
    return cudaGetLastError();
}

cudaError_t flux_local(const GeomDev &G, const double *Fc, double *F, cudaStream_t st)
{
    k_flux_local<<<(G.nvox + 255) / 256, 256, 0, st>>>(G, Fc, F);
    return cudaGetLastError();
}

template cudaError_t gather_block<float2>(int, const int32_t *, const int32_t *, const float2 *, const int64_t *, int,
                                          int, int64_t, const double *, const double *, const double *, const int32_t *,
                                          const int32_t *, const int64_t *, int64_t, double *, double *, double *,
                                          double *, int, cudaStream_t);
template cudaError_t gather_block<double2>(int, const int32_t *, const int32_t *, const double2 *, const int64_t *, int,
                                           int, int64_t, const double *, const double *, const double *, const int32_t *,
                                           const int32_t *, const int64_t *, int64_t, double *, double *, double *,
                                           double *, int, cudaStream_t);

}  // namespace rtk
