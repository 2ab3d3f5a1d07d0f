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

#include <utility>
#include <stdint.h>

#include "rt_internal.h"

namespace rtk {
namespace {

constexpr double FOUR_PI = 12.566370614359172953850573533118;
constexpr int MAX_BLOCK_ANGLES = 256;
constexpr int UNIT_LEN = 32;  // ownership-list entries per gather work unit (one thread each)

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

// Ownership lists by a stable LSD radix sort of the block's segment indices
// keyed by voxel (8-bit digits): the input is in segment order, so every
// voxel's list comes out sorted by segment index, which fixes the summation
// order of the gather.  Tiles of RS_TILE segments per CTA.
constexpr int RS_TILE = 4096;
constexpr int RS_BUCKETS = 256;

__global__ void k_rs_init(const uint32_t *vox, int64_t n, uint32_t *keys, int32_t *vals)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        keys[s] = vox[s] & RTK_VOXMASK;
        vals[s] = (int32_t)s;
    }
}

// Digit counts of one tile, stored digit-major (hist[d * ntiles + t]) so that
// one exclusive scan gives every (digit, tile) its first output position.
__global__ void __launch_bounds__(256) k_rs_hist(const uint32_t *keys, int64_t n, int shift, int64_t ntiles,
                                                 int32_t *hist)
{
    __shared__ int32_t h[RS_BUCKETS];
    for (int i = threadIdx.x; i < RS_BUCKETS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += blockDim.x) {
        const int64_t e = base + i;
        if (e < n) atomicAdd(&h[(keys[e] >> shift) & (RS_BUCKETS - 1)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RS_BUCKETS; i += blockDim.x) hist[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// Stable scatter of one tile: the tile is read in rounds of 256 elements in
// order; an element's rank among equal digits is the count in earlier rounds
// (run), in earlier warps of its round (wcnt) and in earlier lanes of its warp.
__global__ void __launch_bounds__(256) k_rs_scatter(const uint32_t *__restrict__ keys, const int32_t *__restrict__ vals,
                                                    int64_t n, int shift, int64_t ntiles, const int64_t *__restrict__ off,
                                                    uint32_t *__restrict__ keys_out, int32_t *__restrict__ vals_out)
{
    __shared__ int32_t run[RS_BUCKETS];
    __shared__ int32_t wcnt[8][RS_BUCKETS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_BUCKETS; i += blockDim.x) run[i] = 0;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_TILE / 256; ++r) {
        for (int i = threadIdx.x; i < 8 * RS_BUCKETS; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t e = base + r * 256 + threadIdx.x;
        const bool ok = e < n;
        const uint32_t k = ok ? keys[e] : 0u;
        const int32_t val = ok ? vals[e] : 0;
        const int d = ok ? (int)((k >> shift) & (RS_BUCKETS - 1)) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            int before = 0;
            for (int w2 = 0; w2 < warp; ++w2) before += wcnt[w2][d];
            const int64_t pos = off[(int64_t)d * ntiles + blockIdx.x] + run[d] + before + rank;
            keys_out[pos] = k;
            vals_out[pos] = val;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < RS_BUCKETS; i += blockDim.x) {
            int t = 0;
            for (int w2 = 0; w2 < 8; ++w2) t += wcnt[w2][i];
            run[i] += t;
        }
        __syncthreads();
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
__global__ void k_gather_angle(int nvox, const int32_t *off, const int32_t *perm, const P *buf, int64_t base,
                               int64_t s_lo, int64_t s_hi, const double *invL_w, double *Ibar, double *Lbar)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    double aI = 0.0, aL = 0.0;
    for (int e = off[v]; e < off[v + 1]; ++e) {
        int s = perm[e];
        if (s < s_lo || s >= s_hi) continue;
        P val = buf[s - base];
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

// Compensated (Kahan) FP32 accumulation: the running error term c keeps the
// sum accurate to about one rounding of the total, independent of its length.
__device__ __forceinline__ void kadd(float &s, float &c, float x)
{
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// A voxel whose list fits one unit is finished by that unit's thread; the
// units of longer lists leave their sums for k_gather_rows.
__device__ __forceinline__ void finish_unit(int64_t u, int v, int64_t nunits, const int32_t *urow, double r0, double r1,
                                            double r2, double r3, double r4, double *part, double *J, double *Lst,
                                            double *Fc, int first)
{
    const bool single = (u == 0 || urow[u - 1] != v) && (u + 1 == nunits || urow[u + 1] != v);
    if (single) {
        if (!first) {
            r0 += J[v];
            r1 += Lst[v];
            r2 += Fc[3 * (int64_t)v];
            r3 += Fc[3 * (int64_t)v + 1];
            r4 += Fc[3 * (int64_t)v + 2];
        }
        J[v] = r0;
        Lst[v] = r1;
        Fc[3 * (int64_t)v] = r2;
        Fc[3 * (int64_t)v + 1] = r3;
        Fc[3 * (int64_t)v + 2] = r4;
    } else {
        double *o = part + 5 * u;
        o[0] = r0; o[1] = r1; o[2] = r2; o[3] = r3; o[4] = r4;
    }
}

// One thread per work unit (at most UNIT_LEN consecutive entries of one
// voxel's ownership list, sorted by segment hence by solid angle):
//   J += (wt_q / L_qv) (l I),  Lambda* += (wt_q / L_qv) (l lambda),  F += n_q (J term).
// FP32 ray march: FP32 weights and Kahan-compensated FP32 sums.
__global__ void __launch_bounds__(256) k_gather_units32(int nvox, int64_t nunits, const int32_t *__restrict__ urow,
                                                        const int32_t *__restrict__ order, const int32_t *__restrict__ ulen,
                                                        const int64_t *__restrict__ gbase, const int32_t *__restrict__ sell,
                                                        const float2 *__restrict__ buf,
                                                        const int64_t *__restrict__ ang_seg_off, int w0, int nw,
                                                        int64_t seg_lo, const float *__restrict__ wL,
                                                        const double *__restrict__ dirs, double *__restrict__ part,
                                                        double *J, double *Lst, double *Fc, int first)
{
    __shared__ int32_t soff[MAX_BLOCK_ANGLES + 1];
    __shared__ float sdir[3 * MAX_BLOCK_ANGLES];
    for (int q = threadIdx.x; q <= nw; q += blockDim.x) soff[q] = (int32_t)(ang_seg_off[w0 + q] - seg_lo);
    for (int q = threadIdx.x; q < 3 * nw; q += blockDim.x) sdir[q] = (float)dirs[3 * w0 + q];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nunits) return;
    const int u = order[i];
    const int v = urow[u];
    const int len = ulen[u];
    const int32_t *lst = sell + gbase[i >> 5] + (i & 31);
    float sj = 0.f, cj = 0.f, sl = 0.f, cl = 0.f, sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f;
    if (len > 0) {
        int s = lst[0];
        int lo = 0, hi = nw;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (soff[mid] <= s) lo = mid;
            else hi = mid;
        }
        int q = lo;
        float f = wL[(int64_t)(w0 + q) * nvox + v];
        // four entries per step: independent (coalesced) index loads, then buffer loads
        for (int k = 0; k < len; k += 4) {
            int ss[4];
            float2 val[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) ss[j] = (k + j < len) ? lst[32 * (k + j)] : -1;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ss[j] >= 0) val[j] = buf[ss[j]];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (ss[j] < 0) continue;
                while (ss[j] >= soff[q + 1]) {
                    ++q;
                    f = wL[(int64_t)(w0 + q) * nvox + v];
                }
                float tj = f * val[j].x;
                kadd(sj, cj, tj);
                kadd(sl, cl, f * val[j].y);
                kadd(sx, cx, sdir[3 * q] * tj);
                kadd(sy, cy, sdir[3 * q + 1] * tj);
                kadd(sz, cz, sdir[3 * q + 2] * tj);
            }
        }
    }
    const double r0 = (double)sj - (double)cj, r1 = (double)sl - (double)cl, r2 = (double)sx - (double)cx,
                 r3 = (double)sy - (double)cy, r4 = (double)sz - (double)cz;
    finish_unit(u, v, nunits, urow, r0, r1, r2, r3, r4, part, J, Lst, Fc, first);
}

// FP64 ray march: FP64 weights and sums.
__global__ void __launch_bounds__(256) k_gather_units64(int nvox, int64_t nunits, const int32_t *__restrict__ urow,
                                                        const int32_t *__restrict__ order, const int32_t *__restrict__ ulen,
                                                        const int64_t *__restrict__ gbase, const int32_t *__restrict__ sell,
                                                        const double2 *__restrict__ buf,
                                                        const int64_t *__restrict__ ang_seg_off, int w0, int nw,
                                                        int64_t seg_lo, const double *__restrict__ invL,
                                                        const double *__restrict__ wt, const double *__restrict__ dirs,
                                                        double *__restrict__ part, double *J, double *Lst, double *Fc,
                                                        int first)
{
    __shared__ int32_t soff[MAX_BLOCK_ANGLES + 1];
    __shared__ double swt[MAX_BLOCK_ANGLES], sdir[3 * MAX_BLOCK_ANGLES];
    for (int q = threadIdx.x; q <= nw; q += blockDim.x) soff[q] = (int32_t)(ang_seg_off[w0 + q] - seg_lo);
    for (int q = threadIdx.x; q < nw; q += blockDim.x) swt[q] = wt[w0 + q];
    for (int q = threadIdx.x; q < 3 * nw; q += blockDim.x) sdir[q] = dirs[3 * w0 + q];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nunits) return;
    const int u = order[i];
    const int v = urow[u];
    const int len = ulen[u];
    const int32_t *lst = sell + gbase[i >> 5] + (i & 31);
    double aj = 0.0, al = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    if (len > 0) {
        int s = lst[0];
        int lo = 0, hi = nw;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (soff[mid] <= s) lo = mid;
            else hi = mid;
        }
        int q = lo;
        double f = swt[q] * invL[(int64_t)(w0 + q) * nvox + v];
        for (int k = 0; k < len; ++k) {
            s = lst[32 * k];
            while (s >= soff[q + 1]) {
                ++q;
                f = swt[q] * invL[(int64_t)(w0 + q) * nvox + v];
            }
            double2 val = buf[s];
            double tj = f * val.x;
            aj += tj;
            al += f * val.y;
            fx += sdir[3 * q] * tj;
            fy += sdir[3 * q + 1] * tj;
            fz += sdir[3 * q + 2] * tj;
        }
    }
    finish_unit(u, v, nunits, urow, aj, al, fx, fy, fz, part, J, Lst, Fc, first);
}

__global__ void k_make_wL32(int64_t n, int nvox, const double *invL, const double *wt, float *wL)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        wL[i] = (float)(wt[i / nvox] * invL[i]);
}

// One thread per voxel with more than one unit: add its unit sums in order.
__global__ void k_gather_rows(int nmulti, const int32_t *__restrict__ multi, const int64_t *__restrict__ ufirst,
                              const double *__restrict__ part, double *J, double *Lst, double *Fc, int first)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmulti) return;
    const int v = multi[i];
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

// Voxels whose ownership list needs more than one unit (compacted in voxel order).
__global__ void k_multi_flags(int nvox, const int64_t *ufirst, int32_t *flag)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nvox) flag[v] = (ufirst[v + 1] - ufirst[v] > 1) ? 1 : 0;
}

__global__ void k_multi_fill(int nvox, const int32_t *flag, const int64_t *pos, int32_t *multi)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nvox && flag[v]) multi[pos[v]] = v;
}

// Sliced-ELL layout of the work units for coalesced list reads: units are
// bucketed by length (longest first), cut into groups of 32, and the entries
// of a group interleaved: entry k of the group's unit t sits at
// sell[base_g + 32 k + t] (-1 pads short units).  Thread t then reads entry k
// at consecutive addresses with its 31 neighbours.
__global__ void k_unit_len(int64_t nunits, const int32_t *urow, const int32_t *ubeg, const int32_t *off, int32_t *ulen,
                           int32_t *hist)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nunits; u += (int64_t)gridDim.x * blockDim.x) {
        const int v = urow[u];
        const int e1 = (u + 1 < nunits && urow[u + 1] == v) ? ubeg[u + 1] : off[v + 1];
        const int len = e1 - ubeg[u];
        ulen[u] = len;
        atomicAdd(hist + (UNIT_LEN - len), 1);
    }
}

__global__ void k_hist_scan(int32_t *hist)  // exclusive scan of UNIT_LEN + 1 buckets, in place
{
    int run = 0;
    for (int b = 0; b <= UNIT_LEN; ++b) {
        int c = hist[b];
        hist[b] = run;
        run += c;
    }
}

__global__ void k_bucket_fill(int64_t nunits, const int32_t *ulen, int32_t *cursor, int32_t *order)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nunits; u += (int64_t)gridDim.x * blockDim.x) {
        int pos = atomicAdd(cursor + (UNIT_LEN - ulen[u]), 1);
        order[pos] = (int32_t)u;
    }
}

__global__ void k_group_width(int64_t ngroups, const int32_t *order, const int32_t *ulen, int32_t *gw)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < ngroups) gw[g] = 32 * ulen[order[32 * g]];
}

__global__ void k_sell_fill(int64_t nunits, const int32_t *order, const int32_t *ulen, const int32_t *ubeg,
                            const int32_t *perm, const int64_t *gbase, int32_t *sell)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nunits; i += (int64_t)gridDim.x * blockDim.x) {
        const int u = order[i];
        const int64_t g = i >> 5;
        const int t = (int)(i & 31);
        const int width = ulen[order[32 * g]];
        const int len = ulen[u], e0 = ubeg[u];
        int32_t *dst = sell + gbase[g] + t;
        for (int k = 0; k < width; ++k) dst[32 * k] = (k < len) ? perm[e0 + k] : -1;
    }
}

// ---------------------------------------------------------------------------
// J-only gather of the ALI iteration.  Lists of at most SHORT_LEN entries are
// summed by one thread each, from a sliced-ELL copy (voxels sorted by list
// length, 32 per group, entries interleaved so the 32 threads of a warp read
// consecutive words); longer lists are cut into chunks of CHUNK_LEN entries,
// one warp per chunk reading the list coalesced, and the warp that finishes a
// voxel's last chunk adds the chunk sums in chunk order.
constexpr int SHORT_LEN = RTK_JSHORT;
constexpr int CHUNK_LEN = RTK_JCHUNK;

__global__ void k_jclass(int nvox, const int32_t *off, int32_t *hist, int32_t *longflag, int32_t *nch)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    int L = off[v + 1] - off[v];
    if (L <= SHORT_LEN) {
        atomicAdd(hist + (SHORT_LEN - L), 1);
        longflag[v] = 0;
        nch[v] = 0;
    } else {
        longflag[v] = 1;
        nch[v] = (L + CHUNK_LEN - 1) / CHUNK_LEN;
    }
}

__global__ void k_jhist_scan(int32_t *hist)
{
    int run = 0;
    for (int b = 0; b <= SHORT_LEN; ++b) {
        int c = hist[b];
        hist[b] = run;
        run += c;
    }
}

__global__ void k_jshort_fill(int nvox, const int32_t *off, int32_t *cursor, int32_t *jorder)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    int L = off[v + 1] - off[v];
    if (L <= SHORT_LEN) jorder[atomicAdd(cursor + (SHORT_LEN - L), 1)] = v;
}

__global__ void k_jwidth(int64_t ngroups, const int32_t *off, const int32_t *jorder, int32_t *gw)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < ngroups) {
        int v = jorder[32 * g];
        gw[g] = 32 * (off[v + 1] - off[v]);
    }
}

__global__ void k_jsell_fill(int64_t nshort, const int32_t *off, const int32_t *jorder, const int32_t *perm,
                             const int64_t *gbase, int32_t *sell)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nshort; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = jorder[i];
        const int64_t g = i >> 5;
        const int v0 = jorder[32 * g];
        const int width = off[v0 + 1] - off[v0];
        const int L = off[v + 1] - off[v], e0 = off[v];
        int32_t *dst = sell + gbase[g] + (i & 31);
        for (int k = 0; k < width; ++k) dst[32 * k] = (k < L) ? perm[e0 + k] : -1;
    }
}

__global__ void k_jlong_fill(int nvox, const int32_t *off, const int32_t *longflag, const int64_t *lpos,
                             const int64_t *cpos, int32_t *lrows, int32_t *lfirst, int32_t *crow, int32_t *cbeg,
                             int32_t *clr)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox || !longflag[v]) return;
    const int lr = (int)lpos[v];
    const int c0 = (int)cpos[v], c1 = (int)cpos[v + 1];
    lrows[lr] = v;
    lfirst[lr] = c0;
    for (int c = c0; c < c1; ++c) {
        crow[c] = v;
        cbeg[c] = off[v] + (c - c0) * CHUNK_LEN;
        clr[c] = lr;
    }
}

template <typename T> struct JW;
template <> struct JW<float> {
    __device__ static float weight(const float *wL, const double *, const double *, int w, int q, int nvox, int v)
    {
        (void)q;
        return wL[(int64_t)w * nvox + v];
    }
};
template <> struct JW<double> {
    __device__ static double weight(const float *, const double *swt, const double *invL, int w, int q, int nvox, int v)
    {
        return swt[q] * invL[(int64_t)w * nvox + v];
    }
};

template <typename T> struct JAcc;
template <> struct JAcc<float> {  // Kahan-compensated FP32
    float s = 0.f, c = 0.f;
    __device__ void add(float x) { kadd(s, c, x); }
    __device__ double value() const { return (double)s - (double)c; }
    __device__ void warp_reduce()
    {
        for (int o = 16; o > 0; o >>= 1) {
            float s2 = __shfl_xor_sync(0xffffffffu, s, o);
            float c2 = __shfl_xor_sync(0xffffffffu, c, o);
            float t = s + s2;
            float bb = t - s;
            float err = (s - (t - bb)) + (s2 - bb);  // s + s2 = t + err exactly
            c = (c + c2) - err;
            s = t;
        }
    }
};
template <> struct JAcc<double> {
    double s = 0.0;
    __device__ void add(double x) { s += x; }
    __device__ double value() const { return s; }
    __device__ void warp_reduce()
    {
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
};

__device__ __forceinline__ int angle_of(const int32_t *soff, int nw, int s)
{
    int lo = 0, hi = nw;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (soff[mid] <= s) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One short list (thread i of the sliced-ELL order) into J.
template <typename T>
__device__ __forceinline__ void gj_short(int64_t i, int nvox, const int32_t *__restrict__ off,
                                         const int32_t *__restrict__ jorder, const int64_t *__restrict__ jgbase,
                                         const int32_t *__restrict__ jsell, const T *__restrict__ buf,
                                         const int32_t *soff, const double *swt, int w0, int nw,
                                         const float *__restrict__ wL, const double *__restrict__ invL, double *J,
                                         int first)
{
    const int v = jorder[i];
    const int L = off[v + 1] - off[v];
    const int32_t *lst = jsell + jgbase[i >> 5] + (i & 31);
    JAcc<T> acc;
    if (L > 0) {
        int q = angle_of(soff, nw, lst[0]);
        T f = JW<T>::weight(wL, swt, invL, w0 + q, q, nvox, v);
        for (int k = 0; k < L; k += 4) {
            int ss[4];
            T val[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) ss[j] = (k + j < L) ? lst[32 * (k + j)] : -1;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ss[j] >= 0) val[j] = buf[ss[j]];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (ss[j] < 0) continue;
                while (ss[j] >= soff[q + 1]) {
                    ++q;
                    f = JW<T>::weight(wL, swt, invL, w0 + q, q, nvox, v);
                }
                acc.add(f * val[j]);
            }
        }
    }
    const double r = acc.value();
    J[v] = first ? r : J[v] + r;
}

// One chunk of a long list (one warp); the warp that completes a voxel's last
// chunk adds all its chunk sums in chunk order.
template <typename T>
__device__ __forceinline__ void gj_chunk(int64_t c, int lane, int nvox, const int32_t *__restrict__ off,
                                         const int32_t *__restrict__ perm, int64_t nchunks,
                                         const int32_t *__restrict__ crow, const int32_t *__restrict__ cbeg,
                                         const int32_t *__restrict__ clr, const int32_t *__restrict__ lfirst, int nlong,
                                         int *cnt, double *part, const T *__restrict__ buf, const int32_t *soff,
                                         const double *swt, int w0, int nw, const float *__restrict__ wL,
                                         const double *__restrict__ invL, double *J, int first)
{
    const int v = crow[c];
    const int e0 = cbeg[c];
    const int e1 = min(e0 + CHUNK_LEN, off[v + 1]);
    JAcc<T> acc;
    for (int e = e0 + lane; e < e1; e += 32) {
        const int s = perm[e];
        const int q = angle_of(soff, nw, s);
        acc.add(JW<T>::weight(wL, swt, invL, w0 + q, q, nvox, v) * buf[s]);
    }
    acc.warp_reduce();
    if (lane == 0) {
        const int lr = clr[c];
        __stcg(part + c, acc.value());
        __threadfence();
        const int c0 = lfirst[lr], c1 = (lr + 1 < nlong) ? lfirst[lr + 1] : (int)nchunks;
        if (atomicAdd(cnt + lr, 1) == c1 - c0 - 1) {
            __threadfence();
            double r = 0.0;
            for (int cc = c0; cc < c1; ++cc) r += __ldcg(part + cc);
            J[v] = first ? r : J[v] + r;
            cnt[lr] = 0;
        }
    }
}

// Blocks [0, nbs) sum short lists (thread per voxel); the rest are warps over chunks of long lists.
template <typename T>
__global__ void __launch_bounds__(256) k_gatherJ(int nvox, int64_t nshort, int nbs, const int32_t *__restrict__ off,
                                                 const int32_t *__restrict__ jorder, const int64_t *__restrict__ jgbase,
                                                 const int32_t *__restrict__ jsell, int64_t nchunks,
                                                 const int32_t *__restrict__ crow, const int32_t *__restrict__ cbeg,
                                                 const int32_t *__restrict__ clr, const int32_t *__restrict__ lfirst,
                                                 int nlong, int *cnt, double *part, const int32_t *__restrict__ perm,
                                                 const T *__restrict__ buf, const int64_t *__restrict__ ang_seg_off,
                                                 int w0, int nw, int64_t seg_lo, const float *__restrict__ wL,
                                                 const double *__restrict__ invL, const double *__restrict__ wt,
                                                 double *J, int first)
{
    __shared__ int32_t soff[MAX_BLOCK_ANGLES + 1];
    __shared__ double swt[MAX_BLOCK_ANGLES];
    for (int q = threadIdx.x; q <= nw; q += blockDim.x) soff[q] = (int32_t)(ang_seg_off[w0 + q] - seg_lo);
    for (int q = threadIdx.x; q < nw; q += blockDim.x) swt[q] = wt[w0 + q];
    __syncthreads();
    if ((int)blockIdx.x < nbs) {
        const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (i < nshort) gj_short<T>(i, nvox, off, jorder, jgbase, jsell, buf, soff, swt, w0, nw, wL, invL, J, first);
        return;
    }
    const int64_t c = ((int64_t)(blockIdx.x - nbs) * blockDim.x + threadIdx.x) >> 5;
    if (c < nchunks)
        gj_chunk<T>(c, threadIdx.x & 31, nvox, off, perm, nchunks, crow, cbeg, clr, lfirst, nlong, cnt, part, buf, soff,
                    swt, w0, nw, wL, invL, J, first);
}

// Persistent batched J gather (FP32): every CTA takes work units (one block
// worth of short lists or chunks of one member's angle block) from a device
// counter; wpfx[i] = first work unit of item i.
__global__ void __launch_bounds__(256) k_gatherJ_batch(const GatherItem *__restrict__ items,
                                                       const int64_t *__restrict__ wpfx, int n_items, int64_t total,
                                                       unsigned long long *counter)
{
    __shared__ int32_t soff[MAX_BLOCK_ANGLES + 1];
    __shared__ double swt[MAX_BLOCK_ANGLES];
    __shared__ long long s_unit;
    __shared__ int s_item;
    for (int guard = 0; guard < (1 << 30); ++guard) {
        if (threadIdx.x == 0) {
            unsigned long long u = atomicAdd(counter, 1ull);
            int lo = 0, hi = n_items;
            if ((int64_t)u < total) {
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if (wpfx[mid] <= (int64_t)u) lo = mid;
                    else hi = mid;
                }
            }
            s_unit = (long long)u;
            s_item = lo;
        }
        __syncthreads();
        const int64_t u = s_unit;
        if (u >= total) return;
        const GatherItem &it = items[s_item];
        for (int q = threadIdx.x; q <= it.nw; q += blockDim.x)
            soff[q] = (int32_t)(it.ang_seg_off[it.w0 + q] - it.seg_lo);
        for (int q = threadIdx.x; q < it.nw; q += blockDim.x) swt[q] = it.wt[it.w0 + q];
        __syncthreads();
        const int64_t bi = u - wpfx[s_item];
        if (bi < it.nbs) {
            const int64_t i = bi * blockDim.x + threadIdx.x;
            if (i < it.t.nshort)
                gj_short<float>(i, it.nvox, it.off, it.t.jorder, it.t.jgbase, it.t.jsell, it.buf, soff, swt, it.w0,
                                it.nw, it.wL, it.invL, it.J, it.first);
        } else {
            const int64_t c = ((bi - it.nbs) * blockDim.x + threadIdx.x) >> 5;
            if (c < it.t.nchunks)
                gj_chunk<float>(c, threadIdx.x & 31, it.nvox, it.off, it.perm, it.t.nchunks, it.t.crow, it.t.cbeg,
                                it.t.clr, it.t.lfirst, it.t.nlong, it.t.cnt, it.part, it.buf, soff, swt, it.w0, it.nw,
                                it.wL, it.invL, it.J, it.first);
        }
        __syncthreads();
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int64_t radix_tiles(int64_t n) { return (n + RS_TILE - 1) / RS_TILE; }

cudaError_t csr_build(int nvox, const uint32_t *vox_blk, int64_t nseg_blk, int32_t *counts, int32_t *csr_off,
                      int32_t *perm_blk, int64_t *tmp, const RadixScratch &rs, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * nvox, st);
    if (e != cudaSuccess) return e;
    if (nseg_blk > rs.cap) return cudaErrorInvalidValue;
    k_count_vox<<<grid_for(nseg_blk, 256), 256, 0, st>>>(vox_blk, nseg_blk, counts);
    // offsets in int64 scratch, then narrowed (a block holds < 2^31 segments)
    int64_t *off64 = tmp;
    int64_t *stmp = tmp + (nvox + 1);
    if ((e = scan_i32(counts, off64, nvox, stmp, st)) != cudaSuccess) return e;
    k_off32<<<(nvox + 256) / 256, 256, 0, st>>>(off64, csr_off, nvox + 1);
    if (nseg_blk <= 0) return cudaGetLastError();
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)nvox) ++bits;
    const int passes = (bits + 7) / 8;
    k_rs_init<<<grid_for(nseg_blk, 256), 256, 0, st>>>(vox_blk, nseg_blk, rs.kA, passes ? rs.vA : perm_blk);
    const int64_t ntiles = radix_tiles(nseg_blk);
    uint32_t *kin = rs.kA, *kout = rs.kB;
    int32_t *vin = rs.vA, *vout = rs.vB;
    for (int p = 0; p < passes; ++p) {
        if (p == passes - 1) vout = perm_blk;
        k_rs_hist<<<(unsigned)ntiles, 256, 0, st>>>(kin, nseg_blk, 8 * p, ntiles, rs.hist);
        if ((e = scan_i32(rs.hist, rs.off, RS_BUCKETS * ntiles, rs.tmp, st)) != cudaSuccess) return e;
        k_rs_scatter<<<(unsigned)ntiles, 256, 0, st>>>(kin, vin, nseg_blk, 8 * p, ntiles, rs.off, kout, vout);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
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

cudaError_t make_wL32(int n_ang, int nvox, const double *invL, const double *wt, float *wL, cudaStream_t st)
{
    int64_t n = (int64_t)n_ang * nvox;
    k_make_wL32<<<grid_for(n, 256), 256, 0, st>>>(n, nvox, invL, wt, wL);
    return cudaGetLastError();
}

template <typename P>
cudaError_t gather_block(int nvox, const int32_t *csr_off, const int32_t *perm_blk, const P *buf,
                         const int64_t *ang_seg_off, int w0, int nw, int64_t seg_lo, const double *invL,
                         const float *wL32, const double *wt, const double *dirs, const int32_t *urow,
                         const int32_t *ubeg, const int64_t *ufirst, int64_t nunits, const int32_t *multi,
                         int nmulti, const int32_t *order, const int32_t *ulen, const int64_t *gbase,
                         const int32_t *sell, double *part, double *J, double *Lst, double *Fc, int first,
                         cudaStream_t st)
{
    (void)csr_off;
    (void)perm_blk;
    (void)ubeg;
    if (nw > MAX_BLOCK_ANGLES) return cudaErrorInvalidValue;
    unsigned blocks = (unsigned)((nunits + 255) / 256);
    if constexpr (sizeof(P) == sizeof(float2))
        k_gather_units32<<<blocks, 256, 0, st>>>(nvox, nunits, urow, order, ulen, gbase, sell, (const float2 *)buf,
                                                 ang_seg_off, w0, nw, seg_lo, wL32, dirs, part, J, Lst, Fc, first);
    else
        k_gather_units64<<<blocks, 256, 0, st>>>(nvox, nunits, urow, order, ulen, gbase, sell, (const double2 *)buf,
                                                 ang_seg_off, w0, nw, seg_lo, invL, wt, dirs, part, J, Lst, Fc, first);
    if (nmulti > 0) k_gather_rows<<<(nmulti + 255) / 256, 256, 0, st>>>(nmulti, multi, ufirst, part, J, Lst, Fc, first);
    return cudaGetLastError();
}

cudaError_t sell_order(int64_t nunits, const int32_t *urow, const int32_t *ubeg, const int32_t *csr_off, int32_t *ulen,
                       int32_t *hist, int32_t *order, int32_t *gw, cudaStream_t st)
{
    if (nunits <= 0) return cudaSuccess;
    if (!urow || !ubeg || !csr_off || !ulen || !hist || !order || !gw) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (UNIT_LEN + 1), st);
    if (e != cudaSuccess) return e;
    k_unit_len<<<grid_for(nunits, 256), 256, 0, st>>>(nunits, urow, ubeg, csr_off, ulen, hist);
    k_hist_scan<<<1, 1, 0, st>>>(hist);
    k_bucket_fill<<<grid_for(nunits, 256), 256, 0, st>>>(nunits, ulen, hist, order);
    int64_t ng = (nunits + 31) / 32;
    k_group_width<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(ng, order, ulen, gw);
    return cudaGetLastError();
}

cudaError_t sell_fill(int64_t nunits, const int32_t *order, const int32_t *ulen, const int32_t *ubeg,
                      const int32_t *perm_blk, const int64_t *gbase, int32_t *sell, cudaStream_t st)
{
    if (nunits <= 0) return cudaSuccess;
    if (!order || !ulen || !ubeg || !perm_blk || !gbase || !sell) return cudaErrorInvalidValue;
    k_sell_fill<<<grid_for(nunits, 256), 256, 0, st>>>(nunits, order, ulen, ubeg, perm_blk, gbase, sell);
    return cudaGetLastError();
}

cudaError_t gather_multi_rows(int nvox, const int64_t *ufirst, int32_t *flag, int64_t *pos, int64_t *tmp,
                              int32_t *multi, cudaStream_t st)
{
    k_multi_flags<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, ufirst, flag);
    cudaError_t e = scan_i32(flag, pos, nvox, tmp, st);
    if (e != cudaSuccess) return e;
    if (multi) k_multi_fill<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, flag, pos, multi);
    return cudaGetLastError();
}

cudaError_t gather_angle_range(int nvox, const int32_t *csr_off, const int32_t *perm_blk, const void *buf,
                               int64_t buf_base, int fp32, int64_t s_lo, int64_t s_hi, const double *invL_w,
                               double *Ibar, double *Lbar, cudaStream_t st)
{
    if (fp32)
        k_gather_angle<float2><<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, perm_blk, (const float2 *)buf,
                                                                   buf_base, s_lo, s_hi, invL_w, Ibar, Lbar);
    else
        k_gather_angle<double2><<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, perm_blk, (const double2 *)buf,
                                                                    buf_base, s_lo, s_hi, invL_w, Ibar, Lbar);
    return cudaGetLastError();
}

cudaError_t gather_angle_preload()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_gather_angle<float2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_gather_angle<double2>);
    return e;
}

cudaError_t flux_local(const GeomDev &G, const double *Fc, double *F, cudaStream_t st)
{
    k_flux_local<<<(G.nvox + 255) / 256, 256, 0, st>>>(G, Fc, F);
    return cudaGetLastError();
}

cudaError_t gatherJ_classify(int nvox, const int32_t *csr_off, int32_t *hist, int32_t *longflag, int32_t *nch,
                             cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (SHORT_LEN + 1), st);
    if (e != cudaSuccess) return e;
    k_jclass<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, hist, longflag, nch);
    return cudaGetLastError();
}

cudaError_t gatherJ_short(int nvox, const int32_t *csr_off, int32_t *hist, int32_t *jorder, int64_t nshort, int32_t *gw,
                          cudaStream_t st)
{
    k_jhist_scan<<<1, 1, 0, st>>>(hist);
    k_jshort_fill<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, hist, jorder);
    int64_t ng = (nshort + 31) / 32;
    if (ng > 0) k_jwidth<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(ng, csr_off, jorder, gw);
    return cudaGetLastError();
}

cudaError_t gatherJ_sell(int64_t nshort, const int32_t *csr_off, const int32_t *jorder, const int32_t *perm_blk,
                         const int64_t *gbase, int32_t *sell, cudaStream_t st)
{
    if (nshort <= 0) return cudaSuccess;
    k_jsell_fill<<<grid_for(nshort, 256), 256, 0, st>>>(nshort, csr_off, jorder, perm_blk, gbase, sell);
    return cudaGetLastError();
}

cudaError_t gatherJ_long(int nvox, const int32_t *csr_off, const int32_t *longflag, const int64_t *lpos,
                         const int64_t *cpos, int32_t *lrows, int32_t *lfirst, int32_t *crow, int32_t *cbeg,
                         int32_t *clr, cudaStream_t st)
{
    k_jlong_fill<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, csr_off, longflag, lpos, cpos, lrows, lfirst, crow, cbeg, clr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_J(int nvox, const int32_t *csr_off, const GatherJTables &t, const int32_t *perm_blk, const T *buf,
                     const int64_t *ang_seg_off, int w0, int nw, int64_t seg_lo, const float *wL32,
                     const double *invL, const double *wt, double *part, double *J, int first, cudaStream_t st)
{
    if (nw > MAX_BLOCK_ANGLES) return cudaErrorInvalidValue;
    const int nbs = (int)((t.nshort + 255) / 256);
    const int64_t nbc = (t.nchunks * 32 + 255) / 256;
    const int64_t grid = nbs + nbc;
    if (grid <= 0) return cudaSuccess;
    k_gatherJ<T><<<(unsigned)grid, 256, 0, st>>>(nvox, t.nshort, nbs, csr_off, t.jorder, t.jgbase, t.jsell, t.nchunks,
                                                 t.crow, t.cbeg, t.clr, t.lfirst, t.nlong, t.cnt, part, perm_blk, buf,
                                                 ang_seg_off, w0, nw, seg_lo, wL32, invL, wt, J, first);
    return cudaGetLastError();
}

cudaError_t gather_J_batch(const GatherItem *items, const int64_t *wpfx, int n_items, int64_t total,
                           unsigned long long *counter, int grid_blocks, cudaStream_t st)
{
    if (total <= 0) return cudaSuccess;
    k_gatherJ_batch<<<grid_blocks, 256, 0, st>>>(items, wpfx, n_items, total, counter);
    return cudaGetLastError();
}

template cudaError_t gather_J<float>(int, const int32_t *, const GatherJTables &, const int32_t *, const float *,
                                     const int64_t *, int, int, int64_t, const float *, const double *, const double *,
                                     double *, double *, int, cudaStream_t);
template cudaError_t gather_J<double>(int, const int32_t *, const GatherJTables &, const int32_t *, const double *,
                                      const int64_t *, int, int, int64_t, const float *, const double *, const double *,
                                      double *, double *, int, cudaStream_t);

template cudaError_t gather_block<float2>(int, const int32_t *, const int32_t *, const float2 *, const int64_t *, int,
                                          int, int64_t, const double *, const float *, const double *, const double *,
                                          const int32_t *, const int32_t *, const int64_t *, int64_t, const int32_t *,
                                          int, const int32_t *, const int32_t *, const int64_t *, const int32_t *,
                                          double *, double *, double *, double *, int, cudaStream_t);
template cudaError_t gather_block<double2>(int, const int32_t *, const int32_t *, const double2 *, const int64_t *, int,
                                           int, int64_t, const double *, const float *, const double *, const double *,
                                           const int32_t *, const int32_t *, const int64_t *, int64_t, const int32_t *,
                                           int, const int32_t *, const int32_t *, const int64_t *, const int32_t *,
                                           double *, double *, double *, double *, int, cudaStream_t);

}  // namespace rtk
