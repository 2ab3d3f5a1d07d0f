// march.cu -- formal solution along the characteristics (Hauschildt & Baron
// IV, Sect. 2; scheme of Papers I-II, read here as the voxel-node parabolic
// long-characteristic recurrence R6):
//
//   I_k = I_{k-1} e^{-dtau_k} + alpha_k S_{k-1} + beta_k S_k + gamma_k S_{k+1},
//   dtau_k = chi(v_k) l_k,
//
// and the local Lambda* element lambda_k = dI_k/dS_k (R9).
//
// One warp owns a bundle of consecutive whole characteristics (about `chunk`
// segments) and walks their concatenated segment stream 32 segments at a
// time: each lane loads one segment (coalesced id and length streams), gathers
// (chi, S) of its voxel, takes the neighbours' values by shuffles, builds its
// affine map I -> A I + b, and the warp composes the maps with an inclusive
// shuffle scan, so the sequential recurrence costs log2(32) steps per 32
// segments.  A characteristic start sets A = 0, which cuts the scan there.
// Output per segment: (l I_k, l lambda_k) for the ownership gather.
#include <cuda_runtime.h>
#include <stdint.h>

#include "coef.cuh"
#include "rt_internal.h"

namespace rtk {
namespace {

template <typename T> struct Traits;
template <> struct Traits<double> { using C = Coef64; };
template <> struct Traits<float> { using C = Coef32; };

__device__ __forceinline__ int64_t lower_bound64(const int64_t *a, int64_t lo, int64_t hi, int64_t key)
{
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One warp per bundle of whole characteristics; each lane owns K consecutive
// segments of a 32K-segment tile, runs the recurrence over them serially and
// contributes one composed affine map I -> A I + b to a warp shuffle scan, so
// the scan, shuffle and index work per segment is divided by K.  The next
// tile's segment words and lengths are fetched before the current tile is
// processed.
// Bundle wg of one angle block.  BITS: the parabola choice of segment s comes
// from bit s of pbits (per-member choices of a batch) instead of RTK_PARA.
// RAWI: store I_k itself (not l I_k) when LAM is false.
template <typename T, typename P, int K, bool LAM, bool BITS, bool RAWI = false>
__device__ __forceinline__ void march_bundle(const uint32_t *__restrict__ vox, const T *__restrict__ len,
                                             const int64_t *__restrict__ ray_off, int64_t r_lo, int64_t r_hi,
                                             int64_t seg_lo, int64_t nseg, int64_t wg, const P *__restrict__ cs,
                                             const T *__restrict__ Bv, T I_outer, int homog, void *__restrict__ outv,
                                             int chunk, const uint32_t *__restrict__ pbits)
{
    using C = typename Traits<T>::C;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t c_lo = wg * chunk;
    if (c_lo >= nseg) return;
    const int64_t c_hi = (c_lo + chunk < nseg) ? c_lo + chunk : nseg;
    const int64_t ra = lower_bound64(ray_off, r_lo, r_hi, seg_lo + c_lo);
    const int64_t rb = lower_bound64(ray_off, r_lo, r_hi, seg_lo + c_hi);
    const int s_begin = (int)(ray_off[ra] - seg_lo);
    const int s_end = (int)(ray_off[rb] - seg_lo);
    if (s_begin >= s_end) return;
    const uint32_t *vx = vox + seg_lo;
    const T *ln = len + seg_lo;
    T Icarry = 0, Sprev = 0, gprev = 0;
    // segment words and lengths of the current tile; the next tile's are
    // fetched before the current one is processed (software pipelining)
    uint32_t w[K];
    T l[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int s = s_begin + K * lane + j;
        w[j] = (s < s_end) ? __ldcs(vx + s) : 0u;
        l[j] = (s < s_end) ? __ldcs(ln + s) : (T)0;
    }
    for (int base = s_begin; base < s_end; base += 32 * K) {
        const int s0 = base + K * lane;
        uint32_t wN[K];
        T lN[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int s = base + 32 * K + K * lane + j;
            wN[j] = (s < s_end) ? __ldcs(vx + s) : 0u;
            lN[j] = (s < s_end) ? __ldcs(ln + s) : (T)0;
        }
        T chi[K], S[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            chi[j] = 0;
            S[j] = 0;
            if (s0 + j < s_end) {
                P c = cs[w[j] & RTK_VOXMASK];
                chi[j] = c.x;
                S[j] = c.y;
            }
        }
        // the segment after this lane's last one (lane 31: first of the next tile)
        uint32_t wn = __shfl_down_sync(FULL, w[0], 1);
        T lnx = __shfl_down_sync(FULL, l[0], 1);
        T chin = __shfl_down_sync(FULL, chi[0], 1);
        T Snx = __shfl_down_sync(FULL, S[0], 1);
        const uint32_t wn31 = __shfl_sync(FULL, wN[0], 0);
        const T ln31 = __shfl_sync(FULL, lN[0], 0);
        if (lane == 31) {
            const int sn = base + 32 * K;
            if (sn < s_end) {
                wn = wn31;
                lnx = ln31;
                P c = cs[wn & RTK_VOXMASK];
                chin = c.x;
                Snx = c.y;
            } else {
                wn = RTK_RAYSTART;
            }
        }
        // the segment before this lane's first one
        T Sp = __shfl_up_sync(FULL, S[K - 1], 1);
        if (lane == 0) Sp = Sprev;
        T A[K], b[K], lam[K];
        T gam_prev_lane;  // gamma of the previous lane's last segment, filled after the coefficients
        T E[K], al[K], be[K], ga[K];
        bool run0[K], paraj[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int s = s0 + j;
            const bool valid = s < s_end;
            const uint32_t wnx = (j + 1 < K) ? w[j + 1] : wn;
            const T lnn = (j + 1 < K) ? l[j + 1] : lnx;
            const T chn = (j + 1 < K) ? chi[j + 1] : chin;
            const bool last = (s + 1 >= s_end) || ((wnx & (RTK_RAYSTART | RTK_RESTART)) != 0u);
            run0[j] = (w[j] & (RTK_RAYSTART | RTK_RESTART)) != 0u;
            const T x = valid ? chi[j] * l[j] : (T)1;
            const T pp = last ? (T)0 : chn * lnn;
            bool para = (w[j] & RTK_PARA) != 0u;
            if (BITS) {
                const int64_t gs = seg_lo + s;
                para = valid && ((pbits[gs >> 5] >> (gs & 31)) & 1u);
            }
            paraj[j] = para;
            C::eval(x, pp, para, E[j], al[j], be[j], ga[j]);
        }
        gam_prev_lane = __shfl_up_sync(FULL, ga[K - 1], 1);
        if (lane == 0) gam_prev_lane = gprev;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int s = s0 + j;
            const bool valid = s < s_end;
            const T Sm = (j == 0) ? Sp : S[j - 1];
            const T gm = (j == 0) ? gam_prev_lane : ga[j - 1];
            const T Sn = (j + 1 < K) ? S[j + 1] : Snx;
            const bool para = paraj[j];
            const T Skm = run0[j] ? S[j] : Sm;
            const T src = al[j] * Skm + be[j] * S[j] + (para ? ga[j] * Sn : (T)0);
            if (LAM) lam[j] = be[j] + (run0[j] ? al[j] : gm * E[j]);
            A[j] = E[j];
            b[j] = src;
            if (w[j] & RTK_RAYSTART) {
                T Iin = homog ? (T)0 : ((w[j] & RTK_CORE) ? Bv[w[j] & RTK_VOXMASK] : I_outer);
                b[j] = E[j] * Iin + src;
                A[j] = 0;
            }
            if (!valid) {
                A[j] = 1;
                b[j] = 0;
            }
        }
        // compose this lane's maps, then an exclusive warp scan over lanes
        T LA = A[0], LB = b[0];
#pragma unroll
        for (int j = 1; j < K; ++j) {
            LB = A[j] * LB + b[j];
            LA = A[j] * LA;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T Ao = __shfl_up_sync(FULL, LA, o);
            T bo = __shfl_up_sync(FULL, LB, o);
            if (lane >= o) {
                LB = LA * bo + LB;
                LA = LA * Ao;
            }
        }
        // exclusive prefix = inclusive prefix of the previous lane
        T PA = __shfl_up_sync(FULL, LA, 1);
        T PB = __shfl_up_sync(FULL, LB, 1);
        if (lane == 0) {
            PA = 1;
            PB = 0;
        }
        T I = PA * Icarry + PB;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            I = A[j] * I + b[j];
            if (s0 + j < s_end) {
                if (LAM) {
                    P o;
                    o.x = l[j] * I;
                    o.y = l[j] * lam[j];
                    __stcg((P *)outv + s0 + j, o);
                } else {
                    __stcg((T *)outv + s0 + j, RAWI ? I : l[j] * I);
                }
            }
        }
        Icarry = __shfl_sync(FULL, I, 31);
        Sprev = __shfl_sync(FULL, S[K - 1], 31);
        gprev = __shfl_sync(FULL, ga[K - 1], 31);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            w[j] = wN[j];
            l[j] = lN[j];
        }
    }
}

template <typename T, typename P, int K, bool LAM>
__global__ void __launch_bounds__(256) k_march4(const uint32_t *__restrict__ vox, const T *__restrict__ len,
                                                const int64_t *__restrict__ ray_off, int64_t r_lo, int64_t r_hi,
                                                int64_t seg_lo, int64_t nseg, const P *__restrict__ cs,
                                                const T *__restrict__ Bv, T I_outer, int homog,
                                                void *__restrict__ outv, int chunk)
{
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    march_bundle<T, P, K, LAM, false>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, wg, cs, Bv, I_outer, homog, outv,
                                      chunk, nullptr);
}

// FP64 march writing I_k per segment (forward intensities for the adjoint).
__global__ void __launch_bounds__(256) k_march_I(const uint32_t *__restrict__ vox, const double *__restrict__ len,
                                                 const int64_t *__restrict__ ray_off, int64_t r_lo, int64_t r_hi,
                                                 int64_t seg_lo, int64_t nseg, const double2 *__restrict__ cs,
                                                 const double *__restrict__ Bv, double I_outer, int homog,
                                                 double *__restrict__ out, int chunk)
{
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    march_bundle<double, double2, 1, false, false, true>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, wg, cs, Bv,
                                                         I_outer, homog, out, chunk, nullptr);
}

// Full march (l I and l lambda) with the parabola choices of a bitmask.
__global__ void __launch_bounds__(256) k_march_bits(const uint32_t *__restrict__ vox, const float *__restrict__ len,
                                                    const int64_t *__restrict__ ray_off, int64_t r_lo, int64_t r_hi,
                                                    int64_t seg_lo, int64_t nseg, const float2 *__restrict__ cs,
                                                    const float *__restrict__ Bv, float I_outer,
                                                    void *__restrict__ outv, int chunk,
                                                    const uint32_t *__restrict__ pbits)
{
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    march_bundle<float, float2, 2, true, true>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, wg, cs, Bv, I_outer, 0,
                                               outv, chunk, pbits);
}

// FP64 J-only march (l I per segment) with the parabola choices of a bitmask:
// the FP64 residual of a batch member (its chi differs from the grid's).
__global__ void __launch_bounds__(256) k_march_bits64J(const uint32_t *__restrict__ vox, const double *__restrict__ len,
                                                       const int64_t *__restrict__ ray_off, int64_t r_lo, int64_t r_hi,
                                                       int64_t seg_lo, int64_t nseg, const double2 *__restrict__ cs,
                                                       const double *__restrict__ Bv, double I_outer, int homog,
                                                       double *__restrict__ out, int chunk,
                                                       const uint32_t *__restrict__ pbits)
{
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    march_bundle<double, double2, 1, false, true>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, wg, cs, Bv, I_outer,
                                                  homog, out, chunk, pbits);
}

// Persistent batched march (FP32, J only): the warps of a grid sized to the
// GPU take bundles of all work items (member x angle block, uneven grids
// mixed) from a device counter until none is left.
__global__ void __launch_bounds__(256) k_march_batch(const MarchItem *__restrict__ items,
                                                     const int64_t *__restrict__ bpfx, int n_items, int64_t total,
                                                     int chunk, int homog, unsigned long long *counter)
{
    const int lane = threadIdx.x & 31;
    for (int guard = 0; guard < (1 << 30); ++guard) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(counter, 1ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        if ((int64_t)b >= total) return;
        int lo = 0, hi = n_items;  // item: bpfx[item] <= b < bpfx[item+1]
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (bpfx[mid] <= (int64_t)b) lo = mid;
            else hi = mid;
        }
        const MarchItem &it = items[lo];
        march_bundle<float, float2, 2, false, true>(it.vox, it.len, it.ray_off, it.r_lo, it.r_hi, it.seg_lo, it.nseg,
                                                    (int64_t)b - bpfx[lo], it.cs, it.B, it.I_outer, homog, it.out,
                                                    chunk, it.pbits);
    }
}

// Per-member parabola choices as a bitmask (bit s of segment s), from that
// member's chi in FP64 (same rule as k_mark_parabola).
__global__ void k_para_bits(const uint32_t *vox, const double *len64, const double *chi, int64_t nseg, int parabolic,
                            uint32_t *bits)
{
    const int64_t nwords = (nseg + 31) / 32;
    for (int64_t wi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; wi < nwords; wi += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t s = wi * 32 + b;
            if (s >= nseg) break;
            bool para = false;
            if (parabolic && s + 1 < nseg) {
                const uint32_t w = vox[s], wn = vox[s + 1];
                if (!(wn & (RTK_RAYSTART | RTK_RESTART))) {
                    double x = chi[w & RTK_VOXMASK] * len64[s];
                    double p = chi[wn & RTK_VOXMASK] * len64[s + 1];
                    para = p >= 0.5 * x;
                }
            }
            if (para) word |= 1u << b;
        }
        bits[wi] = word;
    }
}

__global__ void k_mark_parabola(uint32_t *vox, const double *len64, const double *chi, int64_t nseg, int parabolic)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        uint32_t w = vox[s];
        bool para = false;
        if (parabolic && s + 1 < nseg) {
            uint32_t wn = vox[s + 1];
            if (!(wn & (RTK_RAYSTART | RTK_RESTART))) {
                double x = chi[w & RTK_VOXMASK] * len64[s];
                double p = chi[wn & RTK_VOXMASK] * len64[s + 1];
                para = p >= 0.5 * x;
            }
        }
        vox[s] = para ? (w | RTK_PARA) : (w & ~RTK_PARA);
    }
}

}  // namespace

cudaError_t mark_parabola(uint32_t *vox, const double *len64, const double *chi, int64_t nseg, int parabolic,
                          cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t blocks = (nseg + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_mark_parabola<<<(unsigned)blocks, 256, 0, st>>>(vox, len64, chi, nseg, parabolic);
    return cudaGetLastError();
}

template <typename T, typename P>
cudaError_t march_block(const uint32_t *vox, const T *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                        int64_t seg_lo, int64_t nseg, const P *chiS, const T *B, T I_outer, int homog,
                        int parabolic, P *out, int chunk, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t warps = (nseg + chunk - 1) / chunk;
    int64_t blocks = (warps + 7) / 8;
    (void)parabolic;  // the interpolant of every segment is in its RTK_PARA bit
    if constexpr (sizeof(T) == sizeof(float))
        k_march4<T, P, 2, true><<<(unsigned)blocks, 256, 0, st>>>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, chiS, B,
                                                                  I_outer, homog, out, chunk);
    else
        k_march4<T, P, 1, true><<<(unsigned)blocks, 256, 0, st>>>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, chiS, B,
                                                                  I_outer, homog, out, chunk);
    return cudaGetLastError();
}

template <typename T, typename P>
cudaError_t march_block_J(const uint32_t *vox, const T *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                          int64_t seg_lo, int64_t nseg, const P *chiS, const T *B, T I_outer, int homog, T *out,
                          int chunk, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t warps = (nseg + chunk - 1) / chunk;
    int64_t blocks = (warps + 7) / 8;
    if constexpr (sizeof(T) == sizeof(float))
        k_march4<T, P, 2, false><<<(unsigned)blocks, 256, 0, st>>>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, chiS, B,
                                                                   I_outer, homog, out, chunk);
    else
        k_march4<T, P, 1, false><<<(unsigned)blocks, 256, 0, st>>>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, chiS, B,
                                                                   I_outer, homog, out, chunk);
    return cudaGetLastError();
}

cudaError_t march_block_I(const uint32_t *vox, const double *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                          int64_t seg_lo, int64_t nseg, const double2 *chiS, const double *B, double I_outer, int homog,
                          double *out, int chunk, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t warps = (nseg + chunk - 1) / chunk;
    int64_t blocks = (warps + 7) / 8;
    k_march_I<<<(unsigned)blocks, 256, 0, st>>>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, chiS, B, I_outer, homog,
                                                out, chunk);
    return cudaGetLastError();
}

cudaError_t march_batch(const MarchItem *items, const int64_t *bpfx, int n_items, int64_t total, int chunk, int homog,
                        unsigned long long *counter, int grid_blocks, cudaStream_t st)
{
    if (total <= 0) return cudaSuccess;
    k_march_batch<<<grid_blocks, 256, 0, st>>>(items, bpfx, n_items, total, chunk, homog, counter);
    return cudaGetLastError();
}

cudaError_t march_block_bits(const uint32_t *vox, const float *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                             int64_t seg_lo, int64_t nseg, const float2 *chiS, const float *B, float I_outer,
                             float2 *out, int chunk, const uint32_t *pbits, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t warps = (nseg + chunk - 1) / chunk;
    int64_t blocks = (warps + 7) / 8;
    k_march_bits<<<(unsigned)blocks, 256, 0, st>>>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, chiS, B, I_outer, out,
                                                   chunk, pbits);
    return cudaGetLastError();
}

cudaError_t march_block_bits64J(const uint32_t *vox, const double *len, const int64_t *ray_off, int64_t r_lo,
                                int64_t r_hi, int64_t seg_lo, int64_t nseg, const double2 *chiS, const double *B,
                                double I_outer, int homog, double *out, int chunk, const uint32_t *pbits,
                                cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t warps = (nseg + chunk - 1) / chunk;
    int64_t blocks = (warps + 7) / 8;
    k_march_bits64J<<<(unsigned)blocks, 256, 0, st>>>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, chiS, B, I_outer,
                                                      homog, out, chunk, pbits);
    return cudaGetLastError();
}

cudaError_t para_bits(const uint32_t *vox, const double *len64, const double *chi, int64_t nseg, int parabolic,
                      uint32_t *bits, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t words = (nseg + 31) / 32;
    int64_t blocks = (words + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_para_bits<<<(unsigned)blocks, 256, 0, st>>>(vox, len64, chi, nseg, parabolic, bits);
    return cudaGetLastError();
}

cudaError_t march_block_preload()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_march4<float, float2, 2, true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_march4<double, double2, 1, true>);
    return e;
}

template cudaError_t march_block_J<double, double2>(const uint32_t *, const double *, const int64_t *, int64_t, int64_t,
                                                    int64_t, int64_t, const double2 *, const double *, double, int,
                                                    double *, int, cudaStream_t);
template cudaError_t march_block_J<float, float2>(const uint32_t *, const float *, const int64_t *, int64_t, int64_t,
                                                  int64_t, int64_t, const float2 *, const float *, float, int, float *,
                                                  int, cudaStream_t);
template cudaError_t march_block<double, double2>(const uint32_t *, const double *, const int64_t *, int64_t, int64_t,
                                                  int64_t, int64_t, const double2 *, const double *, double, int, int,
                                                  double2 *, int, cudaStream_t);
template cudaError_t march_block<float, float2>(const uint32_t *, const float *, const int64_t *, int64_t, int64_t,
                                                int64_t, int64_t, const float2 *, const float *, float, int, int,
                                                float2 *, int, cudaStream_t);

}  // namespace rtk
