// fs_sw.cu -- J-only formal solution of the ALI iteration with streamed
// segment weights (the hot loop of the mixed-precision path, FP32; the same
// march in FP64 for the FP64 path).
//
// The weights of a segment in the recurrence I_k = I_{k-1} E_k + alpha_k
// S_{k-1} + beta_k S_k + gamma_k S_{k+1} (scheme R6 of Papers I-II, Sect. 2)
// depend on chi and the path length only, so for the duration of an ALI solve
// they are loop invariants: k_coef_stream evaluates them once per chi in FP64
// and stores (E, alpha, beta, gamma) as FP32, alpha folded into beta at the
// start of a run (S_0 := S_1) and gamma = 0 where the linear weights apply.
// k_seg_weight stores c = w_Omega l / L_{Omega v} per segment (geometry only),
// so the march writes c_s I_s and J_v (Sect. 3.2.1) is a plain sum of those
// values over v's ownership list, in list order.
//
// The march of angle block b (warps over bundles of whole characteristics,
// bounds from a precomputed table) runs while J of block b - 1 is gathered
// on a second stream from the other half of a double buffer, so the
// latency-bound gather overlaps the march.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "coef.cuh"
#include "rt_internal.h"

namespace rtk {
namespace {

constexpr int CHUNK = RTK_JCHUNK;  // long-list chunk of the J tables (one warp each)

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
    // butterfly over the warp with an error-free combination of the partial sums
    __device__ __forceinline__ void warp_reduce()
    {
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
            const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
            const float t = s + s2;
            const float bb = t - s;
            const float err = (s - (t - bb)) + (s2 - bb);
            c = (c + c2) - err;
            s = t;
        }
    }
};

// Plain FP64 accumulation for the FP64 gathers (same interface as Kahan).
struct Sum64 {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ void warp_reduce()
    {
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
};
template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = Kahan; };
template <> struct AccOf<double> { using type = Sum64; };
// 16-byte vectors of a row and their entries added in order
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    template <typename A> __device__ __forceinline__ static void add_to(A &acc, const float4 &x)
    {
        acc.add(x.x);
        acc.add(x.y);
        acc.add(x.z);
        acc.add(x.w);
    }
};
template <> struct Vec16<double> {
    using type = double2;
    template <typename A> __device__ __forceinline__ static void add_to(A &acc, const double2 &x)
    {
        acc.add(x.x);
        acc.add(x.y);
    }
};
template <typename T> __device__ __forceinline__ const T *gbuf(const SwGather &t);
template <> __device__ __forceinline__ const float *gbuf<float>(const SwGather &t) { return t.buf; }
template <> __device__ __forceinline__ const double *gbuf<double>(const SwGather &t) { return t.buf64; }

__device__ __forceinline__ int64_t lb64(const int64_t *a, int64_t lo, int64_t hi, int64_t key)
{
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Bundle bw of a block: the whole characteristics whose first segment lies in
// [bw * chunk, (bw + 1) * chunk), as segment indices relative to the block.
__global__ void k_bundles(const int64_t *ray_off, int64_t r_lo, int64_t r_hi, int64_t seg_lo, int64_t nseg, int chunk,
                          int64_t nb, int2 *bnd)
{
    for (int64_t bw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; bw < nb; bw += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c_lo = bw * chunk;
        const int64_t c_hi = (c_lo + chunk < nseg) ? c_lo + chunk : nseg;
        const int64_t ra = lb64(ray_off, r_lo, r_hi, seg_lo + c_lo);
        const int64_t rb = lb64(ray_off, r_lo, r_hi, seg_lo + c_hi);
        bnd[bw] = make_int2((int)(ray_off[ra] - seg_lo), (int)(ray_off[rb] - seg_lo));
    }
}

// One warp marches bundle wg: K consecutive segments per lane, the lane maps
// I -> A I + b composed by an inclusive shuffle scan over the warp; the next
// tile's words and weights are fetched before the current one is processed.
__device__ __forceinline__ float4 ldw(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ Wd4 ldw(const Wd4 *p)
{
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    return Wd4{a.x, a.y, b.x, b.y};
}

// SLA: the S lookups of tile t + 1 are issued while tile t is marched (its
// words are loaded two tiles ahead), so no tile waits for its own lookups.
// FOLD: the weights carry the gather weight (k_coef_stream_fold); the c stream
// is not read and the recurrence value is the output itself.
template <typename M, int K, bool SLA, bool FOLD = false>
__device__ __forceinline__ void march_sw(const M &m, int64_t wg)
{
    using T = typename M::T;
    using W = typename M::W;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (wg >= m.nbundles) return;
    const int2 be = m.bnd[wg];
    const int s_begin = be.x, s_end = be.y;
    if (s_begin >= s_end) return;
    const uint32_t *vx = m.vox + m.seg_lo;
    const W *cf = m.cw + m.seg_lo;
    const T *gw = m.cg + m.seg_lo;
    T *o = m.out;
    T Icarry = 0, Sprev = 0;
    const int32_t *ps = m.pos ? m.pos + m.seg_lo : nullptr;
    uint32_t w[K];
    W c[K];
    T g[K];
    int p[K];  // output positions (list order) when scattering
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int s = s_begin + K * lane + j;
        const bool ok = s < s_end;
        w[j] = ok ? __ldcs(vx + s) : 0u;
        c[j] = ok ? ldw(cf + s) : W{1, 0, 0, 0};
        g[j] = FOLD ? T(1) : (ok ? __ldcs(gw + s) : T(0));
        p[j] = (ps && ok) ? __ldcs(ps + s) : 0;
    }
    uint32_t wA[K];  // SLA: words of the next tile
    T Sc[K];         // SLA: S of this tile's segments
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if constexpr (SLA) {
            const int s = s_begin + 32 * K + K * lane + j;
            wA[j] = s < s_end ? __ldcs(vx + s) : 0u;
            Sc[j] = (s_begin + K * lane + j < s_end) ? m.S[w[j] & RTK_VOXMASK] : T(0);
        } else {
            wA[j] = 0u;
            Sc[j] = T(0);
        }
    }
    // The last segment of a tile may use S of the next tile's first segment
    // (gamma); its value is completed and stored at the start of the next tile,
    // so no tile waits for the loads of the one after it.
    T pend_I = 0, pend_gam = 0, pend_g = 0;
    int pend_o = 0;
    bool pend = false;  // warp-uniform
    for (int base = s_begin; base < s_end; base += 32 * K) {
        const int s0 = base + K * lane;
        uint32_t wN[K];
        W cN[K];
        T gN[K];
        int pN[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {  // the next tile's streams, in flight while this one is marched
            const int s = base + 32 * K + K * lane + j;
            const bool ok = s < s_end;
            wN[j] = SLA ? wA[j] : (ok ? __ldcs(vx + s) : 0u);
            cN[j] = ok ? ldw(cf + s) : W{1, 0, 0, 0};
            gN[j] = FOLD ? T(1) : (ok ? __ldcs(gw + s) : T(0));
            pN[j] = (ps && ok) ? __ldcs(ps + s) : 0;
        }
        T S[K], SN[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if constexpr (SLA) {
                S[j] = Sc[j];
                const int s = base + 64 * K + K * lane + j;  // words two tiles ahead
                wA[j] = s < s_end ? __ldcs(vx + s) : 0u;
                SN[j] = (base + 32 * K + K * lane + j < s_end) ? m.S[wN[j] & RTK_VOXMASK] : T(0);
            } else {
                S[j] = (s0 + j < s_end) ? m.S[w[j] & RTK_VOXMASK] : T(0);
                SN[j] = T(0);
            }
        }
        if (pend) {  // complete the previous tile's last segment
            const T Sf = __shfl_sync(FULL, S[0], 0);
            if (lane == 31) {
                pend_I = fma(pend_gam * pend_g, Sf, pend_I);
                __stcg(o + pend_o, pend_I);
            }
            Icarry = fma(pend_gam, Sf, Icarry);
        }
        T Snx = __shfl_down_sync(FULL, S[0], 1);  // S after this lane's last segment
        if (lane == 31) Snx = 0;                    // next tile: added when it is loaded
        T Sp = __shfl_up_sync(FULL, S[K - 1], 1); // S before this lane's first segment
        if (lane == 0) Sp = Sprev;
        T A[K], b[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const T Sm = (j == 0) ? Sp : S[j - 1];
            const T Sn = (j + 1 < K) ? S[j + 1] : Snx;
            const T src = fma(c[j].y, Sm, fma(c[j].z, S[j], c[j].w * Sn));
            A[j] = c[j].x;
            b[j] = src;
            if (w[j] & RTK_RAYSTART) {
                const T Iin = m.homog ? T(0) : ((w[j] & RTK_CORE) ? m.B[w[j] & RTK_VOXMASK] : m.I_outer);
                b[j] = fma(c[j].x, Iin, src);
                A[j] = 0;
            }
            if (s0 + j >= s_end) {
                A[j] = 1;
                b[j] = 0;
            }
        }
        T LA = A[0], LB = b[0];
#pragma unroll
        for (int j = 1; j < K; ++j) {
            LB = fma(A[j], LB, b[j]);
            LA = A[j] * LA;
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T Ao = __shfl_up_sync(FULL, LA, off);
            const T bo = __shfl_up_sync(FULL, LB, off);
            if (lane >= off) {
                LB = fma(LA, bo, LB);
                LA = LA * Ao;
            }
        }
        T PA = __shfl_up_sync(FULL, LA, 1);
        T PB = __shfl_up_sync(FULL, LB, 1);
        if (lane == 0) {
            PA = 1;
            PB = 0;
        }
        pend = base + 32 * K < s_end;
        T I = fma(PA, Icarry, PB);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            I = fma(A[j], I, b[j]);
            const int oi = ps ? p[j] : s0 + j;
            if (j == K - 1 && lane == 31 && pend) {
                pend_I = g[j] * I;
                pend_gam = c[j].w;
                pend_g = g[j];
                pend_o = oi;
            } else if (s0 + j < s_end) {
                __stcg(o + oi, g[j] * I);
            }
        }
        Icarry = __shfl_sync(FULL, I, 31);
        pend_gam = __shfl_sync(FULL, pend_gam, 31);
        Sprev = __shfl_sync(FULL, S[K - 1], 31);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            w[j] = wN[j];
            c[j] = cN[j];
            g[j] = gN[j];
            p[j] = pN[j];
            Sc[j] = SN[j];
        }
    }
}

// ---- staged variant: bulk copies (cp.async.bulk) into a per-warp ring ----
//
// Each warp keeps NS tiles of its bundle in flight: lane 0 issues, per tile,
// one bulk copy of the (E, alpha, beta, gamma) stream and one of each 4-byte
// stream (words, c, list positions) into a shared-memory stage and arms that
// stage's mbarrier with the byte count; the lanes wait on the barrier, copy
// the tile into registers and lane 0 refills the stage with tile t + NS
// before the tile is processed.  A 4-byte stream's copy starts at the
// 16-byte boundary at or below the tile (up to 3 extra words, the arrays
// carry 4 words of padding) and the lanes index past the offset.  Every wait
// is bounded: on timeout the warp raises *err, waits (bounded) for the
// copies it issued and returns.

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false after MBAR_SPINS unsuccessful polls.
constexpr int MBAR_SPINS = 1 << 20;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (int it = 0; it < MBAR_SPINS; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int K>
struct SwStage {
    float4 cw[32 * K];
    uint32_t w[32 * K + 4];
    float cg[32 * K + 4];
    int32_t pos[32 * K + 4];
};

template <int K, int NS>
constexpr size_t tma_smem_bytes()
{
    return 8 * (NS * sizeof(SwStage<K>) + NS * sizeof(uint64_t));
}

template <int K, int NS, bool BULK>
__device__ __forceinline__ void march_tma(const SwMarch &m, int64_t wg, SwStage<K> *stg, uint64_t *bar)
{
    constexpr int T = 32 * K;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (wg >= m.nbundles) return;
    const int2 be = m.bnd[wg];
    const int s_begin = be.x, s_end = be.y;
    if (s_begin >= s_end) return;
    const int ntile = (s_end - s_begin + T - 1) / T;
    const bool scatter = m.pos != nullptr;
    uint64_t policy = 0;
    if (BULK && lane == 0) {
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
        for (int i = 0; i < NS; ++i) mbar_init(bar + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // copy tile t into stage t % NS: bulk copies issued by lane 0 (BULK), or
    // 16-byte cp.async copies spread over the lanes (one commit group per tile)
    auto issue = [&](int t) {
        const int i = t % NS;
        const int64_t gs = m.seg_lo + s_begin + (int64_t)T * t;  // first segment of the tile (global index)
        const int n = min(T, s_end - (s_begin + T * t));
        const int64_t ga = gs & ~(int64_t)3;
        const int cnt = (int)(((gs - ga) + n + 3) & ~3);  // words of the 16-byte aligned window
        if (BULK) {
            const uint32_t b4 = 4u * (uint32_t)cnt;
            const uint32_t b16 = 16u * (uint32_t)n;
            mbar_expect_tx(bar + i, b16 + (scatter ? 3u : 2u) * b4);
            bulk_g2s(stg[i].cw, m.cw + gs, b16, bar + i, policy);
            bulk_g2s(stg[i].w, m.vox + ga, b4, bar + i, policy);
            bulk_g2s(stg[i].cg, m.cg + ga, b4, bar + i, policy);
            if (scatter) bulk_g2s(stg[i].pos, m.pos + ga, b4, bar + i, policy);
        } else {
            for (int q = lane; q < n; q += 32) cp_async16(stg[i].cw + q, m.cw + gs + q);
            for (int q = lane; q < cnt / 4; q += 32) {
                cp_async16(stg[i].w + 4 * q, m.vox + ga + 4 * q);
                cp_async16(stg[i].cg + 4 * q, m.cg + ga + 4 * q);
                if (scatter) cp_async16(stg[i].pos + 4 * q, m.pos + ga + 4 * q);
            }
        }
    };
    if (BULK) {
        if (lane == 0)
            for (int t = 0; t < NS && t < ntile; ++t) issue(t);
    } else {
        for (int t = 0; t < NS - 1; ++t) {
            if (t < ntile) issue(t);
            cp_async_commit();
        }
    }
    float Icarry = 0.f, Sprev = 0.f;
    float *o = m.out;
    float pend_I = 0.f, pend_gam = 0.f, pend_g = 0.f;  // last segment of the previous tile (see march_sw)
    int pend_o = 0;
    bool pend = false;
    for (int t = 0; t < ntile; ++t) {
        const int i = t % NS;
        if (BULK) {
            if (!mbar_wait(bar + i, (uint32_t)((t / NS) & 1))) {
                if (lane == 0) {
                    atomicExch(m.err, 1);
                    for (int u = t; u < ntile && u < t + NS; ++u)
                        (void)mbar_wait(bar + (u % NS), (uint32_t)((u / NS) & 1));
                }
                __syncwarp();
                return;
            }
        } else {
            cp_async_wait<NS - 2>();  // this lane's copies of tile t have landed
            __syncwarp();             // ... and every lane's
            if (t + NS - 1 < ntile) issue(t + NS - 1);  // into the stage read in the previous iteration
            cp_async_commit();
        }
        const int base = s_begin + T * t;
        const int off = (int)((m.seg_lo + base) & 3);
        const int s0 = base + K * lane;
        uint32_t w[K];
        float4 c[K];
        float g[K];
        int pN[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int li = K * lane + j;
            const bool ok = s0 + j < s_end;
            w[j] = ok ? stg[i].w[off + li] : 0u;
            c[j] = ok ? stg[i].cw[li] : make_float4(1.f, 0.f, 0.f, 0.f);
            g[j] = ok ? stg[i].cg[off + li] : 0.f;
            pN[j] = (ok && scatter) ? stg[i].pos[off + li] : 0;
        }
        __syncwarp();
        if (BULK && lane == 0 && t + NS < ntile) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(t + NS);
        }
        float S[K];
#pragma unroll
        for (int j = 0; j < K; ++j) S[j] = (s0 + j < s_end) ? m.S[w[j] & RTK_VOXMASK] : 0.f;
        if (pend) {
            const float Sf = __shfl_sync(FULL, S[0], 0);
            if (lane == 31) {
                pend_I = fmaf(pend_gam * pend_g, Sf, pend_I);
                __stcg(o + pend_o, pend_I);
            }
            Icarry = fmaf(pend_gam, Sf, Icarry);
        }
        float Snx = __shfl_down_sync(FULL, S[0], 1);
        if (lane == 31) Snx = 0.f;
        float Sp = __shfl_up_sync(FULL, S[K - 1], 1);
        if (lane == 0) Sp = Sprev;
        float A[K], b[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float Sm = (j == 0) ? Sp : S[j - 1];
            const float Sn = (j + 1 < K) ? S[j + 1] : Snx;
            const float src = fmaf(c[j].y, Sm, fmaf(c[j].z, S[j], c[j].w * Sn));
            A[j] = c[j].x;
            b[j] = src;
            if (w[j] & RTK_RAYSTART) {
                const float Iin = m.homog ? 0.f : ((w[j] & RTK_CORE) ? m.B[w[j] & RTK_VOXMASK] : m.I_outer);
                b[j] = fmaf(c[j].x, Iin, src);
                A[j] = 0.f;
            }
            if (s0 + j >= s_end) {
                A[j] = 1.f;
                b[j] = 0.f;
            }
        }
        float LA = A[0], LB = b[0];
#pragma unroll
        for (int j = 1; j < K; ++j) {
            LB = fmaf(A[j], LB, b[j]);
            LA = A[j] * LA;
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float Ao = __shfl_up_sync(FULL, LA, d);
            const float bo = __shfl_up_sync(FULL, LB, d);
            if (lane >= d) {
                LB = fmaf(LA, bo, LB);
                LA = LA * Ao;
            }
        }
        float PA = __shfl_up_sync(FULL, LA, 1);
        float PB = __shfl_up_sync(FULL, LB, 1);
        if (lane == 0) {
            PA = 1.f;
            PB = 0.f;
        }
        pend = base + T < s_end;
        float I = fmaf(PA, Icarry, PB);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            I = fmaf(A[j], I, b[j]);
            const int oi = scatter ? pN[j] : s0 + j;
            if (j == K - 1 && lane == 31 && pend) {
                pend_I = g[j] * I;
                pend_gam = c[j].w;
                pend_g = g[j];
                pend_o = oi;
            } else if (s0 + j < s_end) {
                __stcg(o + oi, g[j] * I);
            }
        }
        Icarry = __shfl_sync(FULL, I, 31);
        pend_gam = __shfl_sync(FULL, pend_gam, 31);
        Sprev = __shfl_sync(FULL, S[K - 1], 31);
    }
    if (!BULK) cp_async_wait<0>();
}

template <int K, int NS, bool BULK>
__global__ void __launch_bounds__(256, 5) k_march_tma(SwMarch m)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    SwStage<K> *stg = reinterpret_cast<SwStage<K> *>(smem) + warp * NS;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 8 * NS * sizeof(SwStage<K>)) + warp * NS;
    march_tma<K, NS, BULK>(m, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, stg, bar);
}

// J gather of one block from the values c_s I_s: CTAs [0, nbs) take 256 short
// lists each (thread per voxel over the sliced-ELL entries, 8 loads in
// flight); the other warps take one RTK_JCHUNK-entry chunk of a long list each
// (32 entries per lane, 8 in flight), and the warp that completes a voxel's
// last chunk adds the chunk sums in chunk order.
template <typename T>
__global__ void __launch_bounds__(256) k_gather_sw(SwGather t)
{
    using Acc = typename AccOf<T>::type;
    const T *buf = gbuf<T>(t);
    const int64_t cta = blockIdx.x;
    if (cta < t.nbs) {
        const int64_t i = cta * 256 + threadIdx.x;
        if (i >= t.nshort) return;
        const int v = t.jorder[i];
        const int L = t.off[v + 1] - t.off[v];
        const int32_t *lst = t.jsell + t.jgbase[i >> 5] + (i & 31);
        Acc acc;
        for (int k = 0; k < L; k += 8) {
            int ss[8];
            T val[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) ss[j] = (k + j < L) ? __ldcs(lst + 32 * (k + j)) : -1;
#pragma unroll
            for (int j = 0; j < 8; ++j) val[j] = (ss[j] >= 0) ? __ldcg(buf + ss[j]) : T(0);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (ss[j] >= 0) acc.add(val[j]);
        }
        const double r = acc.value();
        t.J[v] = t.first ? r : t.J[v] + r;
        return;
    }
    const int64_t c = ((cta - t.nbs) * 256 + threadIdx.x) >> 5;
    if (c >= t.nchunks) return;
    const int lane = threadIdx.x & 31;
    const int v = t.crow[c];
    const int e0 = t.cbeg[c];
    const int e1 = min(e0 + CHUNK, t.off[v + 1]);
    Acc acc;
    for (int k = e0 + lane; k < e1; k += 32 * 8) {
        int ss[8];
        T val[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) ss[j] = (k + 32 * j < e1) ? __ldcs(t.perm + k + 32 * j) : -1;
#pragma unroll
        for (int j = 0; j < 8; ++j) val[j] = (ss[j] >= 0) ? __ldcg(buf + ss[j]) : T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (ss[j] >= 0) acc.add(val[j]);
    }
    acc.warp_reduce();
    if (lane == 0) {
        const int lr = t.clr[c];
        __stcg(t.part + c, acc.value());
        __threadfence();
        const int c0 = t.lfirst[lr], c1 = (lr + 1 < t.nlong) ? t.lfirst[lr + 1] : (int)t.nchunks;
        if (atomicAdd(t.cnt + lr, 1) == c1 - c0 - 1) {
            __threadfence();
            double sum = 0.0;
            for (int cc = c0; cc < c1; ++cc) sum += __ldcg(t.part + cc);
            t.J[v] = t.first ? sum : t.J[v] + sum;
            t.cnt[lr] = 0;
        }
    }
}

// J gather of one block from values already in voxel order (the march
// scattered c_s I_s to the list positions): short lists thread per voxel in
// voxel order (adjacent threads read adjacent rows), long lists one warp per
// chunk; same summation order as k_gather_sw.
template <typename T>
__global__ void __launch_bounds__(256) k_gather_rows_sw(SwGather t, int nvox, int64_t nvb)
{
    using Acc = typename AccOf<T>::type;
    const T *buf = gbuf<T>(t);
    const int64_t cta = blockIdx.x;
    if (cta < nvb) {
        const int v = (int)(cta * 256 + threadIdx.x);
        if (v >= nvox) return;
        const int a = t.off[v], L = t.off[v + 1] - a;
        if (L > RTK_JSHORT) return;  // long list: chunk warps
        // A row is one thread's: it is read through the read-only L1 path in
        // 16-byte vectors from its first 16-byte boundary on (scalars before
        // it and after the last whole vector); entries are added in row order.
        Acc acc;
        const T *row = buf + a;
        constexpr int NV = 16 / sizeof(T);
        int head = (int)(((16u - ((uint32_t)(uintptr_t)row & 15u)) & 15u) / sizeof(T));
        if (head > L) head = L;
        for (int k = 0; k < head; ++k) acc.add(__ldg(row + k));
        using V = typename Vec16<T>::type;
        const V *rv = reinterpret_cast<const V *>(row + head);
        const int nvec = (L - head) / NV;
        for (int q = 0; q < nvec; q += 4) {
            V x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q + u < nvec) x[u] = __ldg(rv + q + u);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q + u < nvec) Vec16<T>::add_to(acc, x[u]);
        }
        for (int k = head + nvec * NV; k < L; ++k) acc.add(__ldg(row + k));
        const double r = acc.value();
        t.J[v] = t.first ? r : t.J[v] + r;
        return;
    }
    const int64_t c = ((cta - nvb) * 256 + threadIdx.x) >> 5;
    if (c >= t.nchunks) return;
    const int lane = threadIdx.x & 31;
    const int v = t.crow[c];
    const int e0 = t.cbeg[c];
    const int e1 = min(e0 + CHUNK, t.off[v + 1]);
    Acc acc;
    for (int k = e0 + lane; k < e1; k += 32 * 8) {
        T val[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) val[j] = (k + 32 * j < e1) ? __ldcg(buf + k + 32 * j) : T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (k + 32 * j < e1) acc.add(val[j]);
    }
    acc.warp_reduce();
    if (lane == 0) {
        const int lr = t.clr[c];
        __stcg(t.part + c, acc.value());
        __threadfence();
        const int c0 = t.lfirst[lr], c1 = (lr + 1 < t.nlong) ? t.lfirst[lr + 1] : (int)t.nchunks;
        if (atomicAdd(t.cnt + lr, 1) == c1 - c0 - 1) {
            __threadfence();
            double sum = 0.0;
            for (int cc = c0; cc < c1; ++cc) sum += __ldcg(t.part + cc);
            t.J[v] = t.first ? sum : t.J[v] + sum;
            t.cnt[lr] = 0;
        }
    }
}

// Position of every segment of a block in its ownership-list order.
__global__ void k_inv_perm(const int32_t *perm, int64_t n, int32_t *pos)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        pos[perm[e]] = (int32_t)e;
}

template <typename M, int K, bool SLA, bool FOLD = false>
__global__ void __launch_bounds__(256) k_march_sw(M m)
{
    march_sw<M, K, SLA, FOLD>(m, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
}

// FP64 weights of every segment for the current chi, rounded to FP32.
__global__ void k_coef_stream(const uint32_t *__restrict__ vox, const double *__restrict__ len64,
                              const double *__restrict__ chi, int64_t nseg, float4 *__restrict__ cw)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = vox[s];
        const bool para = (w & RTK_PARA) != 0u;  // set only when segment s + 1 continues the run
        const double x = chi[w & RTK_VOXMASK] * len64[s];
        const double p = para ? chi[vox[s + 1] & RTK_VOXMASK] * len64[s + 1] : 0.0;
        double E, al, be, ga;
        Coef64::eval(x, p, para, E, al, be, ga);
        if (w & (RTK_RAYSTART | RTK_RESTART)) {  // S_0 := S_1 at the start of a run
            be += al;
            al = 0.0;
        }
        cw[s] = make_float4((float)E, (float)al, (float)be, (float)ga);
    }
}

// The weights with the gather weight folded in: the march then carries
// c_s I_s, whose recurrence has the weights (E c_s / c_{s-1}, c_s alpha,
// c_s beta, c_s gamma); at a characteristic start A = 0 and the E slot holds
// c_s E (the incoming intensity's factor).  The optical depths and c_s =
// w_Omega l_s / L_{Omega v_s} are formed in FP64 (as k_seg_weight forms c);
// (E, alpha, beta, gamma) are evaluated in FP32 by the same Coef32 as the
// marches that evaluate them per segment (on the FP32 pipe: GB300's FP64 pipe
// is narrow), and the products with c and the ratio c_s / c_{s-1} in FP32.
__global__ void k_coef_stream_fold(const uint32_t *__restrict__ vox, const double *__restrict__ len64,
                                   const double *__restrict__ chi, const int64_t *__restrict__ ang_seg_off, int n_ang,
                                   const double *__restrict__ wt, const double *__restrict__ invL, int nvox,
                                   int64_t nseg, float4 *__restrict__ cw)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_ang;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ang_seg_off[mid] <= s) lo = mid;
            else hi = mid;
        }
        const uint32_t w = vox[s];
        const bool para = (w & RTK_PARA) != 0u;
        const float x = (float)(chi[w & RTK_VOXMASK] * len64[s]);
        const float p = para ? (float)(chi[vox[s + 1] & RTK_VOXMASK] * len64[s + 1]) : 0.0f;
        float E, al, be, ga;
        Coef32::eval(x, p, para, E, al, be, ga);
        if (w & (RTK_RAYSTART | RTK_RESTART)) {
            be += al;
            al = 0.0f;
        }
        const double *iL = invL + (int64_t)lo * nvox;
        const float c = (float)(wt[lo] * len64[s] * iL[w & RTK_VOXMASK]);
        float A = c * E;
        if (!(w & RTK_RAYSTART)) A = __fdividef(A, (float)(wt[lo] * len64[s - 1] * iL[vox[s - 1] & RTK_VOXMASK]));
        cw[s] = make_float4(A, c * al, c * be, c * ga);
    }
}

// FP64 weights of every segment for the current chi (FP64 streamed march).
__global__ void k_coef_stream64(const uint32_t *__restrict__ vox, const double *__restrict__ len64,
                                const double *__restrict__ chi, int64_t nseg, Wd4 *__restrict__ cw)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = vox[s];
        const bool para = (w & RTK_PARA) != 0u;
        const double x = chi[w & RTK_VOXMASK] * len64[s];
        const double p = para ? chi[vox[s + 1] & RTK_VOXMASK] * len64[s + 1] : 0.0;
        double E, al, be, ga;
        Coef64::eval(x, p, para, E, al, be, ga);
        if (w & (RTK_RAYSTART | RTK_RESTART)) {
            be += al;
            al = 0.0;
        }
        cw[s] = Wd4{E, al, be, ga};
    }
}

__global__ void k_seg_weight64(const uint32_t *__restrict__ vox, const double *__restrict__ len64,
                               const int64_t *__restrict__ ang_seg_off, int n_ang, const double *__restrict__ wt,
                               const double *__restrict__ invL, int nvox, int64_t nseg, double *__restrict__ cg)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_ang;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ang_seg_off[mid] <= s) lo = mid;
            else hi = mid;
        }
        cg[s] = wt[lo] * len64[s] * invL[(int64_t)lo * nvox + (vox[s] & RTK_VOXMASK)];
    }
}

// Gather weight times path length of every segment: w_Omega l_s / L_{Omega v_s}.
__global__ void k_seg_weight(const uint32_t *__restrict__ vox, const double *__restrict__ len64,
                             const int64_t *__restrict__ ang_seg_off, int n_ang, const double *__restrict__ wt,
                             const double *__restrict__ invL, int nvox, int64_t nseg, float *__restrict__ cg)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_ang;  // angle q: ang_seg_off[q] <= s < ang_seg_off[q + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ang_seg_off[mid] <= s) lo = mid;
            else hi = mid;
        }
        const int v = vox[s] & RTK_VOXMASK;
        cg[s] = (float)(wt[lo] * len64[s] * invL[(int64_t)lo * nvox + v]);
    }
}


// ---- S lookups of the FP32 march in a blocked voxel order ----
//
// The march looks S up once per segment; consecutive segments of a
// characteristic are neighbouring voxels in any of the three index
// directions.  In the grid's order (k fastest) a 128-byte line of FP32 S holds
// 32 voxels of one (i, j) row, so most lookups touch a new line; in the blocked
// order a line holds a 4 x 2 x 4 block of (i, j, k), and a characteristic
// crossing it finds several of its voxels there.  vblk maps a voxel to its
// blocked slot; the march reads words whose voxel field holds that slot.
__global__ void k_make_voxb(const uint32_t *__restrict__ vox, int64_t nseg, const int32_t *__restrict__ vblk,
                            uint32_t *__restrict__ voxb)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = vox[s];
        voxb[s] = (w & (RTK_RAYSTART | RTK_CORE | RTK_RESTART)) | (uint32_t)vblk[w & RTK_VOXMASK];
    }
}

__global__ void k_blk_scatter(int nvox, const int32_t *__restrict__ vblk, const float *__restrict__ S,
                              const float *__restrict__ B, float *__restrict__ Sb, float *__restrict__ Bb)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nvox) {
        const int q = vblk[v];
        Sb[q] = S[v];
        Bb[q] = B[v];
    }
}

unsigned grid_cap(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t make_voxb(const uint32_t *vox, int64_t nseg, const int32_t *vblk, uint32_t *voxb, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    k_make_voxb<<<grid_cap(nseg), 256, 0, st>>>(vox, nseg, vblk, voxb);
    return cudaGetLastError();
}

cudaError_t blk_scatter(int nvox, const int32_t *vblk, const float *S, const float *B, float *Sb, float *Bb,
                        cudaStream_t st)
{
    k_blk_scatter<<<(nvox + 255) / 256, 256, 0, st>>>(nvox, vblk, S, B, Sb, Bb);
    return cudaGetLastError();
}

cudaError_t sw_bundles(const int64_t *ray_off, int64_t r_lo, int64_t r_hi, int64_t seg_lo, int64_t nseg, int chunk,
                       int2 *bnd, cudaStream_t st)
{
    const int64_t nb = (nseg + chunk - 1) / chunk;
    if (nb <= 0) return cudaSuccess;
    k_bundles<<<grid_cap(nb), 256, 0, st>>>(ray_off, r_lo, r_hi, seg_lo, nseg, chunk, nb, bnd);
    return cudaGetLastError();
}

template <int K, int NS, bool BULK>
cudaError_t launch_ring(const SwMarch &m, int64_t grid, cudaStream_t st)
{
    constexpr size_t bytes = tma_smem_bytes<K, NS>();
    // the attribute belongs to the kernel on one device: set once per device
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
    if (!bit || !(done.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_march_tma<K, NS, BULK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        done.fetch_or(bit, std::memory_order_acq_rel);
    }
    k_march_tma<K, NS, BULK><<<(unsigned)grid, 256, bytes, st>>>(m);
    return cudaGetLastError();
}

template <bool BULK>
cudaError_t launch_ring_k(const SwMarch &m, int coarsen, int64_t grid, cudaStream_t st)
{
    if (m.stages == 4) return coarsen == 1 ? launch_ring<1, 4, BULK>(m, grid, st) : launch_ring<2, 4, BULK>(m, grid, st);
    if (m.stages == 3) return coarsen == 1 ? launch_ring<1, 3, BULK>(m, grid, st) : launch_ring<2, 3, BULK>(m, grid, st);
    return coarsen == 1 ? launch_ring<1, 2, BULK>(m, grid, st) : launch_ring<2, 2, BULK>(m, grid, st);
}

cudaError_t march_sw_launch(const SwMarch &m, int coarsen, cudaStream_t st)
{
    const int64_t grid = (m.nbundles + 7) / 8;
    if (grid <= 0) return cudaSuccess;
    if (m.stages >= 2) return m.bulk ? launch_ring_k<true>(m, coarsen, grid, st) : launch_ring_k<false>(m, coarsen, grid, st);
    if (m.fold) {  // register prefetch with lookahead only
        if (coarsen == 1) k_march_sw<SwMarch, 1, true, true><<<(unsigned)grid, 256, 0, st>>>(m);
        else k_march_sw<SwMarch, 2, true, true><<<(unsigned)grid, 256, 0, st>>>(m);
        return cudaGetLastError();
    }
    if (m.lookahead) {
        if (coarsen == 4) k_march_sw<SwMarch, 4, true><<<(unsigned)grid, 256, 0, st>>>(m);
        else if (coarsen == 1) k_march_sw<SwMarch, 1, true><<<(unsigned)grid, 256, 0, st>>>(m);
        else k_march_sw<SwMarch, 2, true><<<(unsigned)grid, 256, 0, st>>>(m);
    } else {
        if (coarsen == 4) k_march_sw<SwMarch, 4, false><<<(unsigned)grid, 256, 0, st>>>(m);
        else if (coarsen == 1) k_march_sw<SwMarch, 1, false><<<(unsigned)grid, 256, 0, st>>>(m);
        else k_march_sw<SwMarch, 2, false><<<(unsigned)grid, 256, 0, st>>>(m);
    }
    return cudaGetLastError();
}

cudaError_t gather_rows_sw_launch(const SwGather &t, int nvox, cudaStream_t st)
{
    const int64_t nvb = (nvox + 255) / 256;
    const int64_t grid = nvb + (t.nchunks * 32 + 255) / 256;
    if (grid <= 0) return cudaSuccess;
    if (t.buf64) k_gather_rows_sw<double><<<(unsigned)grid, 256, 0, st>>>(t, nvox, nvb);
    else k_gather_rows_sw<float><<<(unsigned)grid, 256, 0, st>>>(t, nvox, nvb);
    return cudaGetLastError();
}

cudaError_t inv_perm(const int32_t *perm_blk, int64_t n, int32_t *pos_blk, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_inv_perm<<<grid_cap(n), 256, 0, st>>>(perm_blk, n, pos_blk);
    return cudaGetLastError();
}

cudaError_t gather_sw_launch(const SwGather &t, cudaStream_t st)
{
    const int64_t grid = t.nbs + (t.nchunks * 32 + 255) / 256;
    if (grid <= 0) return cudaSuccess;
    if (t.buf64) k_gather_sw<double><<<(unsigned)grid, 256, 0, st>>>(t);
    else k_gather_sw<float><<<(unsigned)grid, 256, 0, st>>>(t);
    return cudaGetLastError();
}

cudaError_t march_sw64_launch(const SwMarch64 &m, int coarsen, cudaStream_t st)
{
    const int64_t grid = (m.nbundles + 7) / 8;
    if (grid <= 0) return cudaSuccess;
    if (coarsen == 2) k_march_sw<SwMarch64, 2, false><<<(unsigned)grid, 256, 0, st>>>(m);
    else k_march_sw<SwMarch64, 1, false><<<(unsigned)grid, 256, 0, st>>>(m);
    return cudaGetLastError();
}

cudaError_t coef_stream64(const uint32_t *vox, const double *len64, const double *chi, int64_t nseg, Wd4 *cw,
                          cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    k_coef_stream64<<<grid_cap(nseg), 256, 0, st>>>(vox, len64, chi, nseg, cw);
    return cudaGetLastError();
}

cudaError_t seg_weight64(const uint32_t *vox, const double *len64, const int64_t *ang_seg_off, int n_ang,
                         const double *wt, const double *invL, int nvox, int64_t nseg, double *cg, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    k_seg_weight64<<<grid_cap(nseg), 256, 0, st>>>(vox, len64, ang_seg_off, n_ang, wt, invL, nvox, nseg, cg);
    return cudaGetLastError();
}

cudaError_t coef_stream(const uint32_t *vox, const double *len64, const double *chi, int64_t nseg, float4 *cw,
                        cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    k_coef_stream<<<grid_cap(nseg), 256, 0, st>>>(vox, len64, chi, nseg, cw);
    return cudaGetLastError();
}

cudaError_t coef_stream_fold(const uint32_t *vox, const double *len64, const double *chi, const int64_t *ang_seg_off,
                             int n_ang, const double *wt, const double *invL, int nvox, int64_t nseg, float4 *cw,
                             cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    k_coef_stream_fold<<<grid_cap(nseg), 256, 0, st>>>(vox, len64, chi, ang_seg_off, n_ang, wt, invL, nvox, nseg, cw);
    return cudaGetLastError();
}

cudaError_t seg_weight(const uint32_t *vox, const double *len64, const int64_t *ang_seg_off, int n_ang,
                       const double *wt, const double *invL, int nvox, int64_t nseg, float *cg, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    k_seg_weight<<<grid_cap(nseg), 256, 0, st>>>(vox, len64, ang_seg_off, n_ang, wt, invL, nvox, nseg, cg);
    return cudaGetLastError();
}

}  // namespace rtk
