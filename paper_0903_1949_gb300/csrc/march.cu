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

#include "rt_internal.h"

namespace rtk {
namespace {

// 1/n! for n = 0..20
__device__ __forceinline__ double inv_fact(int n)
{
    const double f[21] = {1.0,
                          1.0,
                          1.0 / 2.0,
                          1.0 / 6.0,
                          1.0 / 24.0,
                          1.0 / 120.0,
                          1.0 / 720.0,
                          1.0 / 5040.0,
                          1.0 / 40320.0,
                          1.0 / 362880.0,
                          1.0 / 3628800.0,
                          1.0 / 39916800.0,
                          1.0 / 479001600.0,
                          1.0 / 6227020800.0,
                          1.0 / 87178291200.0,
                          1.0 / 1307674368000.0,
                          1.0 / 20922789888000.0,
                          1.0 / 355687428096000.0,
                          1.0 / 6402373705728000.0,
                          1.0 / 121645100408832000.0,
                          1.0 / 2432902008176640000.0};
    return f[n];
}

// Weights of one segment of optical depth x followed by p.
//   e0 = 1 - e^{-x},  f1 = (x - e0)/x,  f2 = (x(2 - e0) - 2 e0)/x
//   parabolic: alpha = e0 - f1 - f2/(x+p), beta = f1 + f2/p, gamma = -x f2/(p (x+p))
//   linear:    alpha = e0 - f1,           beta = f1,         gamma = 0
// f1 and f2 are odd/even power series in x that cancel catastrophically when
// evaluated from e0 at small x; below the threshold they are summed directly
// (Horner), above it they come from expm1.
struct Coef64 {
    static constexpr int NS = 19;  // series terms for x < 0.5
    __device__ __forceinline__ static void eval(double x, double p, bool para, double &E, double &al, double &be,
                                                double &ga)
    {
        double e0, f1, f2;
        if (x < 0.5) {
            double h1 = 0.0, h2 = 0.0;
#pragma unroll
            for (int n = NS + 1; n >= 2; --n) h1 = inv_fact(n) - x * h1;        // sum (-x)^(n-2)/n!
#pragma unroll
            for (int m = NS + 1; m >= 3; --m) h2 = (double)(m - 2) * inv_fact(m) - x * h2;
            f1 = x * h1;
            f2 = (x * x) * h2;
            e0 = x - x * f1;
            E = 1.0 - e0;
        } else {
            double em = expm1(-x);
            e0 = -em;
            E = 1.0 + em;
            f1 = (x - e0) / x;
            f2 = (x * (2.0 - e0) - 2.0 * e0) / x;
        }
        if (para) {
            double iD = 1.0 / (x + p), ip = 1.0 / p;
            al = (e0 - f1) - f2 * iD;
            be = f1 + f2 * ip;
            ga = -(x * f2) * (ip * iD);
        } else {
            al = e0 - f1;
            be = f1;
            ga = 0.0;
        }
    }
};

struct Coef32 {
    static constexpr int NS = 11;  // series terms for x < 1
    __device__ __forceinline__ static void eval(float x, float p, bool para, float &E, float &al, float &be, float &ga)
    {
        float e0, f1, f2;
        if (x < 1.0f) {
            float h1 = 0.0f, h2 = 0.0f;
#pragma unroll
            for (int n = NS + 1; n >= 2; --n) h1 = (float)inv_fact(n) - x * h1;
#pragma unroll
            for (int m = NS + 2; m >= 3; --m) h2 = (float)((double)(m - 2) * inv_fact(m)) - x * h2;
            f1 = x * h1;
            f2 = (x * x) * h2;
            e0 = x - x * f1;
            E = 1.0f - e0;
        } else {
            E = __expf(-x);
            e0 = 1.0f - E;
            float ix = __frcp_rn(x);
            f1 = (x - e0) * ix;
            f2 = (x * (2.0f - e0) - 2.0f * e0) * ix;
        }
        if (para) {
            float iD = __frcp_rn(x + p), ip = __frcp_rn(p);
            al = (e0 - f1) - f2 * iD;
            be = f1 + f2 * ip;
            ga = -(x * f2) * (ip * iD);
        } else {
            al = e0 - f1;
            be = f1;
            ga = 0.0f;
        }
    }
};

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

template <typename T, typename P>
__global__ void __launch_bounds__(256) k_march(const uint32_t *__restrict__ vox, const T *__restrict__ len,
                                               const int64_t *__restrict__ ray_off, int64_t r_lo, int64_t r_hi,
                                               int64_t seg_lo, int64_t nseg, const P *__restrict__ cs,
                                               const T *__restrict__ Bv, T I_outer, int homog, int parabolic,
                                               P *__restrict__ out, int chunk)
{
    using C = typename Traits<T>::C;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t c_lo = wg * chunk;
    if (c_lo >= nseg) return;
    const int64_t c_hi = (c_lo + chunk < nseg) ? c_lo + chunk : nseg;
    // the bundle: whole characteristics that start inside [c_lo, c_hi)
    const int64_t ra = lower_bound64(ray_off, r_lo, r_hi, seg_lo + c_lo);
    const int64_t rb = lower_bound64(ray_off, r_lo, r_hi, seg_lo + c_hi);
    const int64_t s_begin = ray_off[ra] - seg_lo;
    const int64_t s_end = ray_off[rb] - seg_lo;
    if (s_begin >= s_end) return;
    const uint32_t *vx = vox + seg_lo;
    const T *ln = len + seg_lo;
    T Icarry = 0, Sprev = 0, gprev = 0;
    for (int64_t base = s_begin; base < s_end; base += 32) {
        const int64_t s = base + lane;
        const bool valid = s < s_end;
        uint32_t w = 0;
        T l = 0, chi = 0, S = 0;
        if (valid) {
            w = __ldcs(vx + s);
            l = __ldcs(ln + s);
            P c = cs[w & RTK_VOXMASK];
            chi = c.x;
            S = c.y;
        }
        uint32_t wn = __shfl_down_sync(FULL, w, 1);
        T lnx = __shfl_down_sync(FULL, l, 1);
        T chin = __shfl_down_sync(FULL, chi, 1);
        T Sn = __shfl_down_sync(FULL, S, 1);
        if (lane == 31) {
            if (valid && s + 1 < s_end) {
                wn = vx[s + 1];
                lnx = ln[s + 1];
                P c = cs[wn & RTK_VOXMASK];
                chin = c.x;
                Sn = c.y;
            } else {
                wn = RTK_RAYSTART;
            }
        }
        const bool rstart = (w & RTK_RAYSTART) != 0u;
        const bool run0 = (w & (RTK_RAYSTART | RTK_RESTART)) != 0u;
        const bool last = (s + 1 >= s_end) || ((wn & (RTK_RAYSTART | RTK_RESTART)) != 0u);
        const T x = valid ? chi * l : (T)1;
        const T p = last ? (T)0 : chin * lnx;
        const bool para = parabolic && !last && (p >= (T)0.5 * x);
        T E, al, be, ga;
        C::eval(x, p, para, E, al, be, ga);
        T Sp = __shfl_up_sync(FULL, S, 1);
        T gp = __shfl_up_sync(FULL, ga, 1);
        if (lane == 0) {
            Sp = Sprev;
            gp = gprev;
        }
        const T Skm = run0 ? S : Sp;
        const T src = al * Skm + be * S + (para ? ga * Sn : (T)0);
        const T lam = be + (run0 ? al : gp * E);
        T A = E, b = src;
        if (rstart) {
            T Iin = homog ? (T)0 : ((w & RTK_CORE) ? Bv[w & RTK_VOXMASK] : I_outer);
            b = E * Iin + src;
            A = 0;
        }
        if (!valid) {
            A = 1;
            b = 0;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T Ao = __shfl_up_sync(FULL, A, o);
            T bo = __shfl_up_sync(FULL, b, o);
            if (lane >= o) {
                b = A * bo + b;
                A = A * Ao;
            }
        }
        const T I = A * Icarry + b;
        if (valid) {
            P o;
            o.x = l * I;
            o.y = l * lam;
            __stcg(out + s, o);
        }
        Icarry = __shfl_sync(FULL, I, 31);
        Sprev = __shfl_sync(FULL, S, 31);
        gprev = __shfl_sync(FULL, ga, 31);
    }
}

}  // namespace

template <typename T, typename P>
cudaError_t march_block(const uint32_t *vox, const T *len, const int64_t *ray_off, int64_t r_lo, int64_t r_hi,
                        int64_t seg_lo, int64_t nseg, const P *chiS, const T *B, T I_outer, int homog,
                        int parabolic, P *out, int chunk, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    int64_t warps = (nseg + chunk - 1) / chunk;
    int64_t blocks = (warps + 7) / 8;
    k_march<T, P><<<(unsigned)blocks, 256, 0, st>>>(vox, len, ray_off, r_lo, r_hi, seg_lo, nseg, chiS, B, I_outer, homog,
                                                    parabolic, out, chunk);
    return cudaGetLastError();
}

template cudaError_t march_block<double, double2>(const uint32_t *, const double *, const int64_t *, int64_t, int64_t,
                                                  int64_t, int64_t, const double2 *, const double *, double, int, int,
                                                  double2 *, int, cudaStream_t);
template cudaError_t march_block<float, float2>(const uint32_t *, const float *, const int64_t *, int64_t, int64_t,
                                                int64_t, int64_t, const float2 *, const float *, float, int, int,
                                                float2 *, int, cudaStream_t);

}  // namespace rtk
