// nn_krylov.cu -- the operator-splitting step of the nearest-neighbour Lambda*
// (Sect. 3.2.1): (I - (1-eps) L*) x = y, with L* the 27-entry rows of nn.cu.
//
// With D the diagonal of A = I - (1-eps) L*, the Jacobi-preconditioned system
// is (I - M) x = D^-1 y with M_q,v = (1-eps_v) L*_q,v / D_v off the diagonal;
// a Jacobi sweep is x' = D^-1 y + M x and its change r = x' - x is the
// preconditioned residual.  The solve stops when a sweep would change x by at
// most jtol max |x'| and returns that sweep's x' (the criterion of the plain
// Jacobi iteration, which in optically thick grids at small eps contracts by a
// factor close to 1 per sweep: thousands of sweeps at eps = 1e-4, tau = 1e2).
//
// It gets there by defect correction: r is evaluated in FP64, the correction
// (I - M) d = r is solved by BiCGSTAB in FP32 to about 1e-5 of r, and x += d;
// each round gains about five decades.  The FP64 pipe, narrow on this GPU, only
// evaluates r (26 FMAs per voxel per round).  Should a round fail to halve r,
// the corrections are solved by BiCGSTAB in FP64 from then on; should the
// rounds run out, Jacobi sweeps finish the solve.
//
// Each block owns a contiguous range of voxels.  Where it fits in shared
// memory, the FP32 solve keeps the block's halo of the 27-point stencil
// (its range widened by n2 n3 + 2 n3 voxels either side on the spherical grid,
// n2 n3 + n3 + 1 on the cylindrical one) of r, p and v there, and the block's
// FP32 rows of M too where those fit: a phase loads the halo once from L2
// (16-byte asynchronous copies that bypass L1) and forms p = r + beta (p -
// omega v) and s = r - alpha v over it, so a BiCGSTAB iteration needs three
// grid barriers, not five, and the neighbour reads of the matrix-vector
// products are shared-memory reads (neighbours past the halo, across the
// cylindrical grid's phi seam, are formed from L2 the same way).
//
// The whole solve is one cooperative launch.  A vector operation on 1e5 voxels
// is a few microseconds of work, so one launch per BiCGSTAB phase plus a host
// round trip for each stopping test cost more than the arithmetic.  All blocks
// are resident and meet at a grid barrier between phases; every block sums the
// per-block partials of a reduction in the same fixed order, so all blocks
// take the same decisions and the solve is deterministic.  Every barrier wait
// is bounded: a block that has waited a second (or sees that another block
// gave up) raises the fail word and returns, and the host reports a timeout.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "rt_internal.h"

namespace rtk {
namespace {

constexpr int RT_ = 512;              // threads per block
constexpr int OS_BLOCKS_PER_SM = 1;   // resident blocks per SM the launch asks for (at most)
constexpr int MAXB = 2048;            // blocks of the launch at most (partial slots per region)
constexpr int PW = 4;                 // partial words per block and region
constexpr int MAX_ROUNDS = 40;        // defect-correction rounds before Jacobi sweeps take over
constexpr double TOL32 = 1e-5;        // FP32 correction solve: residual relative to r
enum { R_RES, R_START, R_RV, R_TS, R_RR, R_J0, R_J1, R_N };          // reduction regions
enum { W_BAR, W_FAIL, W_ITS, W_SWEEPS, W_STATUS, W_XSEL, W_N };      // control words
constexpr unsigned long long WAIT_NS = 1000000000ull;  // a barrier wait gives up after 1 s
constexpr unsigned WAIT_POLLS = 1u << 26;              // or after this many polls

template <typename T>
struct Inner {  // one BiCGSTAB's vectors and the preconditioned rows in its precision
    T *d, *r, *rh, *p, *v, *s, *t;
    T *M;        // 27 planes (plane 13 unused), written and read by the thread owning the row
    int64_t ms;  // plane stride: n for FP64, n rounded up to 4 for FP32 (16-byte aligned planes)
};

struct Kv {  // the solve's vectors and constants
    int n, sph, n1, n2, n3;
    const double *L27, *eps, *y;
    double *x, *x1, *res, *yd;  // iterate, Jacobi output x', FP64 residual r, D^-1 y
    Inner<double> i64;
    Inner<float> i32;
    double *part;   // R_N regions of PW * MAXB partials
    unsigned *ctl;  // W_N control words (zeroed before the launch)
    double jtol;
    int krylov, kmax, jmax, stall;
    int64_t n4;     // n rounded up to 4: stride of the FP32 vectors
    int rows;       // voxels per block, a multiple of 4: block b owns [b rows, (b + 1) rows)
    int halo;       // halo reach in voxel index either side of the block's range
    int hcap;       // halo buffer length in shared memory (floats, a multiple of 4)
    int tile;       // the FP32 solve keeps its halos in shared memory
    int msm;        // ... and the block's FP32 rows M too
};

#define OWN(i) for (int i = lo + (int)threadIdx.x; i < hi; i += RT_)

__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

// Maxima of non-negative values (or NaN) on their bit patterns: for
// non-negative values the order of the bits is the numeric order, and +inf and
// NaN sort last, so a non-finite entry survives the reduction.  Integer pipe.
__device__ __forceinline__ double maxb(double a, double b)
{
    const unsigned long long x = (unsigned long long)__double_as_longlong(a),
                             y = (unsigned long long)__double_as_longlong(b);
    return __longlong_as_double((long long)(x > y ? x : y));
}
__device__ __forceinline__ float maxb(float a, float b)
{
    const unsigned x = __float_as_uint(a), y = __float_as_uint(b);
    return __uint_as_float(x > y ? x : y);
}

// |a| by clearing the sign bit
__device__ __forceinline__ double absb(double a)
{
    return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ float absb(float a) { return __uint_as_float(__float_as_uint(a) & 0x7fffffffu); }

// Calls f(q, u) for each neighbour u of voxel v that exists, in slot order
// q = 9 (di+1) + 3 (dj+1) + (dk+1), q != 13; the phi axis (k spherical, j
// cylindrical) is periodic.  The offsets along each axis are formed once per
// voxel, so a neighbour costs an add and a predicate.
template <class F>
__device__ __forceinline__ void for_neighbours(const Kv &a, int v, F &&f)
{
    const int n23 = a.n2 * a.n3;
    const int i0 = v / n23, rem = v - i0 * n23, j0 = rem / a.n3, k0 = rem - j0 * a.n3;
    int oij[9], ok3[3];
    bool vij[9], vk3[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int j = j0 + d - 1, k = k0 + d - 1;
        if (a.sph) k = (k < 0) ? k + a.n3 : ((k >= a.n3) ? k - a.n3 : k);
        else j = (j < 0) ? j + a.n2 : ((j >= a.n2) ? j - a.n2 : j);
        ok3[d] = k - k0;
        vk3[d] = k >= 0 && k < a.n3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int i = i0 + c - 1;
            oij[3 * c + d] = (c - 1) * n23 + (j - j0) * a.n3;
            vij[3 * c + d] = i >= 0 && i < a.n1 && j >= 0 && j < a.n2;
        }
    }
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        if (q == 13) continue;
        if (vij[q / 3] && vk3[q % 3]) f(q, v + oij[q / 3] + ok3[q % 3]);
    }
}

// acc +- sum over q != 13 of M_q,v u[neighbour q of v] (minus with NEG); u is
// read past L1, since other blocks of this launch wrote it
template <bool NEG, typename T>
__device__ __forceinline__ T rowdot(const Kv &a, const T *M, int64_t ms, int v, const T *u, T acc)
{
    for_neighbours(a, v, [&](int q, int w) {
        const T m = M[q * ms + v];
        acc = fmat(NEG ? -m : m, __ldcg(u + w), acc);
    });
    return acc;
}

// w[0..K) reduced over the block (a sum, or the maxb maximum where bit c of
// MAXM is set; in T within each warp, then in FP64 over the warps) into the
// block's slot of a reduction region
template <int K, unsigned MAXM, typename T>
__device__ __forceinline__ void block_reduce(T (&w)[K], double *region)
{
    __shared__ double red[K][RT_ / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const T u = __shfl_down_sync(0xffffffffu, w[c], o);
            w[c] = ((MAXM >> c) & 1u) ? maxb(w[c], u) : w[c] + u;
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) red[c][threadIdx.x >> 5] = (double)w[c];
    __syncthreads();
    if (threadIdx.x < K) {
        const int c = threadIdx.x;
        double s = red[c][0];
        for (int q = 1; q < RT_ / 32; ++q) s = ((MAXM >> c) & 1u) ? maxb(s, red[c][q]) : s + red[c][q];
        __stcg(region + PW * blockIdx.x + c, s);
    }
}

// totals of a region's gridDim.x partials in one fixed order (lane l of warp 0
// takes blocks l, l + 32, ..., eight loads in flight; then a fixed shuffle
// tree), given to every thread
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// 16-byte asynchronous copy from global to shared memory, cached in L2 only
// (other blocks of this launch write the source); done at cp_async_wait
__device__ __forceinline__ void cp_async16(float *smem, const float *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// floats [b4, e4) of g (multiples of 4) into h[0 .. e4 - b4), asynchronously
__device__ __forceinline__ void halo_copy(float *h, const float *g, int b4, int e4)
{
    for (int j = 4 * (int)threadIdx.x; j < e4 - b4; j += 4 * RT_) cp_async16(h + j, g + b4 + j);
}

template <int K, unsigned MAXM, bool WAIT = false>
__device__ __forceinline__ void grid_total(const double *region, double (&out)[K])
{
    __shared__ double tot[K];
    if (threadIdx.x < 32) {
        double s[K];
#pragma unroll
        for (int c = 0; c < K; ++c) s[c] = 0.0;
        for (int b0 = threadIdx.x; b0 < (int)gridDim.x; b0 += 256) {
            double u[8][K];
#pragma unroll
            for (int h = 0; h < 8; ++h)
#pragma unroll
                for (int c = 0; c < K; ++c)
                    u[h][c] = b0 + 32 * h < (int)gridDim.x ? __ldcg(region + PW * (b0 + 32 * h) + c) : 0.0;
#pragma unroll
            for (int h = 0; h < 8; ++h)
#pragma unroll
                for (int c = 0; c < K; ++c) s[c] = ((MAXM >> c) & 1u) ? maxb(s[c], u[h][c]) : s[c] + u[h][c];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const double u = __shfl_down_sync(0xffffffffu, s[c], o);
                s[c] = ((MAXM >> c) & 1u) ? maxb(s[c], u) : s[c] + u;
            }
        if (threadIdx.x == 0)
#pragma unroll
            for (int c = 0; c < K; ++c) tot[c] = s[c];
    }
    if (WAIT) cp_async_wait();  // this thread's copies, issued before the totals' loads
    __syncthreads();
#pragma unroll
    for (int c = 0; c < K; ++c) out[c] = tot[c];
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void add_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of the cooperative launch; gen counts the arrivals expected
// so far.  The block's writes are ordered before its release arrival by the
// block barrier; the acquire load that sees every arrival orders the other
// blocks' writes before what follows.  arrive = false leaves this block's
// arrival out (the test hook that makes every wait of the launch run out).
// False when the wait gave up: the fail word is then set and every block
// returns at its next barrier.
__device__ __forceinline__ bool grid_sync(unsigned *ctl, unsigned &gen, bool arrive)
{
    __shared__ int ok;
    __syncthreads();
    gen += gridDim.x;
    if (threadIdx.x == 0) {
        int good = 1;
        if (arrive) add_release(ctl + W_BAR, 1u);
        unsigned long long t0 = 0;
        for (unsigned polls = 1; (int)(ld_acquire(ctl + W_BAR) - gen) < 0; ++polls) {
            if ((polls & 255u) == 0u) {  // every 256 polls: the clock, the fail word
                const unsigned long long t = now_ns();
                if (t0 == 0) t0 = t;
                if (ld_acquire(ctl + W_FAIL) != 0u || polls >= WAIT_POLLS || t - t0 > WAIT_NS) {
                    atomicExch(ctl + W_FAIL, 1u);
                    good = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// BiCGSTAB in T on (I - M) d = r (r the FP64 residual, own rows) from d = 0,
// until max |residual| <= tol, a breakdown, `window` iterations without
// halving the residual, or kmax iterations.  Vectors in global memory; each
// thread owns the same voxels of the block's range in every phase, so only the
// neighbour reads of the matrix-vector products and the partials cross blocks.
// Returns the iterations, or -1 when a barrier wait gave up.
template <typename T, class Sync>
__device__ __forceinline__ int bicgstab(const Kv &a, const Inner<T> &b, double tol, int window, Sync &sync, int lo, int hi)
{
    double *const reg = a.part;
    T w0[1] = {T(0)};
    OWN(i) {
        const T ri = (T)a.res[i];
        b.d[i] = T(0);
        b.r[i] = ri;
        b.rh[i] = ri;
        b.p[i] = T(0);
        b.v[i] = T(0);
        w0[0] = fmat(ri, ri, w0[0]);
    }
    block_reduce<1, 0u>(w0, reg + R_START * PW * MAXB);
    if (!sync()) return -1;
    double t1[1];
    grid_total<1, 0u>(reg + R_START * PW * MAXB, t1);
    double rho = t1[0], alpha = 1.0, omega = 1.0, beta = 0.0, best = INFINITY;
    int best_it = 0, it = 0;
    while (it < a.kmax) {
        ++it;
        bool bad = false;
        // p = r + beta (p - omega v)
        {
            const T bt = (T)beta, om = (T)omega;
            OWN(i) b.p[i] = fmat(bt, fmat(-om, b.v[i], b.p[i]), b.r[i]);
        }
        if (!sync()) return -1;
        // v = (I - M) p; alpha = rho / (rh, v)
        T w1[1] = {T(0)};
        OWN(i) {
            const T vi = rowdot<true>(a, b.M, b.ms, i, b.p, b.p[i]);
            b.v[i] = vi;
            w1[0] = fmat(b.rh[i], vi, w1[0]);
        }
        block_reduce<1, 0u>(w1, reg + R_RV * PW * MAXB);
        if (!sync()) return -1;
        grid_total<1, 0u>(reg + R_RV * PW * MAXB, t1);
        alpha = rho / t1[0];
        if (!(t1[0] != 0.0) || !isfinite(alpha)) {
            bad = true;
            alpha = 0.0;
        }
        // s = r - alpha v
        {
            const T al = (T)alpha;
            OWN(i) b.s[i] = fmat(-al, b.v[i], b.r[i]);
        }
        if (!sync()) return -1;
        // t = (I - M) s; omega = (t, s) / (t, t)
        T w2[2] = {T(0), T(0)};
        OWN(i) {
            const T si = b.s[i];
            const T ti = rowdot<true>(a, b.M, b.ms, i, b.s, si);
            b.t[i] = ti;
            w2[0] = fmat(ti, si, w2[0]);
            w2[1] = fmat(ti, ti, w2[1]);
        }
        block_reduce<2, 0u>(w2, reg + R_TS * PW * MAXB);
        if (!sync()) return -1;
        double t2[2];
        grid_total<2, 0u>(reg + R_TS * PW * MAXB, t2);
        omega = t2[1] > 0.0 ? t2[0] / t2[1] : 0.0;
        if (!isfinite(omega)) {
            bad = true;
            omega = 0.0;
        }
        // d += alpha p + omega s; r = s - omega t; rho = (rh, r); max |r|
        T w3[2] = {T(0), T(0)};
        {
            const T al = (T)alpha, om = (T)omega;
            OWN(i) {
                const T si = b.s[i];
                b.d[i] = fmat(om, si, fmat(al, b.p[i], b.d[i]));
                const T ri = fmat(-om, b.t[i], si);
                b.r[i] = ri;
                w3[0] = fmat(b.rh[i], ri, w3[0]);
                w3[1] = maxb(w3[1], absb(ri));
            }
        }
        block_reduce<2, 2u>(w3, reg + R_RR * PW * MAXB);
        if (!sync()) return -1;
        grid_total<2, 2u>(reg + R_RR * PW * MAXB, t2);
        const double rho_old = rho;
        rho = t2[0];
        beta = (rho / rho_old) * (alpha / omega);
        if (!isfinite(beta) || !(rho != 0.0)) bad = true;
        const double mr = t2[1];
        if (!isfinite(mr) || !(mr > tol) || bad) break;  // the FP64 residual judges the outcome
        if (mr < 0.5 * best) {
            best = mr;
            best_it = it;
        } else if (it - best_it >= window) {
            break;  // stagnation
        }
    }
    return it;
}

// The value at neighbour j of p = r + beta (p - omega v) or s = r - alpha v,
// formed by its owner in shared memory; a block that finds j outside its halo
// forms it from the published vectors with the same operations.
__device__ __forceinline__ float form_p(float r, float p, float v, float bt, float om)
{
    return fmaf(bt, fmaf(-om, v, p), r);
}
__device__ __forceinline__ float form_s(float r, float v, float al) { return fmaf(-al, v, r); }

// u_v - sum over q != 13 of M_q,v u[neighbour q of v], u read from the halo h
// (voxels hb .. he-1) or, past it, formed by far(j); M from the block's copy sm
// (plane stride rows, from voxel lo) or from global memory
template <class F>
__device__ __forceinline__ float rowdot_tile(const Kv &a, const float *sm, int lo, int v, const float *h, int hb, int he,
                                             F &&far, float acc)
{
    const unsigned span = (unsigned)(he - hb);
    for_neighbours(a, v, [&](int q, int u) {
        const float val = (unsigned)(u - hb) < span ? h[u - hb] : far(u);
        const float m = a.msm ? sm[q * a.rows + (v - lo)] : a.i32.M[q * a.i32.ms + v];
        acc = fmaf(-m, val, acc);
    });
    return acc;
}

// FP32 BiCGSTAB as bicgstab<float>, with the halos of r, p and v in shared
// memory and the own-range d, rh and t there too.  Published vectors (global,
// own rows): r, and p and v double-buffered, since a phase reads the previous
// iteration's p and v of its neighbours while their owners write the new ones.
// Phases: A (halos of r, p, v; p over the halo; v = (I - M) p), B (halo of v;
// s over the halo; t = (I - M) s), C (d, r); a grid barrier after each.  Adds
// d to x.  Returns the iterations, or -1 when a barrier wait gave up.
template <class Sync>
__device__ __forceinline__ int bicgstab_tile(const Kv &a, double tol, int window, Sync &sync, int lo, int hi)
{
    extern __shared__ float4 dsm4[];
    float *const dsm = reinterpret_cast<float *>(dsm4);
    double *const reg = a.part;
    // halo [hb, he) widened to 16-byte boundaries; hl floats copied per vector
    const int hb = max(0, lo - a.halo) & ~3;
    const int he = (int)min((long long)((min(a.n, hi + a.halo) + 3) & ~3), (long long)a.n4);
    const int hl = max(0, he - hb);
    float *const hr = dsm, *const hp = hr + a.hcap, *const hv = hp + a.hcap;
    float *const sd = hv + a.hcap, *const srh = sd + a.rows, *const st = srh + a.rows;
    float *const sm = st + a.rows;  // 27 planes of rows floats when a.msm
    if (a.msm && hi > lo) {
        const int e4 = (int)min((long long)((hi + 3) & ~3), (long long)a.n4);
        for (int q = 0; q < 27; ++q)
            if (q != 13) halo_copy(sm + q * a.rows, a.i32.M + q * a.i32.ms, lo, e4);
    }
    float *const gr = a.i32.r;
    // p and v double-buffered: buffer 0 in i32.p / i32.v, buffer 1 in i32.s / i32.t
    auto gp = [&](int c) { return c ? a.i32.s : a.i32.p; };
    auto gv = [&](int c) { return c ? a.i32.t : a.i32.v; };
    float w0[1] = {0.0f};
    OWN(i)
    {
        const float ri = (float)a.res[i];
        gr[i] = ri;
        srh[i - lo] = ri;
        sd[i - lo] = 0.0f;
        gp(0)[i] = 0.0f;
        gv(0)[i] = 0.0f;
        w0[0] = fmaf(ri, ri, w0[0]);
    }
    cp_async_wait();
    block_reduce<1, 0u>(w0, reg + R_START * PW * MAXB);
    if (!sync()) return -1;
    double rho = 0.0, alpha = 1.0, omega = 1.0, beta = 0.0, best = INFINITY;
    int best_it = 0, it = 0, cur = 0;
    bool bad = false;
    for (;;) {
        // A: halos of r, p, v (in flight while the totals that decide this iteration load)
        halo_copy(hr, gr, hb, he);
        halo_copy(hp, gp(cur), hb, he);
        halo_copy(hv, gv(cur), hb, he);
        if (it == 0) {
            double t1[1];
            grid_total<1, 0u, true>(reg + R_START * PW * MAXB, t1);
            rho = t1[0];
        } else {
            double t2[2];
            grid_total<2, 2u, true>(reg + R_RR * PW * MAXB, t2);
            const double rho_old = rho;
            rho = t2[0];
            beta = (rho / rho_old) * (alpha / omega);
            if (!isfinite(beta) || !(rho != 0.0)) bad = true;
            const double mr = t2[1];
            if (!isfinite(mr) || !(mr > tol) || bad) break;  // the FP64 residual judges the outcome
            if (mr < 0.5 * best) {
                best = mr;
                best_it = it;
            } else if (it - best_it >= window) {
                break;  // stagnation
            }
            if (it >= a.kmax) break;
        }
        ++it;
        const float bt = (float)beta, om = (float)omega;
        for (int j = threadIdx.x; j < hl; j += RT_) hp[j] = form_p(hr[j], hp[j], hv[j], bt, om);
        __syncthreads();
        float w1[1] = {0.0f};
        {
            const float *gpc = gp(cur), *gvc = gv(cur);
            float *gpn = gp(cur ^ 1), *gvn = gv(cur ^ 1);
            OWN(i)
            {
                const float pi = hp[i - hb];
                gpn[i] = pi;
                const float vi = rowdot_tile(
                    a, sm, lo, i, hp, hb, he,
                    [&](int u) { return form_p(__ldcg(gr + u), __ldcg(gpc + u), __ldcg(gvc + u), bt, om); }, pi);
                gvn[i] = vi;
                w1[0] = fmaf(srh[i - lo], vi, w1[0]);
            }
        }
        block_reduce<1, 0u>(w1, reg + R_RV * PW * MAXB);
        if (!sync()) return -1;
        // B: halo of v; alpha; s over the halo; t = (I - M) s
        halo_copy(hv, gv(cur ^ 1), hb, he);
        double t1[1];
        grid_total<1, 0u, true>(reg + R_RV * PW * MAXB, t1);
        alpha = rho / t1[0];
        if (!(t1[0] != 0.0) || !isfinite(alpha)) {
            bad = true;
            alpha = 0.0;
        }
        const float al = (float)alpha;
        for (int j = threadIdx.x; j < hl; j += RT_) hv[j] = form_s(hr[j], hv[j], al);
        __syncthreads();
        float w2[2] = {0.0f, 0.0f};
        {
            const float *gvn = gv(cur ^ 1);
            OWN(i)
            {
                const float si = hv[i - hb];
                const float ti =
                    rowdot_tile(a, sm, lo, i, hv, hb, he, [&](int u) { return form_s(__ldcg(gr + u), __ldcg(gvn + u), al); }, si);
                st[i - lo] = ti;
                w2[0] = fmaf(ti, si, w2[0]);
                w2[1] = fmaf(ti, ti, w2[1]);
            }
        }
        block_reduce<2, 0u>(w2, reg + R_TS * PW * MAXB);
        if (!sync()) return -1;
        // C: omega; d += alpha p + omega s; r = s - omega t (published); rho, max |r|
        double t2[2];
        grid_total<2, 0u>(reg + R_TS * PW * MAXB, t2);
        omega = t2[1] > 0.0 ? t2[0] / t2[1] : 0.0;
        if (!isfinite(omega)) {
            bad = true;
            omega = 0.0;
        }
        const float om2 = (float)omega;
        float w3[2] = {0.0f, 0.0f};
        OWN(i)
        {
            const float si = hv[i - hb];
            sd[i - lo] = fmaf(om2, si, fmaf(al, hp[i - hb], sd[i - lo]));
            const float ri = fmaf(-om2, st[i - lo], si);
            gr[i] = ri;
            w3[0] = fmaf(srh[i - lo], ri, w3[0]);
            w3[1] = maxb(w3[1], absb(ri));
        }
        block_reduce<2, 2u>(w3, reg + R_RR * PW * MAXB);
        if (!sync()) return -1;
        cur ^= 1;
    }
    OWN(i) a.x[i] += (double)sd[i - lo];
    return it;
}

__global__ void __launch_bounds__(RT_, 1) k_os_solve(Kv a)
{
    unsigned gen = 0;
    bool hold = a.stall != 0 && blockIdx.x == 0;
    auto sync = [&]() {
        const bool ok = grid_sync(a.ctl, gen, !hold);
        hold = false;
        return ok;
    };
    const int lo = min(a.n, (int)blockIdx.x * a.rows), hi = min(a.n, lo + a.rows);
    double *const reg = a.part;
    // preconditioned rows (FP64 and FP32), D^-1 y and x = 0 (own rows)
    OWN(i) {
        const double e = 1.0 - __ldg(a.eps + i);
        const double id = 1.0 / (1.0 - e * __ldg(a.L27 + 13 * (int64_t)a.n + i));
        const double f = e * id;
#pragma unroll
        for (int q = 0; q < 27; ++q)
            if (q != 13) {
                const double m = f * __ldg(a.L27 + (int64_t)q * a.n + i);
                a.i64.M[q * a.i64.ms + i] = m;
                a.i32.M[q * a.i32.ms + i] = (float)m;
            }
        a.yd[i] = __ldg(a.y + i) * id;
        a.x[i] = 0.0;
    }
    if (!sync()) return;
    int its = 0, sweeps = 0, status = 1;
    bool done = false;
    if (a.krylov) {
        double prev = INFINITY;
        bool fp64 = false;
        for (int round = 0; round <= MAX_ROUNDS; ++round) {
            // x' = D^-1 y + M x, r = x' - x; max |r|, max |x'|
            double w[2] = {0.0, 0.0};
            OWN(i) {
                const double xi = a.x[i];
                const double xn = rowdot<false>(a, a.i64.M, a.i64.ms, i, a.x, a.yd[i]);
                const double ri = xn - xi;
                a.x1[i] = xn;
                a.res[i] = ri;
                w[0] = maxb(w[0], absb(ri));
                w[1] = maxb(w[1], absb(xn));
            }
            block_reduce<2, 3u>(w, reg + R_RES * PW * MAXB);
            if (!sync()) return;
            double t[2];
            grid_total<2, 3u>(reg + R_RES * PW * MAXB, t);
            ++sweeps;
            const double mr = t[0], mx = t[1];
            if (!isfinite(mr) || !isfinite(mx)) {  // as the sweeps would: non-finite
                status = 2;
                done = true;
                break;
            }
            if (!(mr > a.jtol * mx)) {  // x' (in x1) meets the criterion
                status = 0;
                done = true;
                break;
            }
            if (round == MAX_ROUNDS) break;
            if (round > 0 && !(mr < 0.5 * prev)) fp64 = true;  // the FP32 corrections stopped paying
            prev = mr;
            const int k = fp64 ? bicgstab(a, a.i64, 0.5 * a.jtol * mx, 64, sync, lo, hi)
                    : a.tile ? bicgstab_tile(a, TOL32 * mr, 16, sync, lo, hi)
                             : bicgstab(a, a.i32, TOL32 * mr, 16, sync, lo, hi);
            if (k < 0) return;
            its += k;
            // x += d (the shared-memory solve has added its d)
            if (fp64)
                OWN(i) a.x[i] += a.i64.d[i];
            else if (!a.tile)
                OWN(i) a.x[i] += (double)a.i32.d[i];
            if (!sync()) return;
        }
    }
    // Jacobi sweeps from x (zero without Krylov) until one changes x by <= jtol
    // max |x'|, tested after every sweep
    double *xi = a.x, *xo = a.x1;
    if (done) {
        xi = a.x1;  // the result
    } else {
        for (int m = 0;;) {
            double w4[2] = {0.0, 0.0};
            OWN(i) {
                const double xn = rowdot<false>(a, a.i64.M, a.i64.ms, i, xi, a.yd[i]);
                w4[0] = maxb(w4[0], absb(xn - xi[i]));
                w4[1] = maxb(w4[1], absb(xn));
                xo[i] = xn;
            }
            // consecutive sweeps alternate regions: a block may write the next
            // sweep's partials while a slower one still reads this sweep's
            double *rg = reg + ((m & 1) ? R_J1 : R_J0) * PW * MAXB;
            block_reduce<2, 3u>(w4, rg);
            if (!sync()) return;
            double t4[2];
            grid_total<2, 3u>(rg, t4);
            double *const tmp = xi;
            xi = xo;
            xo = tmp;
            ++m;
            ++sweeps;
            if (!isfinite(t4[0]) || !isfinite(t4[1])) {
                status = 2;
                break;
            }
            if (!(t4[0] > a.jtol * t4[1])) {
                status = 0;
                break;
            }
            if (m >= a.jmax) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl[W_ITS] = (unsigned)its;
        a.ctl[W_SWEEPS] = (unsigned)sweeps;
        a.ctl[W_STATUS] = (unsigned)status;
        a.ctl[W_XSEL] = xi == a.x1 ? 1u : 0u;
    }
}

// blocks of the cooperative launch on the current device: SMs x resident
// blocks per SM (at most OS_BLOCKS_PER_SM), cached per device
cudaError_t os_blocks(int *nb)
{
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < 64;
    if (cached && (*nb = cache[dev].load(std::memory_order_acquire)) > 0) return cudaSuccess;
    int sms = 0, coop = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    if (!coop) return cudaErrorNotSupported;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_os_solve, RT_, 0)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorLaunchOutOfResources;
    *nb = std::min(MAXB, sms * std::min(per, OS_BLOCKS_PER_SM));
    if (cached) cache[dev].store(*nb, std::memory_order_release);
    return cudaSuccess;
}

// Dynamic shared memory of the FP32 halo solve: three halo buffers of hcap and
// three own-range vectors of rows floats, plus the block's 27 planes of rows
// (*msm = 1) when that fits too, beside the kernel's static shared memory on
// the current device, with the kernel's attribute raised to it; 0 (the
// global-memory solve) when even the halos do not fit.
cudaError_t os_tile_smem(int hcap, int rows, size_t *smem, int *msm)
{
    *smem = 0;
    *msm = 0;
    int dev = 0, optin = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, k_os_solve)) != cudaSuccess) return e;
    const size_t base = sizeof(float) * (3 * (size_t)hcap + 3 * (size_t)rows);
    const size_t full = base + sizeof(float) * 27 * (size_t)rows;
    if (base + fa.sharedSizeBytes > (size_t)optin) return cudaSuccess;
    const bool rows_too = full + fa.sharedSizeBytes <= (size_t)optin;
    const size_t want = rows_too ? full : base;
    if ((e = cudaFuncSetAttribute(k_os_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_os_solve, RT_, want)) != cudaSuccess) return e;
    if (per >= 1) {
        *smem = want;
        *msm = rows_too;
    }
    return cudaSuccess;
}

// work layout in doubles: x, x1, res, yd (4 n); FP64 BiCGSTAB vectors (7 n);
// FP64 rows (27 n); FP32 vectors and rows (34 n4 floats = 17 n4, n4 = n rounded
// up to 4, so that every FP32 vector and plane starts on 16 bytes); partials;
// control
constexpr int64_t F64_VECS = 11, F64_ROWS = 27, F32_DOUBLES = 17;

int64_t round4(int64_t v) { return (v + 3) & ~(int64_t)3; }

}  // namespace

int64_t nn_os_work_elems(int nvox)
{
    return (F64_VECS + F64_ROWS) * (int64_t)nvox + F32_DOUBLES * round4(nvox) + (int64_t)R_N * PW * MAXB +
           (W_N + 1) / 2;
}

cudaError_t nn_os_solve(const NnOs &o, cudaStream_t st, double **x_out, int *krylov_its, int *sweeps, int *status)
{
    *status = 1;
    *krylov_its = 0;
    *sweeps = 0;
    const int n = o.nvox;
    if ((int64_t)o.n1 * o.n2 * o.n3 != (int64_t)n || n < 1) return cudaErrorInvalidValue;
    int nb = 0;
    cudaError_t e = os_blocks(&nb);
    if (e != cudaSuccess) return e;
    Kv a{};
    a.n = n;
    a.sph = o.sph;
    a.n1 = o.n1;
    a.n2 = o.n2;
    a.n3 = o.n3;
    a.L27 = o.L27;
    a.eps = o.eps;
    a.y = o.y;
    double *w = o.work;
    const int64_t N = n, N4 = round4(n);
    a.x = w;
    a.x1 = w + N;
    a.res = w + 2 * N;
    a.yd = w + 3 * N;
    double **slots64[] = {&a.i64.d, &a.i64.r, &a.i64.rh, &a.i64.p, &a.i64.v, &a.i64.s, &a.i64.t};
    for (int q = 0; q < 7; ++q) *slots64[q] = w + (4 + q) * N;
    a.i64.M = w + F64_VECS * N;
    a.i64.ms = N;
    float *f = reinterpret_cast<float *>(w + (F64_VECS + F64_ROWS) * N);
    float **slots32[] = {&a.i32.d, &a.i32.r, &a.i32.rh, &a.i32.p, &a.i32.v, &a.i32.s, &a.i32.t};
    for (int q = 0; q < 7; ++q) *slots32[q] = f + q * N4;
    a.i32.M = f + 7 * N4;
    a.i32.ms = N4;
    a.n4 = N4;
    a.part = w + (F64_VECS + F64_ROWS) * N + F32_DOUBLES * N4;
    a.ctl = reinterpret_cast<unsigned *>(a.part + (int64_t)R_N * PW * MAXB);
    a.jtol = o.jtol;
    a.krylov = o.krylov;
    a.kmax = std::max(1, o.kmax);
    a.jmax = std::max(1, o.jmax);
    a.stall = o.stall;
    a.rows = (int)round4((N + nb - 1) / nb);
    // stencil reach in voxel index: n2 n3 + n3 + 1, and on the spherical grid also
    // the k neighbours across the phi seam (n3 - 1 away); the cylindrical seam
    // (j, (n2 - 1) n3 away) is read past the halo
    a.halo = o.n2 * o.n3 + (o.sph ? 2 * o.n3 : o.n3 + 1);
    a.hcap = (int)round4(std::min<int64_t>(N4, (int64_t)a.rows + 2 * (int64_t)a.halo + 8));
    size_t smem = 0;
    if ((e = os_tile_smem(a.hcap, a.rows, &smem, &a.msm)) != cudaSuccess) return e;
    a.tile = smem > 0;
    if ((e = cudaMemsetAsync(a.ctl, 0, W_N * sizeof(unsigned), st)) != cudaSuccess) return e;
    void *args[] = {&a};
    if ((e = cudaLaunchCooperativeKernel((const void *)k_os_solve, dim3(nb), dim3(RT_), args, smem, st)) != cudaSuccess)
        return e;
    unsigned h[W_N];
    if ((e = cudaMemcpyAsync(h, a.ctl, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (h[W_FAIL] != 0u) {
        *status = 3;
        return cudaSuccess;
    }
    *krylov_its = (int)h[W_ITS];
    *sweeps = (int)h[W_SWEEPS];
    *status = (int)h[W_STATUS];
    *x_out = h[W_XSEL] ? a.x1 : a.x;
    return cudaSuccess;
}

}  // namespace rtk
