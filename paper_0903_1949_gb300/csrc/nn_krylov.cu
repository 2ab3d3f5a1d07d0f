// nn_krylov.cu -- the operator-splitting step of the nearest-neighbour Lambda*
// (Sect. 3.2.1): (I - (1-eps) L*) x = y, with L* the 27-entry rows of nn.cu.
//
// In optically thick grids at small eps the Jacobi iteration contracts by a
// factor close to 1 per sweep (thousands of sweeps at eps = 1e-4, tau = 1e2).
// BiCGSTAB on the Jacobi-preconditioned system D^-1 A x = D^-1 y (D the
// diagonal of A) reaches the same solution in tens of iterations; it stops when
// its preconditioned residual, which is exactly the change one Jacobi sweep
// would make, is below jtol max |x|, and Jacobi sweeps then confirm that
// criterion on the true residual (or finish the solve if BiCGSTAB breaks down
// or stagnates).
//
// Each launch first scales the operator's off-diagonal entries into the
// preconditioned rows M_q,v = (1-eps_v) L*_q,v / D_v and forms D^-1 y, so that
// a row of D^-1 A is u_v - sum_q M_q,v u_q (26 FMAs, no division) and a Jacobi
// sweep is x_v = (D^-1 y)_v + sum_q M_q,v x_q: the solve is bound by the FP64
// pipe, which is narrow on this GPU, so the maxima of the stopping tests run
// on the integer pipe.
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
enum { R_START, R_RV, R_TS, R_RR, R_J0, R_J1, R_N };                 // reduction regions
enum { W_BAR, W_FAIL, W_ITS, W_SWEEPS, W_STATUS, W_XSEL, W_N };      // control words
constexpr unsigned long long WAIT_NS = 1000000000ull;  // a barrier wait gives up after 1 s
constexpr unsigned WAIT_POLLS = 1u << 26;              // or after this many polls

struct Kv {  // the solve's vectors and constants
    int n, sph, n1, n2, n3;
    const double *L27, *eps, *y;
    double *x, *x1, *r, *rh, *p, *v, *s, *t;
    double *yd;     // D^-1 y
    double *M;      // 27 planes of n: M_q,v (plane 13 unused), written and read by the thread owning v
    double *part;   // R_N regions of PW * MAXB partials
    unsigned *ctl;  // W_N control words (zeroed before the launch)
    double jtol;
    int krylov, kmax, jmax, stall;
};

// Maximum of two non-negative doubles (or NaN) on their bit patterns: for
// non-negative values the order of the bits is the numeric order, and +inf and
// NaN sort last, so a non-finite entry survives the reduction.  Integer pipe.
__device__ __forceinline__ double maxb(double a, double b)
{
    const unsigned long long x = (unsigned long long)__double_as_longlong(a),
                             y = (unsigned long long)__double_as_longlong(b);
    return __longlong_as_double((long long)(x > y ? x : y));
}

// |a| by clearing the sign bit
__device__ __forceinline__ double absb(double a)
{
    return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffll);
}

// acc +- sum over q != 13 of M_q,v u[neighbour q of v] (minus with NEG); u is
// read past L1, since other blocks of this launch wrote it
template <bool NEG>
__device__ __forceinline__ double rowdot(const Kv &a, int v, const double *u, double acc)
{
    const int k0 = v % a.n3, j0 = (v / a.n3) % a.n2, i0 = v / (a.n2 * a.n3);
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        if (q == 13) continue;
        int i = i0 + q / 9 - 1, j = j0 + (q / 3) % 3 - 1, k = k0 + q % 3 - 1;
        if (a.sph) k = (k < 0) ? k + a.n3 : ((k >= a.n3) ? k - a.n3 : k);  // phi periodic
        else j = (j < 0) ? j + a.n2 : ((j >= a.n2) ? j - a.n2 : j);
        if (i < 0 || i >= a.n1 || j < 0 || j >= a.n2 || k < 0 || k >= a.n3) continue;
        const double m = a.M[(int64_t)q * a.n + v];
        acc = fma(NEG ? -m : m, __ldcg(u + (i * a.n2 + j) * a.n3 + k), acc);
    }
    return acc;
}

// w[0..K) reduced over the block (a sum, or the maxb maximum where bit c of
// MAXM is set) into the block's slot of a reduction region
template <int K, unsigned MAXM>
__device__ __forceinline__ void block_reduce(double (&w)[K], double *region)
{
    __shared__ double red[K][RT_ / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const double u = __shfl_down_sync(0xffffffffu, w[c], o);
            w[c] = ((MAXM >> c) & 1u) ? maxb(w[c], u) : w[c] + u;
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) red[c][threadIdx.x >> 5] = w[c];
    __syncthreads();
    if (threadIdx.x < K) {
        const int c = threadIdx.x;
        double s = red[c][0];
        for (int q = 1; q < RT_ / 32; ++q) s = ((MAXM >> c) & 1u) ? maxb(s, red[c][q]) : s + red[c][q];
        __stcg(region + PW * blockIdx.x + c, s);
    }
}

// totals of a region's gridDim.x partials in one fixed order (thread b loads
// blocks b, b + RT_, ...; then the warps' shuffle trees and warp 0 over the
// warp sums), given to every thread
template <int K, unsigned MAXM>
__device__ __forceinline__ void grid_total(const double *region, double (&out)[K])
{
    __shared__ double wsum[K][RT_ / 32];
    __shared__ double tot[K];
    double s[K];
#pragma unroll
    for (int c = 0; c < K; ++c) s[c] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RT_)
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const double u = __ldcg(region + PW * b + c);
            s[c] = ((MAXM >> c) & 1u) ? maxb(s[c], u) : s[c] + u;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const double u = __shfl_down_sync(0xffffffffu, s[c], o);
            s[c] = ((MAXM >> c) & 1u) ? maxb(s[c], u) : s[c] + u;
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) wsum[c][threadIdx.x >> 5] = s[c];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int c = 0; c < K; ++c) s[c] = threadIdx.x < RT_ / 32 ? wsum[c][threadIdx.x] : 0.0;
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

// The OS-step solve; each thread owns the voxels first, first + stride, ...
// in every phase, so only the neighbour reads of the matrix-vector products
// and the partials cross blocks.
__global__ void __launch_bounds__(RT_) k_os_solve(Kv a)
{
    unsigned gen = 0;
    bool hold = a.stall != 0 && blockIdx.x == 0;
    auto sync = [&]() {
        const bool ok = grid_sync(a.ctl, gen, !hold);
        hold = false;
        return ok;
    };
    const int stride = gridDim.x * RT_;
    const int first = blockIdx.x * RT_ + threadIdx.x;
    double *const reg = a.part;
    // preconditioned rows and D^-1 y (own rows only: no barrier needed)
    for (int i = first; i < a.n; i += stride) {
        const double e = 1.0 - __ldg(a.eps + i);
        const double id = 1.0 / (1.0 - e * __ldg(a.L27 + 13 * (int64_t)a.n + i));
        const double f = e * id;
#pragma unroll
        for (int q = 0; q < 27; ++q)
            if (q != 13) a.M[(int64_t)q * a.n + i] = f * __ldg(a.L27 + (int64_t)q * a.n + i);
        a.yd[i] = __ldg(a.y + i) * id;
    }
    int its = 0;
    bool from_zero = true;
    if (a.krylov) {
        // x = 0, r = rh = D^-1 y, p = v = 0; rho = (rh, r); alpha = omega = 1
        double w0[1] = {0.0};
        for (int i = first; i < a.n; i += stride) {
            const double ri = a.yd[i];
            a.x[i] = 0.0;
            a.r[i] = ri;
            a.rh[i] = ri;
            a.p[i] = 0.0;
            a.v[i] = 0.0;
            w0[0] = fma(ri, ri, w0[0]);
        }
        block_reduce<1, 0u>(w0, reg + R_START * PW * MAXB);
        if (!sync()) return;
        double t1[1];
        grid_total<1, 0u>(reg + R_START * PW * MAXB, t1);
        double rho = t1[0], alpha = 1.0, omega = 1.0, beta = 0.0, best = INFINITY;
        int best_it = 0;
        for (int it = 1; it <= a.kmax; ++it) {
            bool bad = false;
            // p = r + beta (p - omega v)
            for (int i = first; i < a.n; i += stride) a.p[i] = fma(beta, fma(-omega, a.v[i], a.p[i]), a.r[i]);
            if (!sync()) return;
            // v = D^-1 A p; alpha = rho / (rh, v)
            double w1[1] = {0.0};
            for (int i = first; i < a.n; i += stride) {
                const double vi = rowdot<true>(a, i, a.p, a.p[i]);
                a.v[i] = vi;
                w1[0] = fma(a.rh[i], vi, w1[0]);
            }
            block_reduce<1, 0u>(w1, reg + R_RV * PW * MAXB);
            if (!sync()) return;
            grid_total<1, 0u>(reg + R_RV * PW * MAXB, t1);
            alpha = rho / t1[0];
            if (!(t1[0] != 0.0) || !isfinite(alpha)) {
                bad = true;
                alpha = 0.0;
            }
            // s = r - alpha v
            for (int i = first; i < a.n; i += stride) a.s[i] = fma(-alpha, a.v[i], a.r[i]);
            if (!sync()) return;
            // t = D^-1 A s; omega = (t, s) / (t, t)
            double w2[2] = {0.0, 0.0};
            for (int i = first; i < a.n; i += stride) {
                const double si = a.s[i];
                const double ti = rowdot<true>(a, i, a.s, si);
                a.t[i] = ti;
                w2[0] = fma(ti, si, w2[0]);
                w2[1] = fma(ti, ti, w2[1]);
            }
            block_reduce<2, 0u>(w2, reg + R_TS * PW * MAXB);
            if (!sync()) return;
            double t2[2];
            grid_total<2, 0u>(reg + R_TS * PW * MAXB, t2);
            omega = t2[1] > 0.0 ? t2[0] / t2[1] : 0.0;
            if (!isfinite(omega)) {
                bad = true;
                omega = 0.0;
            }
            // x += alpha p + omega s; r = s - omega t; rho = (rh, r); max |r|, max |x|
            double w3[3] = {0.0, 0.0, 0.0};
            for (int i = first; i < a.n; i += stride) {
                const double si = a.s[i];
                const double xi = fma(omega, si, fma(alpha, a.p[i], a.x[i]));
                const double ri = fma(-omega, a.t[i], si);
                a.x[i] = xi;
                a.r[i] = ri;
                w3[0] = fma(a.rh[i], ri, w3[0]);
                w3[1] = maxb(w3[1], absb(ri));
                w3[2] = maxb(w3[2], absb(xi));
            }
            block_reduce<3, 6u>(w3, reg + R_RR * PW * MAXB);
            if (!sync()) return;
            double t3[3];
            grid_total<3, 6u>(reg + R_RR * PW * MAXB, t3);
            const double rho_old = rho;
            rho = t3[0];
            beta = (rho / rho_old) * (alpha / omega);
            if (!isfinite(beta) || !(rho != 0.0)) {
                bad = true;
                beta = 0.0;
            }
            its = it;
            const double mr = t3[1], mx = t3[2];
            if (!isfinite(mr) || !isfinite(mx)) {  // the sweeps start again from zero
                from_zero = true;
                break;
            }
            from_zero = false;
            if (!(mr > a.jtol * mx)) break;  // the sweeps confirm it
            if (bad) break;                  // breakdown: the sweeps go on from x
            if (mr < 0.5 * best) {
                best = mr;
                best_it = it;
            } else if (it - best_it >= 64) {
                break;  // stagnation
            }
        }
    }
    if (from_zero)
        for (int i = first; i < a.n; i += stride) a.x[i] = 0.0;
    if (!sync()) return;
    // Jacobi sweeps x' = D^-1 y + M x until one changes x by <= jtol max |x'|
    // (the criterion of the plain iteration), tested after every sweep
    double *xi = a.x, *xo = a.x1;
    int m = 0, status = 1;
    for (;;) {
        double w4[2] = {0.0, 0.0};
        for (int i = first; i < a.n; i += stride) {
            const double xn = rowdot<false>(a, i, xi, a.yd[i]);
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
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl[W_ITS] = (unsigned)its;
        a.ctl[W_SWEEPS] = (unsigned)m;
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

}  // namespace

int64_t nn_os_work_elems(int nvox) { return 36 * (int64_t)nvox + (int64_t)R_N * PW * MAXB + (W_N + 1) / 2; }

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
    a.x = w;
    a.x1 = w + n;
    a.r = w + 2 * (int64_t)n;
    a.rh = w + 3 * (int64_t)n;
    a.p = w + 4 * (int64_t)n;
    a.v = w + 5 * (int64_t)n;
    a.s = w + 6 * (int64_t)n;
    a.t = w + 7 * (int64_t)n;
    a.yd = w + 8 * (int64_t)n;
    a.M = w + 9 * (int64_t)n;
    a.part = w + 36 * (int64_t)n;
    a.ctl = reinterpret_cast<unsigned *>(a.part + (int64_t)R_N * PW * MAXB);
    a.jtol = o.jtol;
    a.krylov = o.krylov;
    a.kmax = o.kmax;
    a.jmax = std::max(1, o.jmax);
    a.stall = o.stall;
    if ((e = cudaMemsetAsync(a.ctl, 0, W_N * sizeof(unsigned), st)) != cudaSuccess) return e;
    void *args[] = {&a};
    if ((e = cudaLaunchCooperativeKernel((const void *)k_os_solve, dim3(nb), dim3(RT_), args, 0, st)) != cudaSuccess)
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
