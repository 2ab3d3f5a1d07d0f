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
// or stagnates).  Every reduction sums block partials in a fixed order, so the
// solve is deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "rt_internal.h"

namespace rtk {
namespace {

constexpr int RT_ = 256;     // threads per block
constexpr int RBLK = 304;    // partial-sum blocks
// device scalars
enum { S_RHO_OLD, S_ALPHA, S_OMEGA, S_RHO, S_BETA, S_MAXR, S_MAXX, S_BAD, S_NSC };

// (A u)_v / D_v, A = I - (1-eps) L*, D_v = 1 - (1-eps_v) L*_v,13
__device__ __forceinline__ double apply_row(int v, int sph, int n1, int n2, int n3, const double *L27,
                                            const double *eps, const double *u)
{
    const int nvox = n1 * n2 * n3;
    const int k0 = v % n3, j0 = (v / n3) % n2, i0 = v / (n2 * n3);
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        if (q == 13) continue;
        int i = i0 + q / 9 - 1, j = j0 + (q / 3) % 3 - 1, k = k0 + q % 3 - 1;
        if (sph) k = (k < 0) ? k + n3 : ((k >= n3) ? k - n3 : k);
        else j = (j < 0) ? j + n2 : ((j >= n2) ? j - n2 : j);
        if (i < 0 || i >= n1 || j < 0 || j >= n2 || k < 0 || k >= n3) continue;
        acc += L27[(int64_t)q * nvox + v] * u[(i * n2 + j) * n3 + k];
    }
    const double e = 1.0 - eps[v];
    const double d = 1.0 - e * L27[13 * (int64_t)nvox + v];
    return u[v] - e * acc / d;  // (u - e L13 u - e acc) / d = u - e acc / d
}

// sum (or max, MAX) of three values over the block into part[3 blockIdx.x + c]
template <bool MAX>
__device__ __forceinline__ void block3(double a, double b, double c, double *part)
{
    __shared__ double red[3][RT_ / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const double xa = __shfl_down_sync(0xffffffffu, a, o), xb = __shfl_down_sync(0xffffffffu, b, o),
                     xc = __shfl_down_sync(0xffffffffu, c, o);
        a = MAX ? fmax(a, xa) : a + xa;
        b = MAX ? fmax(b, xb) : b + xb;
        c = MAX ? fmax(c, xc) : c + xc;
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = a;
        red[1][w] = b;
        red[2][w] = c;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = red[threadIdx.x][0];
        for (int q = 1; q < RT_ / 32; ++q) s = MAX ? fmax(s, red[threadIdx.x][q]) : s + red[threadIdx.x][q];
        part[3 * blockIdx.x + threadIdx.x] = s;
    }
}

// the three totals of the RBLK partials (fixed order) in tot[0..2], by one block
template <bool MAX>
__device__ __forceinline__ void final3(const double *part, double *tot)
{
    __shared__ double red[3][RT_];
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int b = threadIdx.x; b < RBLK; b += RT_) s = MAX ? fmax(s, part[3 * b + c]) : s + part[3 * b + c];
        red[c][threadIdx.x] = s;
    }
    __syncthreads();
    for (int h = RT_ / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 3; ++c)
                red[c][threadIdx.x] = MAX ? fmax(red[c][threadIdx.x], red[c][threadIdx.x + h])
                                          : red[c][threadIdx.x] + red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) tot[threadIdx.x] = red[threadIdx.x][0];
}

struct Kv {  // the solve's vectors and constants
    int n, sph, n1, n2, n3;
    const double *L27, *eps, *y;
    double *x, *r, *rh, *p, *v, *s, *t;
    double *part, *part2, *sc;
};

#define GRID_LOOP(i) for (int i = blockIdx.x * RT_ + threadIdx.x; i < a.n; i += RBLK * RT_)

// x = 0, r = rh = D^-1 y, p = v = 0; rho = (rh, r); alpha = omega = rho_old = 1
__global__ void __launch_bounds__(RT_) k_bi_start(Kv a)
{
    double dot = 0.0;
    GRID_LOOP(i)
    {
        const double e = 1.0 - a.eps[i];
        const double r = a.y[i] / (1.0 - e * a.L27[13 * (int64_t)a.n + i]);
        a.x[i] = 0.0;
        a.r[i] = r;
        a.rh[i] = r;
        a.p[i] = 0.0;
        a.v[i] = 0.0;
        dot += r * r;
    }
    block3<false>(dot, 0.0, 0.0, a.part);
}

__global__ void __launch_bounds__(RT_) k_bi_f0(Kv a)
{
    __shared__ double t3[3];
    final3<false>(a.part, t3);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.sc[S_RHO] = t3[0];
        a.sc[S_RHO_OLD] = 1.0;
        a.sc[S_ALPHA] = 1.0;
        a.sc[S_OMEGA] = 1.0;
        a.sc[S_BETA] = 0.0;
        a.sc[S_BAD] = 0.0;
        a.sc[S_MAXR] = INFINITY;
        a.sc[S_MAXX] = 0.0;
    }
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(RT_) k_bi_p(Kv a)
{
    const double beta = a.sc[S_BETA], omega = a.sc[S_OMEGA];
    GRID_LOOP(i) a.p[i] = a.r[i] + beta * (a.p[i] - omega * a.v[i]);
}

// v = D^-1 A p; partial (rh, v)
__global__ void __launch_bounds__(RT_) k_bi_mv1(Kv a)
{
    double dot = 0.0;
    GRID_LOOP(i)
    {
        const double vi = apply_row(i, a.sph, a.n1, a.n2, a.n3, a.L27, a.eps, a.p);
        a.v[i] = vi;
        dot += a.rh[i] * vi;
    }
    block3<false>(dot, 0.0, 0.0, a.part);
}

// alpha = rho / (rh, v)
__global__ void __launch_bounds__(RT_) k_bi_f1(Kv a)
{
    __shared__ double t3[3];
    final3<false>(a.part, t3);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double al = a.sc[S_RHO] / t3[0];
        if (!(t3[0] != 0.0) || !isfinite(al)) {
            a.sc[S_BAD] = 1.0;
            a.sc[S_ALPHA] = 0.0;
        } else {
            a.sc[S_ALPHA] = al;
        }
    }
}

// s = r - alpha v
__global__ void __launch_bounds__(RT_) k_bi_s(Kv a)
{
    const double al = a.sc[S_ALPHA];
    GRID_LOOP(i) a.s[i] = a.r[i] - al * a.v[i];
}

// t = D^-1 A s; partials (t, s), (t, t)
__global__ void __launch_bounds__(RT_) k_bi_mv2(Kv a)
{
    double ts = 0.0, tt = 0.0;
    GRID_LOOP(i)
    {
        const double ti = apply_row(i, a.sph, a.n1, a.n2, a.n3, a.L27, a.eps, a.s);
        a.t[i] = ti;
        ts += ti * a.s[i];
        tt += ti * ti;
    }
    block3<false>(ts, tt, 0.0, a.part);
}

// omega = (t, s) / (t, t)
__global__ void __launch_bounds__(RT_) k_bi_f2(Kv a)
{
    __shared__ double t3[3];
    final3<false>(a.part, t3);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double om = t3[1] > 0.0 ? t3[0] / t3[1] : 0.0;
        a.sc[S_OMEGA] = isfinite(om) ? om : 0.0;
        if (!isfinite(om)) a.sc[S_BAD] = 1.0;
    }
}

// x += alpha p + omega s; r = s - omega t; partials (rh, r) and max |r|, max |x|
__global__ void __launch_bounds__(RT_) k_bi_xr(Kv a)
{
    const double al = a.sc[S_ALPHA], om = a.sc[S_OMEGA];
    double dot = 0.0, mr = 0.0, mx = 0.0;
    GRID_LOOP(i)
    {
        const double xi = a.x[i] + al * a.p[i] + om * a.s[i];
        const double ri = a.s[i] - om * a.t[i];
        a.x[i] = xi;
        a.r[i] = ri;
        dot += a.rh[i] * ri;
        mr = fmax(mr, fabs(ri));
        mx = fmax(mx, fabs(xi));
    }
    block3<false>(dot, 0.0, 0.0, a.part);
    __syncthreads();
    block3<true>(mr, mx, 0.0, a.part2);
}

// rho_old = rho, rho = (rh, r), beta = (rho / rho_old) (alpha / omega); max |r|, max |x|
__global__ void __launch_bounds__(RT_) k_bi_f3(Kv a)
{
    __shared__ double t3[3], m3[3];
    final3<false>(a.part, t3);
    __syncthreads();
    final3<true>(a.part2, m3);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double rho_old = a.sc[S_RHO], rho = t3[0];
        const double beta = (rho / rho_old) * (a.sc[S_ALPHA] / a.sc[S_OMEGA]);
        a.sc[S_RHO_OLD] = rho_old;
        a.sc[S_RHO] = rho;
        a.sc[S_BETA] = isfinite(beta) ? beta : 0.0;
        if (!isfinite(beta) || !(rho != 0.0)) a.sc[S_BAD] = 1.0;
        a.sc[S_MAXR] = m3[0];
        a.sc[S_MAXX] = m3[1];
    }
}

}  // namespace

int64_t nn_os_work_elems(int nvox) { return 8 * (int64_t)nvox + 6 * RBLK + S_NSC; }

cudaError_t nn_os_solve(const NnOs &o, cudaStream_t st, double **x_out, int *krylov_its, int *sweeps, int *status)
{
    const int n = o.nvox;
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
    double *x1 = w + n;  // second Jacobi buffer
    a.r = w + 2 * (int64_t)n;
    a.rh = w + 3 * (int64_t)n;
    a.p = w + 4 * (int64_t)n;
    a.v = w + 5 * (int64_t)n;
    a.s = w + 6 * (int64_t)n;
    a.t = w + 7 * (int64_t)n;
    a.part = w + 8 * (int64_t)n;
    a.part2 = a.part + 3 * RBLK;
    a.sc = a.part2 + 3 * RBLK;
    *status = 1;
    *krylov_its = 0;
    *sweeps = 0;
    cudaError_t e;
    auto chk = [&]() { return cudaGetLastError(); };
    double *xa = a.x, *xb = x1;
    bool start_zero = true;
    if (o.krylov) {
        k_bi_start<<<RBLK, RT_, 0, st>>>(a);
        k_bi_f0<<<1, RT_, 0, st>>>(a);
        if ((e = chk()) != cudaSuccess) return e;
        double best = INFINITY;
        int best_it = 0;
        for (int it = 1; it <= o.kmax; ++it) {
            k_bi_p<<<RBLK, RT_, 0, st>>>(a);
            k_bi_mv1<<<RBLK, RT_, 0, st>>>(a);
            k_bi_f1<<<1, RT_, 0, st>>>(a);
            k_bi_s<<<RBLK, RT_, 0, st>>>(a);
            k_bi_mv2<<<RBLK, RT_, 0, st>>>(a);
            k_bi_f2<<<1, RT_, 0, st>>>(a);
            k_bi_xr<<<RBLK, RT_, 0, st>>>(a);
            k_bi_f3<<<1, RT_, 0, st>>>(a);
            if ((e = chk()) != cudaSuccess) return e;
            *krylov_its = it;
            if (it % 4 != 0 && it != o.kmax) continue;
            double sc[S_NSC];
            if ((e = cudaMemcpyAsync(sc, a.sc, sizeof(sc), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
            const double mr = sc[S_MAXR], mx = sc[S_MAXX];
            if (!std::isfinite(mr) || !std::isfinite(mx)) break;  // restart the sweeps from zero
            start_zero = false;
            if (!(mr > o.jtol * mx)) break;  // the sweeps confirm it
            if (sc[S_BAD] != 0.0) break;     // breakdown: the sweeps go on from x
            if (mr < 0.5 * best) {
                best = mr;
                best_it = it;
            } else if (it - best_it >= 64) {
                break;  // stagnation
            }
        }
    }
    if (start_zero && (e = cudaMemsetAsync(xa, 0, sizeof(double) * n, st)) != cudaSuccess) return e;
    // Jacobi sweeps to a change <= jtol max |x| (the criterion of the plain iteration), checked on the
    // last sweep of each batch: short batches after a Krylov start, else 4 then 16
    int m = 0;
    for (;;) {
        if ((e = cudaMemsetAsync(o.mx, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess) return e;
        const int batch = (o.krylov && !start_zero) ? (m < 8 ? 2 : 8) : (m < 16 ? 4 : 16);
        for (int q = 0; q < batch; ++q) {
            if ((e = nn_jacobi(n, o.sph, o.n1, o.n2, o.n3, o.L27, o.eps, o.y, xa, xb, q == batch - 1 ? o.mx : nullptr,
                               st)) != cudaSuccess)
                return e;
            std::swap(xa, xb);
            ++m;
        }
        unsigned long long h[2];
        if ((e = cudaMemcpyAsync(h, o.mx, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        double dmax, xmax;
        std::memcpy(&dmax, &h[0], sizeof(double));
        std::memcpy(&xmax, &h[1], sizeof(double));
        if (!std::isfinite(dmax) || !std::isfinite(xmax)) {
            *status = 2;
            break;
        }
        if (!(dmax > o.jtol * xmax)) {
            *status = 0;
            break;
        }
        if (m >= o.jmax) break;
    }
    *sweeps = m;
    *x_out = xa;
    return cudaSuccess;
}

}  // namespace rtk
