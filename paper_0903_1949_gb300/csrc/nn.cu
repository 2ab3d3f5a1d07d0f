// nn.cu -- nearest-neighbour approximate Lambda operator (3^3 neighbour voxels
// built exactly, Sect. 2 and 3.2.1) and its operator-splitting step.
//
// L27[q nvox + v] = dJ_v / dS_u for the voxel u at offset (q/9 - 1, (q/3)%3 - 1,
// q%3 - 1) of v in (i, j, k), the phi index periodic (axis 3 spherical, axis 2
// cylindrical); 27 planes of n_vox, so that the sweeps read them coalesced.  Along a characteristic I_s = E_s I_{s-1} + alpha_s S_prev +
// beta_s S_{v_s} + gamma_s S_{v_{s+1}}, so the derivatives d_u = dI_s/dS_u obey
// d_u <- E_s d_u + (the weight of S_u in segment s's increment).  One thread
// per characteristic carries d_u for the NNW most recently touched voxels (the
// least recently touched makes room when the window is full) and emits, per segment,
// c_s d_u with u's neighbour slot of v_s (c_s = w_Omega l_s / L_{Omega v_s});
// one thread per voxel sums them over its ownership list in list order.  The
// OS step (I - (1-eps) L*) x = y is solved in nn_krylov.cu.  All FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "coef.cuh"
#include "rt_internal.h"

namespace rtk {
namespace {

constexpr int NNW = RTK_NNW;

struct Ijk {
    int i, j, k;
};

__device__ __forceinline__ Ijk decode(int v, int n2, int n3)
{
    Ijk r;
    r.k = v % n3;
    r.j = (v / n3) % n2;
    r.i = v / (n2 * n3);
    return r;
}

// neighbour slot of b in a's 3x3x3 neighbourhood, or -1
__device__ __forceinline__ int slot_of(const Ijk &a, const Ijk &b, int sph, int n2, int n3)
{
    int d0 = b.i - a.i, d1 = b.j - a.j, d2 = b.k - a.k;
    if (sph) {
        if (d2 == n3 - 1) d2 = -1;
        else if (d2 == 1 - n3) d2 = 1;
    } else {
        if (d1 == n2 - 1) d1 = -1;
        else if (d1 == 1 - n2) d1 = 1;
    }
    if (d0 < -1 || d0 > 1 || d1 < -1 || d1 > 1 || d2 < -1 || d2 > 1) return -1;
    return (d0 + 1) * 9 + (d1 + 1) * 3 + (d2 + 1);
}

struct Window {
    int vox[NNW];
    Ijk ijk[NNW];
    double d[NNW];
    int t[NNW];  // segment count at the last touch
};

// d_u += val for voxel u at touch time now (inserted when absent; a full window
// gives up its least recently touched entry, the one farthest back along the
// characteristic)
__device__ __forceinline__ void win_add(Window &W, int u, double val, int now, int n2, int n3)
{
    int hit = -1, empty = -1, old = 0;
    int tmin = 0;
#pragma unroll
    for (int e = 0; e < NNW; ++e) {
        if (W.vox[e] == u) hit = e;
        if (empty < 0 && W.vox[e] < 0) empty = e;
        if (e == 0 || W.t[e] < tmin) {
            tmin = W.t[e];
            old = e;
        }
    }
    const int tgt = hit >= 0 ? hit : (empty >= 0 ? empty : old);
    const Ijk c = decode(u, n2, n3);
#pragma unroll
    for (int e = 0; e < NNW; ++e) {
        if (e == tgt) {
            if (hit >= 0) {
                W.d[e] += val;
            } else {
                W.vox[e] = u;
                W.ijk[e] = c;
                W.d[e] = val;
            }
            W.t[e] = now;
        }
    }
}

__global__ void __launch_bounds__(128) k_nn_walk(NnWalk a)
{
    const int64_t r = a.r_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= a.r_hi) return;
    const int64_t s0 = a.ray_off[r], s1 = a.ray_off[r + 1];
    const int ang = a.ray_angle[r];
    const double wq = a.wt[ang];
    const double *invLq = a.invL + (int64_t)ang * a.nvox;
    Window W;
#pragma unroll
    for (int e = 0; e < NNW; ++e) {
        W.vox[e] = -1;
        W.d[e] = 0.0;
        W.ijk[e] = Ijk{0, 0, 0};
        W.t[e] = -1;
    }
    int now = 0;
    int vprev = -1;
    for (int64_t s = s0; s < s1; ++s) {
        const uint32_t w = a.vox[s];
        const int v = (int)(w & RTK_VOXMASK);
        const bool para = a.pbits ? ((a.pbits[s >> 5] >> (s & 31)) & 1u) != 0u : (w & RTK_PARA) != 0u;
        const bool run0 = (w & (RTK_RAYSTART | RTK_RESTART)) != 0u;
        const double x = a.chi[v] * a.len64[s];
        int vn = -1;
        double p = 0.0;
        if (para) {
            vn = (int)(a.vox[s + 1] & RTK_VOXMASK);
            p = a.chi[vn] * a.len64[s + 1];
        }
        double E, al, be, ga;
        Coef64::eval(x, p, para, E, al, be, ga);
#pragma unroll
        for (int e = 0; e < NNW; ++e) W.d[e] *= E;
        ++now;
        if (run0) {
            win_add(W, v, al + be, now, a.n2, a.n3);  // S_0 := S_1 at the start of a run
        } else {
            win_add(W, vprev, al, now, a.n2, a.n3);
            win_add(W, v, be, now, a.n2, a.n3);
        }
        if (para) win_add(W, vn, ga, now, a.n2, a.n3);
        const double c = wq * a.len64[s] * invLq[v];
        const Ijk cv = decode(v, a.n2, a.n3);
        const int64_t o = (s - a.seg_lo) * NNW;
        // the segment's 16 slots as one 16-byte store, its 16 values as eight
        unsigned sw[4] = {0u, 0u, 0u, 0u};
        double2 *vo = reinterpret_cast<double2 *>(a.val + o);
#pragma unroll
        for (int e = 0; e < NNW; e += 2) {
            const int q0 = W.vox[e] >= 0 ? slot_of(cv, W.ijk[e], a.sph, a.n2, a.n3) : -1;
            const int q1 = W.vox[e + 1] >= 0 ? slot_of(cv, W.ijk[e + 1], a.sph, a.n2, a.n3) : -1;
            sw[e >> 2] |= ((unsigned)(uint8_t)(int8_t)q0) << (8 * (e & 3));
            sw[(e + 1) >> 2] |= ((unsigned)(uint8_t)(int8_t)q1) << (8 * ((e + 1) & 3));
            vo[e >> 1] = make_double2(q0 >= 0 ? c * W.d[e] : 0.0, q1 >= 0 ? c * W.d[e + 1] : 0.0);
        }
        *reinterpret_cast<uint4 *>(a.slot + o) = make_uint4(sw[0], sw[1], sw[2], sw[3]);
        vprev = v;
    }
}

// L27 rows of one block by gather work units (at most a fixed number of
// consecutive entries of one voxel's ownership list each, so that the outer
// voxels crossed by thousands of characteristics do not hold up the launch):
// one thread per unit sums its entries in list order, window slots in order.
// A voxel with one unit is finished here; the units of a longer list leave
// their 27 sums in part for k_nn_gather_rows.
__global__ void __launch_bounds__(128) k_nn_gather_units(int nvox, int64_t nunits, const int32_t *urow,
                                                         const int32_t *ubeg, const int32_t *off, const int32_t *perm,
                                                         const int8_t *slot, const double *val, double *part,
                                                         double *L27, int first)
{
    __shared__ double acc[27][128];
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
#pragma unroll
    for (int q = 0; q < 27; ++q) acc[q][threadIdx.x] = 0.0;
    if (u >= nunits) return;
    const int v = urow[u];
    const bool next_same = u + 1 < nunits && urow[u + 1] == v;
    const bool single = (u == 0 || urow[u - 1] != v) && !next_same;
    const int e1 = next_same ? ubeg[u + 1] : off[v + 1];
    for (int e = ubeg[u]; e < e1; ++e) {
        const int64_t o = (int64_t)perm[e] * NNW;
        // one 16-byte load of the 16 slots, eight of the values
        const uint4 sq = *reinterpret_cast<const uint4 *>(slot + o);
        const unsigned sw[4] = {sq.x, sq.y, sq.z, sq.w};
        const double2 *vi = reinterpret_cast<const double2 *>(val + o);
#pragma unroll
        for (int h = 0; h < NNW / 2; ++h) {
            const double2 d = vi[h];
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const int k = 2 * h + w;
                const int q = (int)(int8_t)(uint8_t)(sw[k >> 2] >> (8 * (k & 3)));
                if (q >= 0) acc[q][threadIdx.x] += w ? d.y : d.x;
            }
        }
    }
    if (single) {
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            double *e = L27 + (int64_t)q * nvox + v;  // slot planes: coalesced over v
            *e = first ? acc[q][threadIdx.x] : *e + acc[q][threadIdx.x];
        }
    } else {
#pragma unroll
        for (int q = 0; q < 27; ++q) part[27 * u + q] = acc[q][threadIdx.x];
    }
}

// One thread per voxel with several units: their sums added in unit order.
__global__ void k_nn_gather_rows(int nvox, int nmulti, const int32_t *multi, const int64_t *ufirst,
                                 const double *part, double *L27, int first)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nmulti) return;
    const int v = multi[i];
    const int64_t u0 = ufirst[v], u1 = ufirst[v + 1];
    for (int q = 0; q < 27; ++q) {
        double a = 0.0;
        for (int64_t u = u0; u < u1; ++u) a += part[27 * u + q];
        double *e = L27 + (int64_t)q * nvox + v;
        *e = first ? a : *e + a;
    }
}

__global__ void k_nn_diag(int nvox, const double *L27, double *L)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nvox) L[v] = L27[13 * (int64_t)nvox + v];
}

__device__ __forceinline__ void max_to(double x, unsigned long long *dst)
{
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dst, (unsigned long long)__double_as_longlong(x));
}

// rows[27 v + q] = planes[q nvox + v]
__global__ void k_nn_rows(int nvox, const double *planes, double *rows)
{
    const int64_t n = 27 * (int64_t)nvox;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / 27, q = e - 27 * v;
        rows[e] = planes[q * nvox + v];
    }
}

// y = (1-eps) J + eps B - S   (ALI step, and the residual of the refinement)
__global__ void k_nn_rhs(int n, const double *S, const double *J, const double *eps, const double *B, double *y)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) y[v] = (1.0 - eps[v]) * J[v] + eps[v] * B[v] - S[v];
}

// y = (1-eps) Jd + r - d   (correction sweep of the refinement)
__global__ void k_nn_rhs_corr(int n, const double *d, const double *Jd, const double *r, const double *eps, double *y)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) y[v] = (1.0 - eps[v]) * Jd[v] + r[v] - d[v];
}

// target += x (when target is not NULL); maxrel of |x| / |ref + target_new| (ref may be NULL)
__global__ void k_nn_apply(int n, double *target, const double *x, const double *ref, double *slot,
                           unsigned long long *maxrel)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    double rel = 0.0;
    if (v < n) {
        const double xv = x[v];
        double t = xv;
        if (target) {
            t = target[v] + xv;
            target[v] = t;
            if (slot) slot[v] = t;
        }
        const double den = (ref ? ref[v] : 0.0) + t;
        rel = fabs(xv) / fabs(den);
    }
    max_to(rel, maxrel);
}

unsigned nb(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t nn_walk(const NnWalk &a, cudaStream_t st)
{
    if (a.r_hi <= a.r_lo) return cudaSuccess;
    k_nn_walk<<<nb(a.r_hi - a.r_lo, 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t nn_gather(int nvox, const int32_t *off, const int32_t *perm, const int8_t *slot, const double *val,
                      const NnUnits &un, double *part, double *L27, int first, cudaStream_t st)
{
    if (un.nunits > 0)
        k_nn_gather_units<<<(unsigned)((un.nunits + 127) / 128), 128, 0, st>>>(nvox, un.nunits, un.urow, un.ubeg, off, perm,
                                                                              slot, val, part, L27, first);
    if (un.nmulti > 0)
        k_nn_gather_rows<<<(unsigned)((un.nmulti + 127) / 128), 128, 0, st>>>(nvox, (int)un.nmulti, un.multi, un.ufirst,
                                                                             part, L27, first);
    return cudaGetLastError();
}

cudaError_t nn_diag(int nvox, const double *L27, double *L, cudaStream_t st)
{
    k_nn_diag<<<nb(nvox, 256), 256, 0, st>>>(nvox, L27, L);
    return cudaGetLastError();
}

cudaError_t nn_rows(int nvox, const double *planes, double *rows, cudaStream_t st)
{
    k_nn_rows<<<152 * 8, 256, 0, st>>>(nvox, planes, rows);
    return cudaGetLastError();
}

cudaError_t nn_rhs(int n, const double *S, const double *J, const double *eps, const double *B, double *y,
                   cudaStream_t st)
{
    k_nn_rhs<<<nb(n, 256), 256, 0, st>>>(n, S, J, eps, B, y);
    return cudaGetLastError();
}

cudaError_t nn_rhs_corr(int n, const double *d, const double *Jd, const double *r, const double *eps, double *y,
                        cudaStream_t st)
{
    k_nn_rhs_corr<<<nb(n, 256), 256, 0, st>>>(n, d, Jd, r, eps, y);
    return cudaGetLastError();
}

cudaError_t nn_apply(int n, double *target, const double *x, const double *ref, double *slot,
                     unsigned long long *maxrel, cudaStream_t st)
{
    k_nn_apply<<<nb(n, 256), 256, 0, st>>>(n, target, x, ref, slot, maxrel);
    return cudaGetLastError();
}

}  // namespace rtk
