// adjoint.cu -- gradients of the converged source function, the mean
// intensity and the flux with respect to per-voxel chi, eps and B.
//
// The converged S solves R(S) = S - (1 - eps) J(S; chi, B) - eps B = 0 with
// J = Lambda(chi) S + J_bc(chi, B) (formal solution, Sect. 2; ALI, Sect.
// 3.2.1).  For a loss L(S, J, F):
//   adjoint ALI     (I - Lambda^T diag(1-eps)) lam = gS + Lambda^T gJ + Lambda_F^T gF
//   dL/dchi  = (dJ/dchi)^T (gJ + (1-eps) lam) + (dF/dchi)^T gF
//   dL/dB    = eps lam + (dJ/dB)^T (gJ + (1-eps) lam) + (dF/dB)^T gF
//   dL/deps  = lam (B - J)
// Lambda^T is the transpose of the ray march: along every characteristic the
// adjoint intensity runs backwards, It_k = a_k + E_{k+1} It_{k+1}, with a_k the
// sensitivity of the loss to I_k (path-length weight of the gather times the
// voxel's adjoint source), and each segment returns It_k times its weights
// (alpha, beta, gamma) to the voxels whose S it used.  dJ/dchi needs dI_k /
// d dtau (coefficient derivatives, coef.cuh) and the forward intensities,
// which are recomputed per angle block (a forward march) before the backward
// pass of that block.  Everything here is FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "coef.cuh"
#include "grid.h"
#include "rt_internal.h"

namespace rtk {
namespace {

constexpr int MAXB = 256;
constexpr double FOUR_PI_A = 12.566370614359172953850573533118;

__device__ __forceinline__ int64_t lb64(const int64_t *a, int64_t lo, int64_t hi, int64_t key)
{
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// FULL = false: only the S-adjoint per segment (outS).  FULL = true: the chi
// and B sensitivities per segment (outC, outB), using the forward (l I) of
// the block in fwd.
template <bool FULL>
__global__ void __launch_bounds__(256) k_adjoint(const uint32_t *__restrict__ vox, const double *__restrict__ len,
                                                 const int64_t *__restrict__ ray_off, int64_t r_lo, int64_t r_hi,
                                                 int64_t seg_lo, int64_t nseg, const double2 *__restrict__ cs,
                                                 const double *__restrict__ Bv, double I_outer, int homog,
                                                 const double *__restrict__ u, const double *__restrict__ gc,
                                                 const double *__restrict__ invL, const double *__restrict__ wt,
                                                 const double *__restrict__ dirs, const int64_t *__restrict__ ang_seg_off,
                                                 int w0, int nw, int nvox, const double *__restrict__ fwd,
                                                 double *__restrict__ outS, double *__restrict__ outC,
                                                 double *__restrict__ outB, int chunk)
{
    __shared__ int32_t soff[MAXB + 1];
    __shared__ double swt[MAXB], sdir[3 * MAXB];
    for (int q = threadIdx.x; q <= nw; q += blockDim.x) soff[q] = (int32_t)(ang_seg_off[w0 + q] - seg_lo);
    for (int q = threadIdx.x; q < nw; q += blockDim.x) swt[q] = wt[w0 + q];
    for (int q = threadIdx.x; q < 3 * nw; q += blockDim.x) sdir[q] = dirs[3 * w0 + q];
    __syncthreads();
    const unsigned FULLM = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t c_lo = wg * chunk;
    if (c_lo >= nseg) return;
    const int64_t c_hi = (c_lo + chunk < nseg) ? c_lo + chunk : nseg;
    const int64_t ra = lb64(ray_off, r_lo, r_hi, seg_lo + c_lo);
    const int64_t rb = lb64(ray_off, r_lo, r_hi, seg_lo + c_hi);
    const int s_begin = (int)(ray_off[ra] - seg_lo);
    const int s_end = (int)(ray_off[rb] - seg_lo);
    if (s_begin >= s_end) return;
    const uint32_t *vx = vox + seg_lo;
    const double *ln = len + seg_lo;
    // carries from the tile after this one (already processed)
    double It_n = 0.0, E_n = 0.0, al_n = 0.0, l_n = 0.0;
    uint32_t w_n = RTK_RAYSTART;
    const int ntile = (s_end - s_begin + 31) / 32;
    for (int t = ntile - 1; t >= 0; --t) {
        const int base = s_begin + 32 * t;
        const int s = base + lane;
        const bool valid = s < s_end;
        uint32_t w = 0;
        double l = 0.0, chi = 0.0, S = 0.0;
        if (valid) {
            w = vx[s];
            l = ln[s];
            double2 c = cs[w & RTK_VOXMASK];
            chi = c.x;
            S = c.y;
        }
        // next segment (s + 1) and previous one (s - 1)
        uint32_t wn = __shfl_down_sync(FULLM, w, 1);
        double lnx = __shfl_down_sync(FULLM, l, 1), chin = __shfl_down_sync(FULLM, chi, 1);
        double Sn = __shfl_down_sync(FULLM, S, 1);
        if (lane == 31) {
            if (valid && s + 1 < s_end) {
                wn = vx[s + 1];
                lnx = ln[s + 1];
                double2 c = cs[wn & RTK_VOXMASK];
                chin = c.x;
                Sn = c.y;
            } else {
                wn = RTK_RAYSTART;
            }
        }
        if (valid && s + 1 >= s_end) wn = RTK_RAYSTART;
        double Sp = __shfl_up_sync(FULLM, S, 1);
        if (lane == 0 && valid && s - 1 >= s_begin) Sp = cs[vx[s - 1] & RTK_VOXMASK].y;
        const bool rstart = (w & RTK_RAYSTART) != 0u;
        const bool run0 = (w & (RTK_RAYSTART | RTK_RESTART)) != 0u;
        const bool para = (w & RTK_PARA) != 0u;
        const bool last_ray = (wn & RTK_RAYSTART) != 0u;  // the characteristic ends after s
        const double x = valid ? chi * l : 1.0;
        const double p = para ? chin * lnx : 0.0;
        double E, al, be, ga, dE, dal_x, dbe_x, dga_x, dal_p, dbe_p, dga_p;
        Coef64D::eval(x, p, para, E, al, be, ga, dE, dal_x, dbe_x, dga_x, dal_p, dbe_p, dga_p);
        const double Skm = run0 ? S : Sp;
        const double Skp = para ? Sn : 0.0;
        // adjoint source of I_s: gather weight wt_q l / L_qv times the voxel's adjoint
        double a = 0.0;
        int q = 0;
        if (valid) {
            int lo = 0, hi = nw;
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (soff[mid] <= s) lo = mid;
                else hi = mid;
            }
            q = lo;
            const int v = w & RTK_VOXMASK;
            double ueff = u ? u[v] : 0.0;
            if (gc)
                ueff += FOUR_PI_A * (sdir[3 * q] * gc[3 * (int64_t)v] + sdir[3 * q + 1] * gc[3 * (int64_t)v + 1] +
                                     sdir[3 * q + 2] * gc[3 * (int64_t)v + 2]);
            a = swt[q] * l * invL[(int64_t)(w0 + q) * nvox + v] * ueff;
        }
        // It_s = a_s + m_s It_{s+1}, m_s = E_{s+1} unless the characteristic ends at s
        double En = __shfl_down_sync(FULLM, E, 1);
        if (lane == 31) En = E_n;
        double M = (valid && !last_ray) ? En : 0.0;
        double Bc = valid ? a : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double Mo = __shfl_down_sync(FULLM, M, o);
            double Bo = __shfl_down_sync(FULLM, Bc, o);
            if (lane + o < 32) {
                Bc = M * Bo + Bc;
                M = M * Mo;
            }
        }
        const double It = M * It_n + Bc;
        double Itn = __shfl_down_sync(FULLM, It, 1);
        double aln = __shfl_down_sync(FULLM, al, 1);
        if (lane == 31) {
            Itn = It_n;
            aln = al_n;
        }
        const bool next_run0 = (wn & (RTK_RAYSTART | RTK_RESTART)) != 0u;
        // contributions handed to the next segment's voxel: gamma (S_{s+1}) and
        // dI_s/d dtau_{s+1} (the next segment's optical depth)
        const double toS = ga * It;
        double dIdp = 0.0;
        if (FULL && para) dIdp = dal_p * Skm + dbe_p * S + dga_p * Skp;
        double toSp = __shfl_up_sync(FULLM, toS, 1);
        double dIdpp = __shfl_up_sync(FULLM, dIdp * It, 1);
        if (lane == 0) {
            toSp = 0.0;  // added by lane 31 of the tile before this one
            dIdpp = 0.0;
        }
        if (!FULL) {
            double tS = It * (be + (run0 ? al : 0.0)) + toSp;
            if (!last_ray && !next_run0) tS += aln * Itn;
            if (valid) outS[s] = tS;
        } else {
            // forward intensity entering segment s (I_{s-1}, or the boundary value)
            double Ip = __shfl_up_sync(FULLM, valid ? fwd[s] : 0.0, 1);
            if (lane == 0 && valid && !rstart) Ip = fwd[s - 1];
            const double Iin = rstart ? (homog ? 0.0 : ((w & RTK_CORE) ? Bv[w & RTK_VOXMASK] : I_outer)) : Ip;
            const double dIdx = dE * Iin + dal_x * Skm + dbe_x * S + dga_x * Skp;
            if (valid) {
                outC[s] = l * (It * dIdx + dIdpp);
                outB[s] = (rstart && (w & RTK_CORE) && !homog) ? E * It : 0.0;
            }
        }
        __syncwarp();
        // lane 31 of this tile completes the first segment of the tile after it
        if (lane == 31 && valid && !last_ray) {
            const int sn = base + 32;
            if (sn < s_end) {
                if (!FULL) outS[sn] += toS;
                else outC[sn] += l_n * (dIdp * It);
            }
        }
        __syncwarp();
        It_n = __shfl_sync(FULLM, It, 0);
        E_n = __shfl_sync(FULLM, E, 0);
        al_n = __shfl_sync(FULLM, al, 0);
        l_n = __shfl_sync(FULLM, l, 0);
        w_n = __shfl_sync(FULLM, w, 0);
    }
    (void)w_n;
}

// Per-voxel sums of per-segment values over one block's ownership lists
// (first = 1 overwrites the outputs).
__global__ void k_adj_gather(int nvox, const int32_t *off, const int32_t *perm, const double *a, const double *b,
                             double *oa, double *ob, int first)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    double sa = 0.0, sb = 0.0;
    for (int e = off[v]; e < off[v + 1]; ++e) {
        const int s = perm[e];
        sa += a[s];
        if (b) sb += b[s];
    }
    oa[v] = first ? sa : oa[v] + sa;
    if (ob) ob[v] = first ? sb : ob[v] + sb;
}

// Flux adjoint from the local basis (r, theta, phi) or (R, phi, z) to Cartesian.
__global__ void k_flux_T(GeomDev G, const double *gF, double *gc)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G.nvox) return;
    int k = v % G.n3, j = (v / G.n3) % G.n2;
    double e[3][3];
    if (G.coord == RT_SPHERICAL) {
        double st = G.stm[j], ct = G.ctm[j], c = G.cpm[k], s = G.spm[k];
        e[0][0] = st * c; e[0][1] = st * s; e[0][2] = ct;
        e[1][0] = ct * c; e[1][1] = ct * s; e[1][2] = -st;
        e[2][0] = -s; e[2][1] = c; e[2][2] = 0.0;
    } else {
        double c = G.cpm[j], s = G.spm[j];
        e[0][0] = c; e[0][1] = s; e[0][2] = 0.0;
        e[1][0] = -s; e[1][1] = c; e[1][2] = 0.0;
        e[2][0] = 0.0; e[2][1] = 0.0; e[2][2] = 1.0;
    }
    const double *g = gF + 3 * (int64_t)v;
    for (int a = 0; a < 3; ++a) gc[3 * (int64_t)v + a] = e[0][a] * g[0] + e[1][a] * g[1] + e[2][a] * g[2];
}

__global__ void k_adj_prep(int n, const double *eps, const double *lam, double *out)  // (1 - eps) lam
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) out[v] = (1.0 - eps[v]) * lam[v];
}

__global__ void k_adj_ali(int n, double *lam, const double *gbar, const double *y, const double *eps, const double *L,
                          unsigned long long *maxd, unsigned long long *maxl)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0, m = 0.0;
    if (v < n) {
        const double e = eps[v];
        const double ln = lam[v] + (gbar[v] + y[v] - lam[v]) / (1.0 - (1.0 - e) * L[v]);
        d = fabs(ln - lam[v]);
        m = fabs(ln);
        lam[v] = ln;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxd, (unsigned long long)__double_as_longlong(d));
        atomicMax(maxl, (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void k_adj_final(int n, const double *lam, const double *eps, const double *B, const double *J,
                            const double *dBc, double *dB, double *deps)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        dB[v] = eps[v] * lam[v] + dBc[v];
        deps[v] = lam[v] * (B[v] - J[v]);
    }
}

// Transpose of the nearest-neighbour operator with the (1 - eps) factor of its
// columns moved in: T[q][v] = L27[26 - q][u_q] (1 - eps[u_q]), u_q the voxel at
// slot q of v (v sits at slot 26 - q of u_q: the offsets are opposite, phi
// periodic), so that sum_q T[q][v] x[u_q] = ((Lambda*_NN)^T diag(1 - eps) x)_v,
// the preconditioner of the adjoint iteration in the form the OS-step solver
// takes (with eps = 0 there).
__global__ void k_nn_transpose(int nvox, int sph, int n1, int n2, int n3, const double *L27, const double *eps,
                               double *T)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const int i0 = v / (n2 * n3), j0 = (v / n3) % n2, k0 = v % n3;
    for (int q = 0; q < 27; ++q) {
        int i = i0 + q / 9 - 1, j = j0 + (q / 3) % 3 - 1, k = k0 + q % 3 - 1;
        if (sph) k = (k < 0) ? k + n3 : ((k >= n3) ? k - n3 : k);
        else j = (j < 0) ? j + n2 : ((j >= n2) ? j - n2 : j);
        double t = 0.0;
        if (i >= 0 && i < n1 && j >= 0 && j < n2 && k >= 0 && k < n3) {
            const int u = (i * n2 + j) * n3 + k;
            t = L27[(int64_t)(26 - q) * nvox + u] * (1.0 - eps[u]);
        }
        T[(int64_t)q * nvox + v] = t;
    }
}

// r = gbar + y - lam  (residual of the adjoint fixed point)
__global__ void k_adj_res(int n, const double *gbar, const double *y, const double *lam, double *r)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) r[v] = gbar[v] + y[v] - lam[v];
}

// lam += x; maxd <- max |x|, maxl <- max |lam|
__global__ void k_adj_add(int n, double *lam, const double *x, unsigned long long *maxd, unsigned long long *maxl)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0, m = 0.0;
    if (v < n) {
        const double ln = lam[v] + x[v];
        d = fabs(x[v]);
        m = fabs(ln);
        lam[v] = ln;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxd, (unsigned long long)__double_as_longlong(d));
        atomicMax(maxl, (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void k_axpy(int n, const double *x, double *y)  // y += x
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) y[v] += x[v];
}

}  // namespace
}  // namespace rtk

using namespace rtk;

namespace {

int afail(int code, const std::string &m)
{
    set_last_error(m.c_str());
    return code;
}

#define ACK(...)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (__VA_ARGS__);                                                                   \
        if (e_ != cudaSuccess) return afail(RT_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Tmp {
    std::vector<void *> p;
    ~Tmp()
    {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    T *get(size_t n)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return (T *)q;
    }
};

// Lambda^T-type pass over all blocks.  FULL: chi / B sensitivities (needs a
// forward march per block into the grid's segment buffer).
int adjoint_pass(rt_grid *g, bool full, int homog, const double *u, const double *gc, double *tS, double *tC,
                 double *tB, double *oS, double *oC, double *oB)
{
    const int n = g->nvox;
    ACK(pack_chiS64(n, g->d_chi, g->d_S, g->d_cs64, g->st));
    for (int b = 0; b < g->nblk; ++b) {
        const int w0 = g->blk_w0[b], nw = g->blk_nw[b];
        const int64_t r_lo = g->h_ang_ray_off[w0], r_hi = g->h_ang_ray_off[w0 + nw];
        const int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
        const int32_t *off = g->d_csr_off + (size_t)b * (n + 1);
        const int chunk = 512;
        const int64_t blocks = ((ns + chunk - 1) / chunk + 7) / 8;
        if (ns <= 0) continue;
        if (full) {
            ACK(march_block_I(g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs64, g->d_B, g->I_outer,
                              homog, (double *)g->d_segbuf, g->march_chunk, g->st));
            k_adjoint<true><<<(unsigned)blocks, 256, 0, g->st>>>(
                g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs64, g->d_B, g->I_outer, homog, u, gc,
                g->d_invL, g->d_wt, g->d_dirs, g->d_ang_seg_off, w0, nw, n, (const double *)g->d_segbuf, nullptr, tC,
                tB, chunk);
            ACK(cudaGetLastError());
            k_adj_gather<<<(n + 255) / 256, 256, 0, g->st>>>(n, off, g->d_perm + lo, tC, tB, oC, oB, b == 0);
        } else {
            k_adjoint<false><<<(unsigned)blocks, 256, 0, g->st>>>(
                g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs64, g->d_B, g->I_outer, homog, u, gc,
                g->d_invL, g->d_wt, g->d_dirs, g->d_ang_seg_off, w0, nw, n, nullptr, tS, nullptr, nullptr, chunk);
            ACK(cudaGetLastError());
            k_adj_gather<<<(n + 255) / 256, 256, 0, g->st>>>(n, off, g->d_perm + lo, tS, nullptr, oS, nullptr, b == 0);
        }
        ACK(cudaGetLastError());
    }
    return RT_OK;
}

}  // namespace

extern "C" int rt_adjoint(rt_grid *g, const double *dL_dS, const double *dL_dJ, const double *dL_dF, double tol,
                          int max_iter, double *dchi, double *deps, double *dB, int where, int *iters)
{
    if (!g || !dchi || !deps || !dB) return afail(RT_EINVAL, "NULL argument");
    if (where != RT_HOST && where != RT_DEVICE) return afail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    if (!(tol > 0.0) || max_iter < 1) return afail(RT_EINVAL, "need tol > 0 and max_iter >= 1");
    if (g->lost) return afail(RT_EDEVICE, "the grid has characteristics that could not be tracked");
    if (!g->use_lstar) return afail(RT_EINVAL, "the adjoint iteration needs use_lstar = 1");
    ACK(cudaSetDevice(g->device));
    const int n = g->nvox;
    const cudaMemcpyKind kin = where == RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    Tmp tmp;
    double *gS = tmp.get<double>(n), *gJ = tmp.get<double>(n), *gF = tmp.get<double>(3 * (size_t)n);
    double *gc = tmp.get<double>(3 * (size_t)n), *gbar = tmp.get<double>(n), *lam = tmp.get<double>(n);
    double *y = tmp.get<double>(n), *v1 = tmp.get<double>(n), *oC = tmp.get<double>(n), *oB = tmp.get<double>(n);
    double *tS = tmp.get<double>(g->max_blk_seg), *tC = tmp.get<double>(g->max_blk_seg);
    double *tB = tmp.get<double>(g->max_blk_seg), *dBd = tmp.get<double>(n), *ded = tmp.get<double>(n);
    unsigned long long *mx = tmp.get<unsigned long long>(2);
    if (!gS || !gJ || !gF || !gc || !gbar || !lam || !y || !v1 || !oC || !oB || !tS || !tC || !tB || !dBd || !ded || !mx)
        return afail(RT_ENOMEM, "adjoint work arrays could not be allocated");
    if (dL_dS) ACK(cudaMemcpyAsync(gS, dL_dS, sizeof(double) * n, kin, g->st));
    else ACK(cudaMemsetAsync(gS, 0, sizeof(double) * n, g->st));
    if (dL_dJ) ACK(cudaMemcpyAsync(gJ, dL_dJ, sizeof(double) * n, kin, g->st));
    else ACK(cudaMemsetAsync(gJ, 0, sizeof(double) * n, g->st));
    if (dL_dF) {
        ACK(cudaMemcpyAsync(gF, dL_dF, sizeof(double) * 3 * n, kin, g->st));
        k_flux_T<<<(n + 255) / 256, 256, 0, g->st>>>(g->G, gF, gc);
        ACK(cudaGetLastError());
    }
    // J and the FP64 Lambda* at the current S
    int rc = rt_formal_solution_ex(g, RT_FP64, 0);
    if (rc != RT_OK) return rc;
    // gbar = gS + Lambda^T gJ + Lambda_F^T gF
    rc = adjoint_pass(g, false, 1, gJ, dL_dF ? gc : nullptr, tS, nullptr, nullptr, y, nullptr, nullptr);
    if (rc != RT_OK) return rc;
    ACK(cudaMemcpyAsync(gbar, gS, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->st));
    k_axpy<<<(n + 255) / 256, 256, 0, g->st>>>(n, y, gbar);
    ACK(cudaMemcpyAsync(lam, gbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->st));
    // adjoint ALI: lam <- lam + M^-1 (gbar + Lambda^T((1-eps) lam) - lam), M = 1 - (1-eps) Lambda*
    // (diagonal), or M = I - (Lambda*_NN)^T diag(1-eps) solved like the forward OS step
    const bool nn = g->use_lstar == RT_LSTAR_NN;
    double *T27 = nullptr, *zeros = nullptr, *r = nullptr;
    if (nn) {
        rc = rt_grid_build_nn(g);
        if (rc != RT_OK) return rc;
        T27 = tmp.get<double>(27 * (size_t)n);
        zeros = tmp.get<double>(n);
        r = tmp.get<double>(n);
        if (!T27 || !zeros || !r) return afail(RT_ENOMEM, "adjoint NN work arrays could not be allocated");
        ACK(cudaMemsetAsync(zeros, 0, sizeof(double) * n, g->st));
        k_nn_transpose<<<(n + 127) / 128, 128, 0, g->st>>>(n, g->coord == RT_SPHERICAL, g->n1, g->n2, g->n3,
                                                           g->d_L27, g->d_eps, T27);
        ACK(cudaGetLastError());
    }
    int it = 0;
    bool conv = false;
    for (it = 1; it <= max_iter; ++it) {
        k_adj_prep<<<(n + 255) / 256, 256, 0, g->st>>>(n, g->d_eps, lam, v1);
        rc = adjoint_pass(g, false, 1, v1, nullptr, tS, nullptr, nullptr, y, nullptr, nullptr);
        if (rc != RT_OK) return rc;
        ACK(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), g->st));
        if (nn) {
            k_adj_res<<<(n + 255) / 256, 256, 0, g->st>>>(n, gbar, y, lam, r);
            NnOs o{};
            o.nvox = n;
            o.sph = g->coord == RT_SPHERICAL;
            o.n1 = g->n1;
            o.n2 = g->n2;
            o.n3 = g->n3;
            o.L27 = T27;
            o.eps = zeros;
            o.y = r;
            o.work = g->d_nnx;
            o.jtol = g->nn_jtol;
            o.jmax = g->nn_jmax;
            o.krylov = g->nn_krylov;
            o.kmax = 1000;
            double *x = nullptr;
            int kits = 0, sweeps = 0, status = 0;
            ACK(nn_os_solve(o, g->st, &x, &kits, &sweeps, &status));
            ++g->launches;
            if (status == 3) return afail(RT_ETIMEOUT, "adjoint NN OS step: a grid-barrier wait gave up");
            if (status == 2) return afail(RT_EDEVICE, "adjoint NN OS step diverged");
            if (status == 1) return afail(RT_ENOTCONVERGED, "adjoint NN OS step did not converge");
            ACK(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), g->st));
            k_adj_add<<<(n + 255) / 256, 256, 0, g->st>>>(n, lam, x, mx, mx + 1);
        } else {
            k_adj_ali<<<(n + 255) / 256, 256, 0, g->st>>>(n, lam, gbar, y, g->d_eps, g->d_L, mx, mx + 1);
        }
        unsigned long long h[2];
        ACK(cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, g->st));
        ACK(cudaStreamSynchronize(g->st));
        double dmax, lmax;
        std::memcpy(&dmax, &h[0], sizeof(double));
        std::memcpy(&lmax, &h[1], sizeof(double));
        if (!std::isfinite(dmax) || !std::isfinite(lmax))
            return afail(RT_EDEVICE, "adjoint ALI produced a non-finite iterate");
        if (!(dmax > tol * lmax)) {
            conv = true;
            break;
        }
    }
    if (iters) *iters = conv ? it : max_iter;
    // sensitivities to chi and to B through the core, with u = gJ + (1-eps) lam
    k_adj_prep<<<(n + 255) / 256, 256, 0, g->st>>>(n, g->d_eps, lam, v1);
    k_axpy<<<(n + 255) / 256, 256, 0, g->st>>>(n, gJ, v1);
    rc = adjoint_pass(g, true, 0, v1, dL_dF ? gc : nullptr, nullptr, tC, tB, nullptr, oC, oB);
    if (rc != RT_OK) return rc;
    k_adj_final<<<(n + 255) / 256, 256, 0, g->st>>>(n, lam, g->d_eps, g->d_B, g->d_J, oB, dBd, ded);
    ACK(cudaGetLastError());
    const cudaMemcpyKind kout = where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    ACK(cudaMemcpyAsync(dchi, oC, sizeof(double) * n, kout, g->st));
    ACK(cudaMemcpyAsync(deps, ded, sizeof(double) * n, kout, g->st));
    ACK(cudaMemcpyAsync(dB, dBd, sizeof(double) * n, kout, g->st));
    ACK(cudaStreamSynchronize(g->st));
    if (!conv) return afail(RT_ENOTCONVERGED, "adjoint ALI did not reach tol in max_iter iterations");
    return RT_OK;
}
