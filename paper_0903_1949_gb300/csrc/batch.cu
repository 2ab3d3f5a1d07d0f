// batch.cu -- many opacity fields (wavelengths of a line profile, or models)
// solved together on one or more grids of uneven size (the paper distributes
// wavelengths over MPI "clusters", Sect. 3.2.2; here they share one GPU).
//
// Every member m has its own chi, eps, B, S, J and Lambda* and its own
// parabola choices (a bit per crossing segment, from its chi in FP64); the
// crossing lists and ownership lists are those of the member's grid.  One
// ALI iteration of all members is: pack (chi, S) in FP32, then for each wave
// k (angle block k of every member that has one) a persistent FP32 J-only
// march over the bundles of all the wave's items and a persistent J gather
// over their lists, then the FP64 ALI update of every member.  Each member
// appears at most once per wave, so its J accumulates over its angle blocks
// in a fixed order.  The whole iteration is captured once as a CUDA graph and
// replayed; rt_batch_autotune picks the bundle size and the persistent grid.
//
// A two-level-atom line problem (rt_line_*) is a batch whose members are the
// frequencies of one grid: each iteration sets S_k from the line source
// function S_l, solves the n_freq formal solutions and updates S_l from
// Jbar = sum_k w_k phi_k J_k with the frequency-averaged diagonal Lambda*
// (Sect. 3.1, 3.2.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "grid.h"
#include "rt_internal.h"

using namespace rtk;

namespace {

int bfail(int code, const std::string &m)
{
    set_last_error(m.c_str());
    return code;
}

#define BCK(...)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (__VA_ARGS__);                                                                  \
        if (e_ != cudaSuccess) return bfail(RT_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define BRCK(call)                  \
    do {                            \
        int r_ = (call);            \
        if (r_ != RT_OK) return r_; \
    } while (0)

__global__ void k_bpack(int64_t n, const double *chi, const double *S, const double *B, float2 *cs, float *B32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        cs[i] = make_float2((float)chi[i], (float)S[i]);
        B32[i] = (float)B[i];
    }
}

// ALI update of every member's voxels; per-member max |dS| / |S_new|.
__global__ void k_bali(int64_t n, const int64_t *voff, int nm, double *S, const double *J, const double *L,
                       const double *eps, const double *B, unsigned long long *maxrel)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nm;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (voff[mid] <= i) lo = mid;
            else hi = mid;
        }
        const double e = eps[i], s = S[i];
        const double sn = s + ((1.0 - e) * J[i] + e * B[i] - s) / (1.0 - (1.0 - e) * L[i]);
        const double rel = fabs(sn - s) / fabs(sn);
        S[i] = sn;
        atomicMax(maxrel + lo, (unsigned long long)__double_as_longlong(rel));
    }
}

// FP64 residual of the refined batch solve: r = (1-eps) J64 + eps B - S for the
// members still iterating (active[m]), 0 for the others; per member the max of
// |dS| / |S + dS| over its voxels for the ALI update dS = r / (1 - (1-eps) L).
__global__ void k_bresid(int64_t n, const int64_t *voff, int nm, const int *active, const double *S, const double *J,
                         const double *L, const double *eps, const double *B, double *R, unsigned long long *maxrel)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nm;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (voff[mid] <= i) lo = mid;
            else hi = mid;
        }
        if (!active[lo]) {
            R[i] = 0.0;
            continue;
        }
        const double e = eps[i], s = S[i];
        const double r = (1.0 - e) * J[i] + e * B[i] - s;
        R[i] = r;
        const double d = r / (1.0 - (1.0 - e) * L[i]);
        atomicMax(maxrel + lo, (unsigned long long)__double_as_longlong(fabs(d) / fabs(s + d)));
    }
}

// One FP32-march correction sweep of the refined solve for every member:
// D <- D + [(1-eps) J(D) + R - D] / (1 - (1-eps) L), J(D) the formal solution of
// D with no incoming radiation; per member the max |change| / |S + D|.
__global__ void k_bcorr(int64_t n, const int64_t *voff, int nm, double *D, const double *J, const double *R,
                        const double *L, const double *eps, const double *S, unsigned long long *maxrel)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nm;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (voff[mid] <= i) lo = mid;
            else hi = mid;
        }
        const double e = eps[i], d = D[i];
        const double dn = d + ((1.0 - e) * J[i] + R[i] - d) / (1.0 - (1.0 - e) * L[i]);
        D[i] = dn;
        atomicMax(maxrel + lo, (unsigned long long)__double_as_longlong(fabs(dn - d) / fabs(S[i] + dn)));
    }
}

__global__ void k_badd(int64_t n, double *S, const double *D)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        S[i] += D[i];
}

__global__ void k_bpack64(int64_t n, const double *chi, const double *S, double2 *cs)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cs[i] = make_double2(chi[i], S[i]);
}

// Line mode.  S_k = (chi_c B + chi_l phi_k S_l) / chi_k for every frequency k
// (members k*nvox .. (k+1)*nvox - 1 of the concatenated arrays).
__global__ void k_line_src(int nvox, int nf, const double *chi, const double *chi_c, const double *chi_l,
                           const double *B, const double *phi, const double *S_l, double *S)
{
    const int64_t n = (int64_t)nvox * nf;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / nvox), v = (int)(i % nvox);
        S[i] = (chi_c[v] * B[v] + chi_l[v] * phi[k] * S_l[v]) / chi[i];
    }
}

__global__ void k_line_chik(int nvox, const double *chi_c, const double *chi_l, double phik, double *chik)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nvox) chik[v] = fma(chi_l[v], phik, chi_c[v]);
}

// Lbar* = sum_k w_k phi_k (chi_l phi_k / chi_k) Lambda*_k
__global__ void k_line_lbar(int nvox, int nf, const double *L, const double *chi, const double *chi_l,
                            const double *phi, const double *wq, double *Lbar)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    double acc = 0.0;
    for (int k = 0; k < nf; ++k) {
        const int64_t i = (int64_t)k * nvox + v;
        acc += wq[k] * phi[k] * (chi_l[v] * phi[k] / chi[i]) * L[i];
    }
    Lbar[v] = acc;
}

// Jbar = sum_k w_k phi_k J_k (k ascending); S_l <- S_l + [(1-eps_l) Jbar + eps_l B - S_l] / (1 - (1-eps_l) Lbar*)
__global__ void k_line_update(int nvox, int nf, const double *J, const double *phi, const double *wq,
                              const double *eps_l, const double *B, const double *Lbar, double *S_l, double *Jbar,
                              unsigned long long *maxrel)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    double rel = 0.0;
    if (v < nvox) {
        double jb = 0.0;
        for (int k = 0; k < nf; ++k) jb += wq[k] * phi[k] * J[(int64_t)k * nvox + v];
        const double e = eps_l[v], s = S_l[v];
        const double sn = s + ((1.0 - e) * jb + e * B[v] - s) / (1.0 - (1.0 - e) * Lbar[v]);
        rel = fabs(sn - s) / fabs(sn);
        S_l[v] = sn;
        Jbar[v] = jb;
    }
    for (int o = 16; o > 0; o >>= 1) rel = fmax(rel, __shfl_down_sync(0xffffffffu, rel, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxrel, (unsigned long long)__double_as_longlong(rel));
}

// Nearest-neighbour line operator, frequency k's share (slot planes, [q nvox + v]):
// Lbar27[q][v] (+)= w_k phi_k L27_k[q][v] (chi_l phi_k / chi_k) at the voxel u in slot q.
__global__ void k_line_lbar_nn(int nvox, int sph, int n1, int n2, int n3, const double *L27k, const double *chi_c,
                               const double *chi_l, double phik, double wphi, double *Lbar27, int first)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const int c3 = v % n3, c2 = (v / n3) % n2, c1 = v / (n3 * n2);
    for (int q = 0; q < 27; ++q) {
        int i = c1 + q / 9 - 1, j = c2 + (q / 3) % 3 - 1, k = c3 + q % 3 - 1;
        if (sph) k = (k + n3) % n3;
        else j = (j + n2) % n2;
        double f = 0.0;
        if (i >= 0 && i < n1 && j >= 0 && j < n2 && k >= 0 && k < n3) {
            const int u = (i * n2 + j) * n3 + k;
            f = chi_l[u] * phik / fma(chi_l[u], phik, chi_c[u]);
        }
        const int64_t e = (int64_t)q * nvox + v;  // slot planes
        const double add = wphi * L27k[e] * f;
        Lbar27[e] = first ? add : Lbar27[e] + add;
    }
}

// Jbar = sum_k w_k phi_k J_k (k ascending) and the right-hand side of the
// nearest-neighbour OS step, y = (1 - eps_l) Jbar + eps_l B - S_l.
__global__ void k_line_rhs(int nvox, int nf, const double *J, const double *phi, const double *wq,
                           const double *eps_l, const double *B, const double *S_l, double *Jbar, double *y)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    double jb = 0.0;
    for (int k = 0; k < nf; ++k) jb += wq[k] * phi[k] * J[(int64_t)k * nvox + v];
    Jbar[v] = jb;
    y[v] = (1.0 - eps_l[v]) * jb + eps_l[v] * B[v] - S_l[v];
}

struct Wave {
    int n = 0;            // items
    int64_t mi0 = 0;      // first item in the concatenated item arrays
    int64_t pf0 = 0;      // first prefix entry (n + 1 per wave)
    int64_t bundles = 0;  // total march bundles
    int64_t work = 0;     // total gather work units
};

}  // namespace

struct rt_batch {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<rt_grid *> grids;
    std::vector<int> mgrid;
    std::vector<int64_t> voff;  // member voxel offsets (n_members + 1)
    std::vector<char> ready;
    int nm = 0;
    int64_t ntot = 0;
    std::vector<void *> allocs;
    double *chi = nullptr, *eps = nullptr, *B = nullptr, *S = nullptr, *J = nullptr, *L = nullptr, *Fc = nullptr;
    float2 *cs = nullptr;
    float *B32 = nullptr;
    int64_t *d_voff = nullptr;
    std::vector<uint32_t *> pbits;
    unsigned long long *maxrel = nullptr;
    std::vector<unsigned long long> h_maxrel;
    std::vector<Wave> waves;
    std::vector<MarchItem> h_mi;
    std::vector<GatherItem> h_gi;
    MarchItem *d_mi = nullptr;
    GatherItem *d_gi = nullptr;
    int64_t *d_bpfx = nullptr, *d_wpfx = nullptr;
    float *wbuf = nullptr;
    double *wpart = nullptr;
    int *wcnt = nullptr;
    unsigned long long *counters = nullptr;
    int chunk = 1024;
    int grid_march = 152 * 5, grid_gather = 152 * 5;
    cudaGraphExec_t graph = nullptr;
    // refined solve (rt_batch_solve): FP64 residual R, FP32 correction D, its graph
    double *R = nullptr, *D = nullptr;
    double2 *cs64 = nullptr;
    int *d_active = nullptr;
    cudaGraphExec_t graph_corr = nullptr;
    int refine_every = 16;
    std::vector<double> history;  // max over members of max rel dS per iteration
    // two-level line mode (rt_line_*): the members are the frequencies of one grid
    int line = 0;
    int nf = 0, lnvox = 0;
    double *chi_c = nullptr, *chi_l = nullptr, *eps_l = nullptr, *Bl = nullptr;
    double *phi = nullptr, *wq = nullptr, *S_l = nullptr, *Jbar = nullptr, *Lbar = nullptr, *ones = nullptr, *tmp = nullptr;
    std::vector<double> h_phi, h_wq;
    bool line_ready = false;
    int lstar = RT_LSTAR_DIAG;  // line operator: diagonal or nearest-neighbour
    double *Lbar27 = nullptr, *L27k = nullptr, *nnx = nullptr, *nny = nullptr;
    int nn_sweeps = 0;
    int ng = 0;  // Ng extrapolation of S_l
    double *H = nullptr, *ng_part = nullptr, *ng_coef = nullptr;
    int hs[4] = {0, 1, 2, 3}, nh = 0;
};

namespace {

template <typename T>
int balloc(rt_batch *b, T **p, size_t count)
{
    void *q = nullptr;
    size_t nbytes = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = cudaMalloc(&q, nbytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(RT_ENOMEM, "cudaMalloc of " + std::to_string(nbytes) + " bytes failed");
    }
    b->allocs.push_back(q);
    *p = (T *)q;
    return RT_OK;
}

void bfree_all(rt_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (b->graph_corr) cudaGraphExecDestroy(b->graph_corr);
    b->graph_corr = nullptr;
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    b->st = nullptr;
}

// Bundle and work-unit prefixes of every wave for the current bundle size.
int build_prefixes(rt_batch *b)
{
    std::vector<int64_t> bp, wp;
    for (Wave &w : b->waves) {
        w.pf0 = (int64_t)bp.size();
        int64_t acc_b = 0, acc_w = 0;
        bp.push_back(0);
        wp.push_back(0);
        for (int i = 0; i < w.n; ++i) {
            const MarchItem &m = b->h_mi[w.mi0 + i];
            const GatherItem &g = b->h_gi[w.mi0 + i];
            acc_b += (m.nseg + b->chunk - 1) / b->chunk;
            acc_w += g.nbs + g.nbc;
            bp.push_back(acc_b);
            wp.push_back(acc_w);
        }
        w.bundles = acc_b;
        w.work = acc_w;
    }
    if (!b->d_bpfx) {
        BRCK(balloc(b, &b->d_bpfx, bp.size()));
        BRCK(balloc(b, &b->d_wpfx, wp.size()));
    }
    BCK(cudaMemcpyAsync(b->d_bpfx, bp.data(), sizeof(int64_t) * bp.size(), cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemcpyAsync(b->d_wpfx, wp.data(), sizeof(int64_t) * wp.size(), cudaMemcpyHostToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));
    return RT_OK;
}

// The kernels of one ALI iteration of all members (captured into the graph).
int enqueue_iteration(rt_batch *b)
{
    if (b->line) {
        k_line_src<<<152 * 8, 256, 0, b->st>>>(b->lnvox, b->nf, b->chi, b->chi_c, b->chi_l, b->Bl, b->phi, b->S_l,
                                                b->S);
        BCK(cudaGetLastError());
    }
    k_bpack<<<152 * 8, 256, 0, b->st>>>(b->ntot, b->chi, b->S, b->B, b->cs, b->B32);
    BCK(cudaGetLastError());
    for (const Wave &w : b->waves) {
        BCK(cudaMemsetAsync(b->counters, 0, 2 * sizeof(unsigned long long), b->st));
        BCK(march_batch(b->d_mi + w.mi0, b->d_bpfx + w.pf0, w.n, w.bundles, b->chunk, 0, b->counters, b->grid_march,
                        b->st));
        BCK(gather_J_batch(b->d_gi + w.mi0, b->d_wpfx + w.pf0, w.n, w.work, b->counters + 1, b->grid_gather, b->st));
    }
    BCK(cudaMemsetAsync(b->maxrel, 0, sizeof(unsigned long long) * b->nm, b->st));
    if (b->line && b->lstar == RT_LSTAR_NN) {  // the OS solve follows the graph (line_nn_os)
        k_line_rhs<<<(b->lnvox + 255) / 256, 256, 0, b->st>>>(b->lnvox, b->nf, b->J, b->phi, b->wq, b->eps_l, b->Bl,
                                                              b->S_l, b->Jbar, b->nny);
    } else if (b->line) {
        k_line_update<<<(b->lnvox + 255) / 256, 256, 0, b->st>>>(b->lnvox, b->nf, b->J, b->phi, b->wq, b->eps_l, b->Bl,
                                                                 b->Lbar, b->S_l, b->Jbar, b->maxrel);
    } else {
        k_bali<<<152 * 8, 256, 0, b->st>>>(b->ntot, b->d_voff, b->nm, b->S, b->J, b->L, b->eps, b->B, b->maxrel);
    }
    BCK(cudaGetLastError());
    return RT_OK;
}

// One correction sweep of the refined solve for all members (captured).
int enqueue_correction(rt_batch *b)
{
    k_bpack<<<152 * 8, 256, 0, b->st>>>(b->ntot, b->chi, b->D, b->B, b->cs, b->B32);
    BCK(cudaGetLastError());
    for (const Wave &w : b->waves) {
        BCK(cudaMemsetAsync(b->counters, 0, 2 * sizeof(unsigned long long), b->st));
        BCK(march_batch(b->d_mi + w.mi0, b->d_bpfx + w.pf0, w.n, w.bundles, b->chunk, 1, b->counters, b->grid_march,
                        b->st));
        BCK(gather_J_batch(b->d_gi + w.mi0, b->d_wpfx + w.pf0, w.n, w.work, b->counters + 1, b->grid_gather, b->st));
    }
    BCK(cudaMemsetAsync(b->maxrel, 0, sizeof(unsigned long long) * b->nm, b->st));
    k_bcorr<<<152 * 8, 256, 0, b->st>>>(b->ntot, b->d_voff, b->nm, b->D, b->J, b->R, b->L, b->eps, b->S, b->maxrel);
    BCK(cudaGetLastError());
    return RT_OK;
}

int capture_corr(rt_batch *b)
{
    if (b->graph_corr) {
        cudaGraphExecDestroy(b->graph_corr);
        b->graph_corr = nullptr;
    }
    cudaGraph_t gr = nullptr;
    BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_correction(b);
    cudaError_t e = cudaStreamEndCapture(b->st, &gr);
    if (rc != RT_OK) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
    }
    if (e != cudaSuccess) return bfail(RT_ECUDA, std::string("stream capture failed: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph_corr, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return bfail(RT_ECUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e));
    return RT_OK;
}

int read_member_rel(rt_batch *b, std::vector<double> &rel)
{
    BCK(cudaMemcpyAsync(b->h_maxrel.data(), b->maxrel, sizeof(unsigned long long) * b->nm, cudaMemcpyDeviceToHost,
                        b->st));
    BCK(cudaStreamSynchronize(b->st));
    for (int m = 0; m < b->nm; ++m) std::memcpy(&rel[m], &b->h_maxrel[m], sizeof(double));
    return RT_OK;
}

int capture(rt_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t gr = nullptr;
    BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iteration(b);
    cudaError_t e = cudaStreamEndCapture(b->st, &gr);
    if (rc != RT_OK) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
    }
    if (e != cudaSuccess) return bfail(RT_ECUDA, std::string("stream capture failed: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return bfail(RT_ECUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e));
    return RT_OK;
}

// Nearest-neighbour OS step of the line: (I - (1 - eps_l) Lbar27) dS_l = y by
// BiCGSTAB on the Jacobi-preconditioned system and Jacobi sweeps until one
// changes dS_l by <= 1e-14 max |dS_l|, then S_l += dS_l and the max rel dS_l.
int line_nn_os(rt_batch *b)
{
    const rt_grid *g = b->grids[0];
    NnOs o{};
    o.nvox = b->lnvox;
    o.sph = g->coord == RT_SPHERICAL;
    o.n1 = g->n1;
    o.n2 = g->n2;
    o.n3 = g->n3;
    o.L27 = b->Lbar27;
    o.eps = b->eps_l;
    o.y = b->nny;
    o.work = b->nnx;
    o.jtol = 1e-14;
    o.jmax = 100000;
    o.krylov = 1;
    o.kmax = 1000;
    double *x = nullptr;
    int its = 0, sweeps = 0, status = 0;
    BCK(nn_os_solve(o, b->st, &x, &its, &sweeps, &status));
    if (status == 3) return bfail(RT_ETIMEOUT, "line NN OS step: a grid-barrier wait gave up");
    if (status == 2) return bfail(RT_EDEVICE, "line NN OS step diverged");
    if (status == 1) return bfail(RT_ENOTCONVERGED, "line NN OS step: no convergence in 100000 sweeps");
    b->nn_sweeps = sweeps;
    BCK(nn_apply(b->lnvox, b->S_l, x, nullptr, nullptr, b->maxrel, b->st));
    return RT_OK;
}

// Ng of the line: S_l joins the four-iterate history; once four have
// accumulated since the last extrapolation, S_l is replaced by the order-2 Ng
// combination (when its 2x2 system is regular).
int line_ng(rt_batch *b)
{
    const size_t n = b->lnvox;
    if (b->nh == 4) {
        const int t = b->hs[0];
        b->hs[0] = b->hs[1];
        b->hs[1] = b->hs[2];
        b->hs[2] = b->hs[3];
        b->hs[3] = t;
        b->nh = 3;
    }
    BCK(cudaMemcpyAsync(b->H + b->hs[b->nh] * n, b->S_l, sizeof(double) * n, cudaMemcpyDeviceToDevice, b->st));
    if (++b->nh < 4) return RT_OK;
    BCK(ng_extrapolate(b->lnvox, b->H + b->hs[3] * n, b->H + b->hs[2] * n, b->H + b->hs[1] * n, b->H + b->hs[0] * n,
                       nullptr, b->ng_part, b->ng_coef, b->S_l, b->st));
    double applied = 0.0;
    BCK(cudaMemcpyAsync(&applied, b->ng_coef + 2, sizeof(double), cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    if (applied != 0.0) b->nh = 0;
    return RT_OK;
}

int step(rt_batch *b, double *rel_out)
{
    for (int m = 0; m < b->nm; ++m)
        if (!b->ready[m]) return bfail(RT_EINVAL, "member " + std::to_string(m) + " has no opacity yet");
    if (!b->graph) BRCK(capture(b));
    BCK(cudaGraphLaunch(b->graph, b->st));
    if (b->line && b->lstar == RT_LSTAR_NN) BRCK(line_nn_os(b));
    BCK(cudaMemcpyAsync(b->h_maxrel.data(), b->maxrel, sizeof(unsigned long long) * b->nm, cudaMemcpyDeviceToHost,
                        b->st));
    BCK(cudaStreamSynchronize(b->st));
    double mx = 0.0;
    for (int m = 0; m < b->nm; ++m) {
        double r;
        std::memcpy(&r, &b->h_maxrel[m], sizeof(r));
        if (rel_out) rel_out[m] = r;
        mx = std::max(mx, r);
    }
    b->history.push_back(mx);
    return RT_OK;
}

}  // namespace

extern "C" {

int rt_batch_create(rt_batch **out, rt_grid *const *grids, int n_grids, int n_members, const int32_t *member_grid,
                    void *stream)
{
    if (!out || !grids || n_grids < 1 || n_members < 1 || !member_grid) return bfail(RT_EINVAL, "bad arguments");
    for (int q = 0; q < n_grids; ++q)
        if (!grids[q]) return bfail(RT_EINVAL, "grid " + std::to_string(q) + " is NULL");
    for (int m = 0; m < n_members; ++m)
        if (member_grid[m] < 0 || member_grid[m] >= n_grids) return bfail(RT_EINVAL, "member_grid out of range");
    for (int q = 0; q < n_grids; ++q) {
        if (grids[q]->device != grids[0]->device) return bfail(RT_EINVAL, "all grids must live on one device");
        if (grids[q]->lost) return bfail(RT_EDEVICE, "a grid has characteristics that could not be tracked");
        for (int k = 0; k < grids[q]->nblk; ++k)
            if (grids[q]->h_ang_seg_off[grids[q]->blk_w0[k] + grids[q]->blk_nw[k]] - grids[q]->h_ang_seg_off[grids[q]->blk_w0[k]] >= (1ll << 31))
                return bfail(RT_EINVAL, "angle block too large");
    }
    if (cudaSetDevice(grids[0]->device) != cudaSuccess) return bfail(RT_ECUDA, "cudaSetDevice failed");
    rt_batch *b = new rt_batch();
    b->device = grids[0]->device;
    b->grids.assign(grids, grids + n_grids);
    b->mgrid.assign(member_grid, member_grid + n_members);
    b->nm = n_members;
    b->ready.assign(n_members, 0);
    b->h_maxrel.assign(n_members, 0ull);
    auto fail_and_free = [&](int rc) {
        std::string keep = rt_last_error();
        if (b->st) cudaStreamSynchronize(b->st);
        bfree_all(b);
        delete b;
        set_last_error(keep.c_str());
        return rc;
    };
    if (stream) {
        b->st = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess)
            return fail_and_free(bfail(RT_ECUDA, "stream creation failed"));
        b->own_stream = true;
    }
    b->voff.assign(n_members + 1, 0);
    int max_vox = 0;
    for (int m = 0; m < n_members; ++m) {
        b->voff[m + 1] = b->voff[m] + grids[member_grid[m]]->nvox;
        max_vox = std::max(max_vox, grids[member_grid[m]]->nvox);
    }
    b->ntot = b->voff[n_members];
    int rc = RT_OK;
#define TRY(x)                          \
    do {                                \
        if ((rc = (x)) != RT_OK) return fail_and_free(rc); \
    } while (0)
    TRY(balloc(b, &b->chi, b->ntot));
    TRY(balloc(b, &b->eps, b->ntot));
    TRY(balloc(b, &b->B, b->ntot));
    TRY(balloc(b, &b->S, b->ntot));
    TRY(balloc(b, &b->J, b->ntot));
    TRY(balloc(b, &b->L, b->ntot));
    TRY(balloc(b, &b->Fc, 3 * (size_t)max_vox));
    TRY(balloc(b, &b->cs, b->ntot));
    TRY(balloc(b, &b->B32, b->ntot));
    TRY(balloc(b, &b->d_voff, n_members + 1));
    TRY(balloc(b, &b->maxrel, n_members));
    TRY(balloc(b, &b->counters, 2));
    TRY(balloc(b, &b->R, b->ntot));
    TRY(balloc(b, &b->D, b->ntot));
    TRY(balloc(b, &b->cs64, max_vox));
    TRY(balloc(b, &b->d_active, n_members));
    if (cudaMemcpyAsync(b->d_voff, b->voff.data(), sizeof(int64_t) * (n_members + 1), cudaMemcpyHostToDevice, b->st) !=
        cudaSuccess)
        return fail_and_free(bfail(RT_ECUDA, "copy failed"));
    b->pbits.assign(n_members, nullptr);
    for (int m = 0; m < n_members; ++m)
        TRY(balloc(b, &b->pbits[m], (grids[member_grid[m]]->n_seg + 31) / 32));
    // waves: wave k holds angle block k of every member whose grid has one
    int maxblk = 0;
    for (rt_grid *g : b->grids) maxblk = std::max(maxblk, g->nblk);
    int64_t max_buf = 0, max_part = 0, max_cnt = 0;
    for (int k = 0; k < maxblk; ++k) {
        Wave w;
        w.mi0 = (int64_t)b->h_mi.size();
        int64_t buf = 0, part = 0, cnt = 0;
        for (int m = 0; m < n_members; ++m) {
            rt_grid *g = b->grids[b->mgrid[m]];
            if (k >= g->nblk) continue;
            const int w0 = g->blk_w0[k], nw = g->blk_nw[k];
            const int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
            MarchItem mi;
            mi.vox = g->d_vox;
            mi.len = g->d_len32;
            mi.ray_off = g->d_ray_off;
            mi.r_lo = g->h_ang_ray_off[w0];
            mi.r_hi = g->h_ang_ray_off[w0 + nw];
            mi.seg_lo = lo;
            mi.nseg = ns;
            mi.cs = b->cs + b->voff[m];
            mi.B = b->B32 + b->voff[m];
            mi.pbits = b->pbits[m];
            mi.I_outer = (float)g->I_outer;
            mi.out = (float *)(intptr_t)buf;  // offset for now
            GatherItem gi;
            gi.t = g->jt[k];
            gi.t.cnt = (int *)(intptr_t)cnt;
            gi.off = g->d_csr_off + (size_t)k * (g->nvox + 1);
            gi.perm = g->d_perm + lo;
            gi.buf = (const float *)(intptr_t)buf;
            gi.ang_seg_off = g->d_ang_seg_off;
            gi.wL = g->d_wL32;
            gi.invL = g->d_invL;
            gi.wt = g->d_wt;
            gi.part = (double *)(intptr_t)part;
            gi.J = b->J + b->voff[m];
            gi.seg_lo = lo;
            gi.w0 = w0;
            gi.nw = nw;
            gi.nvox = g->nvox;
            gi.first = (k == 0);
            gi.nbs = (gi.t.nshort + 255) / 256;
            gi.nbc = (gi.t.nchunks * 32 + 255) / 256;
            b->h_mi.push_back(mi);
            b->h_gi.push_back(gi);
            buf += ns;
            part += std::max<int64_t>(1, gi.t.nchunks);
            cnt += std::max(1, gi.t.nlong);
            w.n++;
        }
        b->waves.push_back(w);
        max_buf = std::max(max_buf, buf);
        max_part = std::max(max_part, part);
        max_cnt = std::max(max_cnt, cnt);
    }
    TRY(balloc(b, &b->wbuf, max_buf));
    TRY(balloc(b, &b->wpart, max_part));
    TRY(balloc(b, &b->wcnt, max_cnt));
    if (cudaMemsetAsync(b->wcnt, 0, sizeof(int) * max_cnt, b->st) != cudaSuccess)
        return fail_and_free(bfail(RT_ECUDA, "memset failed"));
    for (size_t i = 0; i < b->h_mi.size(); ++i) {  // turn offsets into pointers
        b->h_mi[i].out = b->wbuf + (intptr_t)b->h_mi[i].out;
        b->h_gi[i].buf = b->wbuf + (intptr_t)b->h_gi[i].buf;
        b->h_gi[i].part = b->wpart + (intptr_t)b->h_gi[i].part;
        b->h_gi[i].t.cnt = b->wcnt + (intptr_t)b->h_gi[i].t.cnt;
    }
    TRY(balloc(b, &b->d_mi, b->h_mi.size()));
    TRY(balloc(b, &b->d_gi, b->h_gi.size()));
    if (cudaMemcpyAsync(b->d_mi, b->h_mi.data(), sizeof(MarchItem) * b->h_mi.size(), cudaMemcpyHostToDevice, b->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_gi, b->h_gi.data(), sizeof(GatherItem) * b->h_gi.size(), cudaMemcpyHostToDevice, b->st) !=
            cudaSuccess)
        return fail_and_free(bfail(RT_ECUDA, "copy failed"));
    TRY(build_prefixes(b));
#undef TRY
    *out = b;
    return RT_OK;
}

int rt_batch_destroy(rt_batch *b)
{
    if (!b) return RT_OK;
    cudaSetDevice(b->device);
    if (b->st) cudaStreamSynchronize(b->st);
    bfree_all(b);
    delete b;
    return RT_OK;
}

int batch_set_member(rt_batch *b, int m, const double *chi, const double *eps, const double *B, int where);

int rt_batch_set_member(rt_batch *b, int m, const double *chi, const double *eps, const double *B, int where)
{
    if (b && b->line) return bfail(RT_EINVAL, "the frequencies of a line problem are set by rt_line_set");
    return batch_set_member(b, m, chi, eps, B, where);
}

int batch_set_member(rt_batch *b, int m, const double *chi, const double *eps, const double *B, int where)
{
    if (!b || !chi || !eps || !B) return bfail(RT_EINVAL, "NULL argument");
    if (m < 0 || m >= b->nm) return bfail(RT_EINVAL, "member out of range");
    if (where != RT_HOST && where != RT_DEVICE) return bfail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    BCK(cudaSetDevice(b->device));
    rt_grid *g = b->grids[b->mgrid[m]];
    const int64_t n = g->nvox, o = b->voff[m];
    if (where == RT_HOST) {
        for (int64_t v = 0; v < n; ++v) {
            if (!(chi[v] > 0.0) || !std::isfinite(chi[v])) return bfail(RT_EINVAL, "chi must be > 0 and finite");
            if (!(eps[v] > 0.0 && eps[v] <= 1.0)) return bfail(RT_EINVAL, "eps must be in (0, 1]");
            if (!(B[v] >= 0.0) || !std::isfinite(B[v])) return bfail(RT_EINVAL, "B must be >= 0 and finite");
        }
    }
    const cudaMemcpyKind kind = where == RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    BCK(cudaMemcpyAsync(b->chi + o, chi, sizeof(double) * n, kind, b->st));
    BCK(cudaMemcpyAsync(b->eps + o, eps, sizeof(double) * n, kind, b->st));
    BCK(cudaMemcpyAsync(b->B + o, B, sizeof(double) * n, kind, b->st));
    BCK(cudaMemcpyAsync(b->S + o, b->B + o, sizeof(double) * n, cudaMemcpyDeviceToDevice, b->st));
    BCK(para_bits(g->d_vox, g->d_len64, b->chi + o, g->n_seg, g->interp == RT_PARABOLIC, b->pbits[m], b->st));
    // this member's Lambda* (depends on its chi only): one full FP32 formal solution
    k_bpack<<<152 * 4, 256, 0, b->st>>>(n, b->chi + o, b->S + o, b->B + o, b->cs + o, b->B32 + o);
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(b->st));
    BCK(cudaStreamSynchronize(g->st));
    BRCK(rt_grid_member_fs(g, b->cs + o, b->B32 + o, b->pbits[m], b->J + o, b->L + o, b->Fc, b->st));
    BCK(cudaStreamSynchronize(b->st));
    b->ready[m] = 1;
    b->history.clear();
    return RT_OK;
}

int rt_batch_ali_step(rt_batch *b, double *max_rel_dS)
{
    if (!b) return bfail(RT_EINVAL, "batch is NULL");
    if (b->line) return bfail(RT_EINVAL, "a line problem iterates with rt_line_step");
    BCK(cudaSetDevice(b->device));
    return step(b, max_rel_dS);
}

int rt_batch_solve(rt_batch *b, double tol, int max_iter, int32_t *iters)
{
    if (!b) return bfail(RT_EINVAL, "batch is NULL");
    if (b->line) return bfail(RT_EINVAL, "a line problem iterates with rt_line_solve");
    if (!(tol > 0.0) || max_iter < 1) return bfail(RT_EINVAL, "need tol > 0 and max_iter >= 1");
    BCK(cudaSetDevice(b->device));
    for (int m = 0; m < b->nm; ++m)
        if (!b->ready[m]) return bfail(RT_EINVAL, "member " + std::to_string(m) + " has no opacity yet");
    for (rt_grid *g : b->grids) BCK(cudaStreamSynchronize(g->st));
    // Mixed precision with FP64 refinement, per member as rt_solve does for one grid:
    // an FP64 formal solution gives the exact residual r = (1-eps) J64 + eps B - S,
    // then up to refine_every batched FP32 J-only sweeps solve for the correction D
    // with the diagonal Lambda*, and S += D.  A member is done when the ALI update
    // its FP64 residual asks for is below tol; its residual is then held at zero.
    std::vector<double> rel(b->nm, 0.0);
    std::vector<int32_t> done(b->nm, 0);
    std::vector<int> active(b->nm, 1);
    b->history.clear();
    if (!b->graph_corr) BRCK(capture_corr(b));
    const double inner_tol = 0.01 * tol;
    int total = 0;
    while (total < max_iter) {
        for (int m = 0; m < b->nm; ++m) {
            if (!active[m]) continue;
            rt_grid *g = b->grids[b->mgrid[m]];
            const int64_t o = b->voff[m], n = g->nvox;
            k_bpack64<<<152 * 4, 256, 0, b->st>>>(n, b->chi + o, b->S + o, b->cs64);
            BCK(cudaGetLastError());
            BRCK(rt_grid_member_fs64J(g, b->cs64, b->B + o, b->pbits[m], b->J + o, b->st));
        }
        total++;
        BCK(cudaMemcpyAsync(b->d_active, active.data(), sizeof(int) * b->nm, cudaMemcpyHostToDevice, b->st));
        BCK(cudaMemsetAsync(b->maxrel, 0, sizeof(unsigned long long) * b->nm, b->st));
        k_bresid<<<152 * 8, 256, 0, b->st>>>(b->ntot, b->d_voff, b->nm, b->d_active, b->S, b->J, b->L, b->eps, b->B,
                                             b->R, b->maxrel);
        BCK(cudaGetLastError());
        BRCK(read_member_rel(b, rel));
        double mx = 0.0;
        bool all = true;
        for (int m = 0; m < b->nm; ++m) {
            if (!active[m]) continue;
            mx = std::max(mx, rel[m]);
            if (rel[m] < tol) {
                done[m] = total;
                active[m] = 0;
            }
            all = all && !active[m];
        }
        b->history.push_back(mx);
        if (all) {
            if (iters) std::copy(done.begin(), done.end(), iters);
            return RT_OK;
        }
        BCK(cudaMemsetAsync(b->D, 0, sizeof(double) * b->ntot, b->st));
        for (int k = 0; k < b->refine_every && total < max_iter; ++k) {
            BCK(cudaGraphLaunch(b->graph_corr, b->st));
            BRCK(read_member_rel(b, rel));
            total++;
            double rd = 0.0;
            for (int m = 0; m < b->nm; ++m)
                if (active[m]) rd = std::max(rd, rel[m]);
            if (rd < inner_tol) break;
        }
        k_badd<<<152 * 8, 256, 0, b->st>>>(b->ntot, b->S, b->D);
        BCK(cudaGetLastError());
    }
    BCK(cudaStreamSynchronize(b->st));
    if (iters) std::copy(done.begin(), done.end(), iters);
    return bfail(RT_ENOTCONVERGED, "not every member converged in " + std::to_string(max_iter) + " formal solutions");
}

int rt_batch_get(const rt_batch *b, int m, int what, double *out, int where)
{
    if (!b || !out) return bfail(RT_EINVAL, "NULL argument");
    if (m < 0 || m >= b->nm) return bfail(RT_EINVAL, "member out of range");
    if (where != RT_HOST && where != RT_DEVICE) return bfail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    const double *src = what == 0 ? b->S : what == 1 ? b->J : what == 2 ? b->L : nullptr;
    if (!src) return bfail(RT_EINVAL, "what must be 0 (S), 1 (J) or 2 (Lambda*)");
    BCK(cudaSetDevice(b->device));
    const int64_t n = b->voff[m + 1] - b->voff[m];
    BCK(cudaMemcpyAsync(out, src + b->voff[m], sizeof(double) * n,
                        where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));
    return RT_OK;
}

int rt_batch_autotune(rt_batch *b, int32_t *chunk_out, int32_t *grid_out, double *ms_out)
{
    if (!b) return bfail(RT_EINVAL, "batch is NULL");
    BCK(cudaSetDevice(b->device));
    for (int m = 0; m < b->nm; ++m)
        if (!b->ready[m]) return bfail(RT_EINVAL, "set every member before autotuning");
    double *saveS = nullptr;  // line mode: the iteration also moves S_l, kept after the member S
    const size_t nsave = b->ntot + (b->line ? b->lnvox : 0);
    BRCK(balloc(b, &saveS, nsave));
    BCK(cudaMemcpyAsync(saveS, b->S, sizeof(double) * b->ntot, cudaMemcpyDeviceToDevice, b->st));
    if (b->line)
        BCK(cudaMemcpyAsync(saveS + b->ntot, b->S_l, sizeof(double) * b->lnvox, cudaMemcpyDeviceToDevice, b->st));
    const int chunks[3] = {512, 1024, 2048};
    const int grids[2] = {152 * 4, 152 * 8};
    double best = 1e300;
    int bc = b->chunk, bg = b->grid_march;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    for (int c : chunks)
        for (int gsz : grids) {
            b->chunk = c;
            b->grid_march = b->grid_gather = gsz;
            BRCK(build_prefixes(b));
            BRCK(capture(b));
            BCK(cudaGraphLaunch(b->graph, b->st));
            BCK(cudaEventRecord(e0, b->st));
            BCK(cudaGraphLaunch(b->graph, b->st));
            BCK(cudaGraphLaunch(b->graph, b->st));
            BCK(cudaEventRecord(e1, b->st));
            BCK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms / 2 < best) {
                best = ms / 2;
                bc = c;
                bg = gsz;
            }
            BCK(cudaMemcpyAsync(b->S, saveS, sizeof(double) * b->ntot, cudaMemcpyDeviceToDevice, b->st));
            if (b->line)
                BCK(cudaMemcpyAsync(b->S_l, saveS + b->ntot, sizeof(double) * b->lnvox, cudaMemcpyDeviceToDevice,
                                    b->st));
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chunk = bc;
    b->grid_march = b->grid_gather = bg;
    BRCK(build_prefixes(b));
    BRCK(capture(b));
    if (b->graph_corr) {  // recaptured with the chosen bundle size at the next rt_batch_solve
        cudaGraphExecDestroy(b->graph_corr);
        b->graph_corr = nullptr;
    }
    BCK(cudaStreamSynchronize(b->st));
    auto it = std::find(b->allocs.begin(), b->allocs.end(), (void *)saveS);
    if (it != b->allocs.end()) b->allocs.erase(it);
    cudaFree(saveS);
    b->history.clear();
    if (chunk_out) *chunk_out = bc;
    if (grid_out) *grid_out = bg;
    if (ms_out) *ms_out = best;
    return RT_OK;
}

// ---- two-level-atom line transfer (the members are the frequencies) ----

int rt_line_create(rt_batch **out, rt_grid *g, int n_freq, const double *phi, const double *wq, int use_lstar, int ng,
                   void *stream)
{
    if (!out || !g || n_freq < 1 || !phi || !wq) return bfail(RT_EINVAL, "bad arguments");
    if (use_lstar != RT_LSTAR_DIAG && use_lstar != RT_LSTAR_NN)
        return bfail(RT_EINVAL, "use_lstar must be RT_LSTAR_DIAG or RT_LSTAR_NN");
    if (ng != 0 && ng != 1) return bfail(RT_EINVAL, "ng must be 0 or 1");
    if (use_lstar == RT_LSTAR_NN && g->nphi < 3) return bfail(RT_EINVAL, "the nearest-neighbour Lambda* needs n_phi >= 3");
    double norm = 0.0;
    for (int k = 0; k < n_freq; ++k) {
        if (!(phi[k] >= 0.0) || !std::isfinite(phi[k]) || !(wq[k] >= 0.0) || !std::isfinite(wq[k]))
            return bfail(RT_EINVAL, "phi and wq must be >= 0 and finite");
        norm += wq[k] * phi[k];
    }
    if (!(std::fabs(norm - 1.0) <= 1e-10)) return bfail(RT_EINVAL, "sum_k wq_k phi_k must be 1");
    std::vector<int32_t> mg(n_freq, 0);
    rt_grid *gs[1] = {g};
    rt_batch *b = nullptr;
    BRCK(rt_batch_create(&b, gs, 1, n_freq, mg.data(), stream));
    b->line = 1;
    b->lstar = use_lstar;
    b->ng = ng;
    b->nf = n_freq;
    b->lnvox = g->nvox;
    b->h_phi.assign(phi, phi + n_freq);
    b->h_wq.assign(wq, wq + n_freq);
    const int n = g->nvox;
    int rc = RT_OK;
    if ((rc = balloc(b, &b->chi_c, n)) != RT_OK || (rc = balloc(b, &b->chi_l, n)) != RT_OK ||
        (rc = balloc(b, &b->eps_l, n)) != RT_OK || (rc = balloc(b, &b->Bl, n)) != RT_OK ||
        (rc = balloc(b, &b->phi, n_freq)) != RT_OK || (rc = balloc(b, &b->wq, n_freq)) != RT_OK ||
        (rc = balloc(b, &b->S_l, n)) != RT_OK || (rc = balloc(b, &b->Jbar, n)) != RT_OK ||
        (rc = balloc(b, &b->Lbar, n)) != RT_OK || (rc = balloc(b, &b->ones, n)) != RT_OK ||
        (rc = balloc(b, &b->tmp, n)) != RT_OK ||
        (use_lstar == RT_LSTAR_NN &&
         ((rc = balloc(b, &b->Lbar27, 27 * (size_t)n)) != RT_OK || (rc = balloc(b, &b->L27k, 27 * (size_t)n)) != RT_OK ||
          (rc = balloc(b, &b->nnx, (size_t)nn_os_work_elems(n))) != RT_OK || (rc = balloc(b, &b->nny, n)) != RT_OK)) ||
        (ng && ((rc = balloc(b, &b->H, 4 * (size_t)n)) != RT_OK ||
                (rc = balloc(b, &b->ng_part, ng_partial_elems(n))) != RT_OK ||
                (rc = balloc(b, &b->ng_coef, 4)) != RT_OK))) {
        std::string keep = rt_last_error();
        rt_batch_destroy(b);
        set_last_error(keep.c_str());
        return rc;
    }
    if (cudaMemcpyAsync(b->phi, phi, sizeof(double) * n_freq, cudaMemcpyHostToDevice, b->st) != cudaSuccess ||
        cudaMemcpyAsync(b->wq, wq, sizeof(double) * n_freq, cudaMemcpyHostToDevice, b->st) != cudaSuccess ||
        fill_const(n, b->ones, 1.0, b->st) != cudaSuccess || cudaStreamSynchronize(b->st) != cudaSuccess) {
        rt_batch_destroy(b);
        return bfail(RT_ECUDA, "line set-up copies failed");
    }
    *out = b;
    return RT_OK;
}

int rt_line_set(rt_batch *b, const double *chi_c, const double *chi_l, const double *eps_l, const double *B, int where)
{
    if (!b || !chi_c || !chi_l || !eps_l || !B) return bfail(RT_EINVAL, "NULL argument");
    if (!b->line) return bfail(RT_EINVAL, "not a line problem (rt_line_create)");
    if (where != RT_HOST && where != RT_DEVICE) return bfail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    BCK(cudaSetDevice(b->device));
    const int n = b->lnvox;
    if (where == RT_HOST) {
        for (int v = 0; v < n; ++v) {
            if (!(chi_c[v] >= 0.0) || !(chi_l[v] >= 0.0) || !std::isfinite(chi_c[v]) || !std::isfinite(chi_l[v]))
                return bfail(RT_EINVAL, "chi_c and chi_l must be >= 0 and finite");
            for (int k = 0; k < b->nf; ++k)
                if (!(chi_c[v] + chi_l[v] * b->h_phi[k] > 0.0)) return bfail(RT_EINVAL, "chi_c + chi_l phi_k must be > 0");
            if (!(eps_l[v] > 0.0 && eps_l[v] <= 1.0)) return bfail(RT_EINVAL, "eps_l must be in (0, 1]");
            if (!(B[v] >= 0.0) || !std::isfinite(B[v])) return bfail(RT_EINVAL, "B must be >= 0 and finite");
        }
    }
    const cudaMemcpyKind kind = where == RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    BCK(cudaMemcpyAsync(b->chi_c, chi_c, sizeof(double) * n, kind, b->st));
    BCK(cudaMemcpyAsync(b->chi_l, chi_l, sizeof(double) * n, kind, b->st));
    BCK(cudaMemcpyAsync(b->eps_l, eps_l, sizeof(double) * n, kind, b->st));
    BCK(cudaMemcpyAsync(b->Bl, B, sizeof(double) * n, kind, b->st));
    for (int k = 0; k < b->nf; ++k) {  // frequency k: chi_k, its parabola choices and Lambda*_k
        k_line_chik<<<(n + 255) / 256, 256, 0, b->st>>>(n, b->chi_c, b->chi_l, b->h_phi[k], b->tmp);
        BCK(cudaGetLastError());
        BRCK(batch_set_member(b, k, b->tmp, b->ones, b->Bl, RT_DEVICE));
        if (b->lstar == RT_LSTAR_NN) {
            const rt_grid *g = b->grids[0];
            BRCK(rt_grid_nn_lstar(b->grids[0], b->tmp, b->pbits[k], b->L27k, b->st));
            k_line_lbar_nn<<<(n + 127) / 128, 128, 0, b->st>>>(n, g->coord == RT_SPHERICAL, g->n1, g->n2, g->n3, b->L27k,
                                                                b->chi_c, b->chi_l, b->h_phi[k],
                                                                b->h_wq[k] * b->h_phi[k], b->Lbar27, k == 0);
            BCK(cudaGetLastError());
        }
    }
    k_line_lbar<<<(n + 255) / 256, 256, 0, b->st>>>(n, b->nf, b->L, b->chi, b->chi_l, b->phi, b->wq, b->Lbar);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(b->S_l, b->Bl, sizeof(double) * n, cudaMemcpyDeviceToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));
    b->line_ready = true;
    b->history.clear();
    b->nh = 0;
    return RT_OK;
}

// One line iteration; Ng follows unless the iterate has met tol.
int line_iterate(rt_batch *b, double tol, double *rel_out)
{
    std::vector<double> rel(b->nm);
    BRCK(step(b, rel.data()));
    *rel_out = rel[0];
    if (b->ng && !(rel[0] < tol)) BRCK(line_ng(b));
    return RT_OK;
}

int rt_line_step(rt_batch *b, double *max_rel_dSl)
{
    if (!b) return bfail(RT_EINVAL, "batch is NULL");
    if (!b->line) return bfail(RT_EINVAL, "not a line problem (rt_line_create)");
    if (!b->line_ready) return bfail(RT_EINVAL, "rt_line_set first");
    BCK(cudaSetDevice(b->device));
    double rel = 0.0;
    BRCK(line_iterate(b, 0.0, &rel));
    if (max_rel_dSl) *max_rel_dSl = rel;
    return RT_OK;
}

int rt_line_solve(rt_batch *b, double tol, int max_iter, int32_t *iters)
{
    if (!b) return bfail(RT_EINVAL, "batch is NULL");
    if (!b->line) return bfail(RT_EINVAL, "not a line problem (rt_line_create)");
    if (!b->line_ready) return bfail(RT_EINVAL, "rt_line_set first");
    if (!(tol > 0.0) || max_iter < 1) return bfail(RT_EINVAL, "need tol > 0 and max_iter >= 1");
    BCK(cudaSetDevice(b->device));
    if (iters) *iters = 0;
    b->nh = 0;
    for (int it = 1; it <= max_iter; ++it) {
        double rel = 0.0;
        BRCK(line_iterate(b, tol, &rel));
        if (iters) *iters = it;
        if (rel < tol) return RT_OK;
    }
    return bfail(RT_ENOTCONVERGED, "line source function not converged in " + std::to_string(max_iter) + " iterations");
}

int rt_line_get(const rt_batch *b, int what, double *out, int where)
{
    if (!b || !out) return bfail(RT_EINVAL, "NULL argument");
    if (!b->line) return bfail(RT_EINVAL, "not a line problem (rt_line_create)");
    if (where != RT_HOST && where != RT_DEVICE) return bfail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    const double *src = what == 0 ? b->S_l : what == 1 ? b->Jbar : what == 2 ? b->Lbar : what == 3 ? b->Lbar27 : nullptr;
    if (!src) return bfail(RT_EINVAL, "what must be 0 (S_l), 1 (Jbar), 2 (Lbar*) or 3 (Lbar*_NN of a NN line)");
    BCK(cudaSetDevice(b->device));
    if (what == 3) {  // slot planes to rows of 27, through L27k as scratch
        BCK(nn_rows(b->lnvox, b->Lbar27, b->L27k, b->st));
        src = b->L27k;
    }
    BCK(cudaMemcpyAsync(out, src, sizeof(double) * b->lnvox * (what == 3 ? 27 : 1),
                        where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));
    return RT_OK;
}

}  // extern "C"
