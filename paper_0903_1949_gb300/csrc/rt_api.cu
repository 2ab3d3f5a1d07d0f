// rt_api.cu -- C ABI (include/rt.h): grid construction, formal solution,
// ALI / Ng iteration and mixed-precision refinement, all on one GPU.
//
// Host code here only validates, allocates, orders launches on the grid's
// stream and moves the few scalars the iteration control needs; every step
// of the method runs in the kernels of geom.cu, march.cu, gather.cu, ali.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "geom_pred.cuh"
#include "rt_internal.h"

using namespace rtk;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(...)                                                                                             \
    do {                                                                                                    \
        cudaError_t e_ = (__VA_ARGS__);                                                                     \
        if (e_ != cudaSuccess) return fail(RT_ECUDA, "%s failed: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
    } while (0)

#define RCK(call)             \
    do {                      \
        int r_ = (call);      \
        if (r_ != RT_OK) return r_; \
    } while (0)

constexpr int64_t BLOCK_SEG_TARGET = 6000000;  // segments per angle block (FP32 pair buffer ~48 MB, L2-resident)
constexpr int MAX_BLOCK_ANGLES = 256;

}  // namespace

namespace rtk {
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace rtk

#include "grid.h"

namespace {

template <typename T>
int dalloc(rt_grid *g, T **p, size_t count)
{
    void *q = nullptr;
    size_t nbytes = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = cudaMalloc(&q, nbytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RT_ENOMEM, "cudaMalloc of %zu bytes failed: %s", nbytes, cudaGetErrorString(e));
    }
    g->allocs.push_back(q);
    g->bytes += (int64_t)nbytes;
    *p = (T *)q;
    return RT_OK;
}

void dfree(rt_grid *g, void *p)
{
    if (!p) return;
    auto it = std::find(g->allocs.begin(), g->allocs.end(), p);
    if (it != g->allocs.end()) {
        g->allocs.erase(it);
        cudaFree(p);
    }
}

// Forget the captured J-only formal solution (its arguments, knobs or the
// arrays it reads may have changed).
void drop_graph(rt_grid *g)
{
    for (rt_grid::FsGraph &f : g->fsg) {
        if (f.exec) cudaGraphExecDestroy(f.exec);
        f = rt_grid::FsGraph{};
    }
}

void release(rt_grid *g)
{
    drop_graph(g);
    if (g->stc) cudaStreamDestroy(g->stc);
    g->stc = nullptr;
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    g->ev.clear();
    for (cudaEvent_t &e : g->sev)
        if (e) cudaEventDestroy(e), e = nullptr;
    if (g->st2) cudaStreamDestroy(g->st2);
    g->st2 = nullptr;
    if (g->st3) cudaStreamDestroy(g->st3);
    g->st3 = nullptr;
    if (g->st4) cudaStreamDestroy(g->st4);
    g->st4 = nullptr;
    for (void *p : g->allocs) cudaFree(p);
    g->allocs.clear();
    if (g->h_pin) cudaFreeHost(g->h_pin);
    g->h_pin = nullptr;
}

int sync(rt_grid *g)
{
    CK(cudaStreamSynchronize(g->st));
    return RT_OK;
}

// Start event of a timed launch of `kind` (0 march, 1 gather) on stream st
// (default: the grid's stream); returns its slot, or -1 when this launch is not
// timed (timing off, or sampling every timing_every-th march launch only).
int tstart(rt_grid *g, int kind, cudaStream_t st = nullptr)
{
    if (!st) st = g->st;
    if (!g->timing) return -1;
    if (g->timing_every > 1) {
        if (kind != 0) return -1;
        if (g->timing_count++ % g->timing_every != 0) return -1;
    }
    if (g->ev_used + 2 > g->ev.size()) {
        for (int q = 0; q < 64; ++q) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            g->ev.push_back(e);
        }
    }
    int slot = (int)g->ev_used;
    g->ev_used += 2;
    cudaEventRecord(g->ev[slot], st);
    return slot;
}

void tstop(rt_grid *g, int slot, int kind, int64_t segs, int64_t bytes = 0, cudaStream_t st = nullptr)
{
    if (slot < 0) return;
    cudaEventRecord(g->ev[slot + 1], st ? st : g->st);
    g->ev_kind.push_back(kind);
    g->ev_segs.push_back(segs);
    g->ev_bytes.push_back(bytes);
}

int check_desc(const rt_grid_desc *d)
{
    if (!d) return fail(RT_EINVAL, "descriptor is NULL");
    if (d->coord != RT_SPHERICAL && d->coord != RT_CYLINDRICAL) return fail(RT_EINVAL, "coord must be RT_SPHERICAL or RT_CYLINDRICAL");
    for (int a = 0; a < 3; ++a) {
        if (d->n[a] < 1) return fail(RT_EINVAL, "n[%d] = %d must be >= 1", a, d->n[a]);
        if (!d->edges[a]) return fail(RT_EINVAL, "edges[%d] is NULL", a);
        for (int q = 0; q < d->n[a]; ++q)
            if (!(d->edges[a][q + 1] > d->edges[a][q]) || !std::isfinite(d->edges[a][q + 1]) ||
                !std::isfinite(d->edges[a][q]))
                return fail(RT_EINVAL, "edges[%d] must be finite and strictly increasing (index %d)", a, q);
    }
    int64_t nvox = (int64_t)d->n[0] * d->n[1] * d->n[2];
    if (nvox >= (int64_t)RTK_VOXMASK) return fail(RT_EINVAL, "too many voxels (%lld)", (long long)nvox);
    const double TWO_PI = 6.283185307179586476925286766559;
    if (d->coord == RT_SPHERICAL) {
        if (!(d->edges[0][0] > 0.0)) return fail(RT_EINVAL, "spherical grids need r_0 > 0 (core or hole)");
        if (d->edges[1][0] != 0.0 || std::fabs(d->edges[1][d->n[1]] - 3.141592653589793238462643383279) > 1e-12)
            return fail(RT_EINVAL, "theta edges must run from 0 to pi");
        if (std::fabs(d->edges[2][d->n[2]] - d->edges[2][0] - TWO_PI) > 1e-12)
            return fail(RT_EINVAL, "phi edges must span 2 pi");
    } else {
        if (!(d->edges[0][0] >= 0.0)) return fail(RT_EINVAL, "cylindrical grids need R_0 >= 0");
        if (std::fabs(d->edges[1][d->n[1]] - d->edges[1][0] - TWO_PI) > 1e-12)
            return fail(RT_EINVAL, "phi edges must span 2 pi");
    }
    if (d->n_angles < 1 || !d->dirs || !d->weights) return fail(RT_EINVAL, "need n_angles >= 1, dirs and weights");
    double wsum = 0.0;
    for (int w = 0; w < d->n_angles; ++w) {
        const double *n = d->dirs + 3 * w;
        double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        if (!(std::fabs(nn - 1.0) < 1e-12)) return fail(RT_EINVAL, "direction %d is not a unit vector", w);
        if (!(d->weights[w] > 0.0) || !std::isfinite(d->weights[w])) return fail(RT_EINVAL, "weight %d must be > 0", w);
        wsum += d->weights[w];
    }
    if (!(std::fabs(wsum - 1.0) < 1e-10)) return fail(RT_EINVAL, "weights must sum to 1 (got %.17g)", wsum);
    if (d->inner_bc != RT_CORE_B && d->inner_bc != RT_TRANSPARENT) return fail(RT_EINVAL, "bad inner_bc");
    if (d->interp != RT_PARABOLIC && d->interp != RT_LINEAR) return fail(RT_EINVAL, "bad interp");
    if (d->precision != RT_FP64 && d->precision != RT_MIXED) return fail(RT_EINVAL, "bad precision");
    if (!std::isfinite(d->I_outer) || d->I_outer < 0.0) return fail(RT_EINVAL, "I_outer must be finite and >= 0");
    if (d->angle_block < 0 || d->angle_block > MAX_BLOCK_ANGLES) return fail(RT_EINVAL, "angle_block must be in [0, 256]");
    if (d->use_lstar != RT_LSTAR_NONE && d->use_lstar != RT_LSTAR_DIAG && d->use_lstar != RT_LSTAR_NN)
        return fail(RT_EINVAL, "use_lstar must be RT_LSTAR_NONE, RT_LSTAR_DIAG or RT_LSTAR_NN");
    if (d->use_lstar == RT_LSTAR_NN && (d->coord == RT_SPHERICAL ? d->n[2] : d->n[1]) < 3)
        return fail(RT_EINVAL, "the nearest-neighbour Lambda* needs at least 3 phi cells");
    if (d->refine_every < 0) return fail(RT_EINVAL, "refine_every must be >= 0");
    return RT_OK;
}

// Trigonometric tables of the angular edges and mid-points (G0), uploaded.
int upload_tables(rt_grid *g)
{
    const bool sph = g->coord == RT_SPHERICAL;
    const std::vector<double> &pe = sph ? g->h_e[2] : g->h_e[1];
    int nphi = g->nphi;
    std::vector<double> cp(nphi), sp(nphi), cpm(nphi), spm(nphi);
    for (int k = 0; k < nphi; ++k) {
        double pm = 0.5 * (pe[k] + pe[k + 1]);
        cp[k] = std::cos(pe[k]);
        sp[k] = std::sin(pe[k]);
        cpm[k] = std::cos(pm);
        spm[k] = std::sin(pm);
    }
    std::vector<double> ct, ctm, stm;
    if (sph) {
        ct.resize(g->n2 + 1);
        ctm.resize(g->n2);
        stm.resize(g->n2);
        for (int j = 0; j <= g->n2; ++j) ct[j] = std::cos(g->h_e[1][j]);
        for (int j = 0; j < g->n2; ++j) {
            double tm = 0.5 * (g->h_e[1][j] + g->h_e[1][j + 1]);
            ctm[j] = std::cos(tm);
            stm[j] = std::sin(tm);
        }
    } else {
        ct.assign(1, 0.0);
        ctm.assign(1, 0.0);
        stm.assign(1, 0.0);
    }
    auto up = [&](const std::vector<double> &h, const double **out) -> int {
        double *p = nullptr;
        RCK(dalloc(g, &p, h.size()));
        CK(cudaMemcpyAsync(p, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, g->st));
        *out = p;
        return RT_OK;
    };
    RCK(up(g->h_e[0], &g->G.e1));
    RCK(up(g->h_e[1], &g->G.e2));
    RCK(up(g->h_e[2], &g->G.e3));
    RCK(up(ct, &g->G.ct));
    RCK(up(ctm, &g->G.ctm));
    RCK(up(stm, &g->G.stm));
    RCK(up(cp, &g->G.cp));
    RCK(up(sp, &g->G.sp));
    RCK(up(cpm, &g->G.cpm));
    RCK(up(spm, &g->G.spm));
    const double *pd = nullptr, *pw = nullptr;
    RCK(up(g->h_dirs, &pd));
    RCK(up(g->h_wt, &pw));
    g->d_dirs = (double *)pd;
    g->d_wt = (double *)pw;
    g->G.coord = g->coord;
    g->G.n1 = g->n1;
    g->G.n2 = g->n2;
    g->G.n3 = g->n3;
    g->G.nphi = g->nphi;
    g->G.inner_bc = g->inner_bc;
    g->G.nvox = g->nvox;
    return RT_OK;
}

// Launch set, crossing lists and ownership lists of every solid angle.
// Library-wide: grids created from now on complete their launch sets with the
// float-guided completion (RT_TUNE_GEOM_PREDICT on a NULL grid).
int g_geom_predict = 0;

// Float copies of the geometry tables for the guided completion, on the device
// (freed by the caller through dfree).
int upload_tables_f(rt_grid *g, GeomF &F, std::vector<void *> &owned)
{
    const bool sph = g->coord == RT_SPHERICAL;
    const std::vector<double> &pe = sph ? g->h_e[2] : g->h_e[1];
    const int nphi = g->nphi;
    std::vector<float> cp(nphi), sp(nphi), cpm(nphi), spm(nphi), ct(1, 0.0f), ctm(1, 0.0f), stm(1, 0.0f);
    for (int k = 0; k < nphi; ++k) {
        const double pm = 0.5 * (pe[k] + pe[k + 1]);
        cp[k] = (float)std::cos(pe[k]);
        sp[k] = (float)std::sin(pe[k]);
        cpm[k] = (float)std::cos(pm);
        spm[k] = (float)std::sin(pm);
    }
    if (sph) {
        ct.resize(g->n2 + 1);
        ctm.resize(g->n2);
        stm.resize(g->n2);
        for (int j = 0; j <= g->n2; ++j) ct[j] = (float)std::cos(g->h_e[1][j]);
        for (int j = 0; j < g->n2; ++j) {
            const double tm = 0.5 * (g->h_e[1][j] + g->h_e[1][j + 1]);
            ctm[j] = (float)std::cos(tm);
            stm[j] = (float)std::sin(tm);
        }
    }
    std::vector<float> e1(g->h_e[0].begin(), g->h_e[0].end()), e3(g->h_e[2].begin(), g->h_e[2].end());
    auto up = [&](const std::vector<float> &h, const float **out) -> int {
        float *p = nullptr;
        RCK(dalloc(g, &p, h.size()));
        owned.push_back(p);
        CK(cudaMemcpyAsync(p, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, g->st));
        *out = p;
        return RT_OK;
    };
    RCK(up(e1, &F.e1));
    RCK(up(e3, &F.e3));
    RCK(up(ct, &F.ct));
    RCK(up(ctm, &F.ctm));
    RCK(up(stm, &F.stm));
    RCK(up(cp, &F.cp));
    RCK(up(sp, &F.sp));
    RCK(up(cpm, &F.cpm));
    RCK(up(spm, &F.spm));
    F.coord = g->coord;
    F.n1 = g->n1;
    F.n2 = g->n2;
    F.n3 = g->n3;
    F.nphi = g->nphi;
    F.inner_bc = g->inner_bc;
    F.nvox = g->nvox;
    return RT_OK;
}

int build_geometry(rt_grid *g)
{
    auto t0 = std::chrono::steady_clock::now();
    const int nvox = g->nvox, n_ang = g->n_ang;
    const int words = (nvox + 31) / 32;
    RCK(dalloc(g, &g->d_lost, 1));
    CK(cudaMemsetAsync(g->d_lost, 0, sizeof(int), g->st));
    uint32_t *comp = nullptr;
    RCK(dalloc(g, &comp, (size_t)n_ang * words));
    CK(cudaMemsetAsync(comp, 0, sizeof(uint32_t) * (size_t)n_ang * words, g->st));
    // launch set: boundary marks, then serial-order coverage completion, in angle chunks
    const int cap = geom_scratch_cap(g->G);
    const bool guided = g_geom_predict != 0;
    const int64_t per_angle =
        (int64_t)words * 4 + (int64_t)32 * cap * 4 + (guided ? (int64_t)32 * cap * 4 + (int64_t)nvox * 4 : 0);
    int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(n_ang, ((int64_t)1 << 31) / per_angle));
    uint32_t *hit = nullptr;
    int32_t *scratch = nullptr, *pscr = nullptr, *stamp = nullptr;
    RCK(dalloc(g, &hit, (size_t)chunk * words));
    RCK(dalloc(g, &scratch, (size_t)chunk * 32 * cap));
    GeomF F{};
    std::vector<void *> ftab;
    if (guided) {
        RCK(dalloc(g, &pscr, (size_t)chunk * 32 * cap));
        RCK(dalloc(g, &stamp, (size_t)chunk * nvox));
        RCK(upload_tables_f(g, F, ftab));
    }
    // walk counts of every launched characteristic (n_ang x n_vox), recorded by the launch-set passes
    uint32_t *wcnt = nullptr;
    RCK(dalloc(g, &wcnt, (size_t)n_ang * nvox));
    for (int w0 = 0; w0 < n_ang; w0 += chunk) {
        int nw = std::min(chunk, n_ang - w0);
        CK(cudaMemsetAsync(hit, 0, sizeof(uint32_t) * (size_t)nw * words, g->st));
        CK(geom_mark_boundary(g->G, g->d_dirs, w0, nw, hit, words, g->d_lost, wcnt, g->st));
        if (guided) {
            CK(cudaMemsetAsync(stamp, 0, sizeof(int32_t) * (size_t)nw * nvox, g->st));
            CK(geom_complete_pred(g->G, F, g->d_dirs, w0, nw, hit, comp + (size_t)w0 * words, words, scratch, pscr,
                                  stamp, cap, g->d_lost, wcnt, g->st));
        } else {
            CK(geom_complete(g->G, g->d_dirs, w0, nw, hit, comp + (size_t)w0 * words, words, scratch, cap, g->d_lost,
                             wcnt, g->st));
        }
    }
    dfree(g, hit);
    dfree(g, scratch);
    dfree(g, pscr);
    dfree(g, stamp);
    for (void *p : ftab) dfree(g, p);
    // ordered ray lists
    int32_t *counts = nullptr;
    RCK(dalloc(g, &counts, n_ang));
    CK(geom_count_rays(g->G, g->d_dirs, n_ang, comp, words, counts, g->st));
    std::vector<int32_t> hc(n_ang);
    CK(cudaMemcpyAsync(hc.data(), counts, sizeof(int32_t) * n_ang, cudaMemcpyDeviceToHost, g->st));
    RCK(sync(g));
    g->h_ang_ray_off.assign(n_ang + 1, 0);
    for (int w = 0; w < n_ang; ++w) g->h_ang_ray_off[w + 1] = g->h_ang_ray_off[w] + hc[w];
    g->n_rays = g->h_ang_ray_off[n_ang];
    int64_t *d_aro = nullptr;
    RCK(dalloc(g, &d_aro, n_ang + 1));
    CK(cudaMemcpyAsync(d_aro, g->h_ang_ray_off.data(), sizeof(int64_t) * (n_ang + 1), cudaMemcpyHostToDevice, g->st));
    RCK(dalloc(g, &g->d_ray_origin, g->n_rays));
    RCK(dalloc(g, &g->d_ray_angle, g->n_rays));
    CK(geom_list_rays(g->G, g->d_dirs, n_ang, comp, words, d_aro, g->d_ray_origin, g->d_ray_angle, g->st));
    dfree(g, comp);
    dfree(g, counts);
    // segment counts, offsets, lists
    int32_t *nseg = nullptr, *nback = nullptr;
    RCK(dalloc(g, &nseg, g->n_rays));
    RCK(dalloc(g, &nback, g->n_rays));
    CK(geom_gather_counts(nvox, g->n_rays, g->d_ray_origin, g->d_ray_angle, wcnt, nseg, nback, g->st));
    dfree(g, wcnt);
    RCK(dalloc(g, &g->d_ray_off, g->n_rays + 1));
    int64_t *tmp = nullptr;
    RCK(dalloc(g, &tmp, scan_tmp_elems(g->n_rays)));
    CK(scan_i32(nseg, g->d_ray_off, g->n_rays, tmp, g->st));
    dfree(g, tmp);
    CK(cudaMemcpyAsync(&g->n_seg, g->d_ray_off + g->n_rays, sizeof(int64_t), cudaMemcpyDeviceToHost, g->st));
    RCK(sync(g));
    dfree(g, nseg);
    RCK(dalloc(g, &g->d_vox, g->n_seg + 4));  // 4 words of padding: 16-byte bulk-copy windows
    RCK(dalloc(g, &g->d_len64, g->n_seg));
    RCK(dalloc(g, &g->d_len32, g->n_seg));
    CK(cudaMemsetAsync(g->d_vox, 0, sizeof(uint32_t) * (size_t)g->n_seg, g->st));
    CK(geom_write_segs(g->G, g->d_dirs, g->n_rays, g->d_ray_origin, g->d_ray_angle, g->d_ray_off, nback, g->d_vox,
                       g->d_len64, g->d_len32, g->d_lost, g->st));
    dfree(g, nback);
    // segment offsets of every solid angle
    RCK(dalloc(g, &g->d_ang_seg_off, n_ang + 1));
    CK(gather_i64(g->d_ray_off, d_aro, g->d_ang_seg_off, n_ang + 1, g->st));
    g->h_ang_seg_off.assign(n_ang + 1, 0);
    CK(cudaMemcpyAsync(g->h_ang_seg_off.data(), g->d_ang_seg_off, sizeof(int64_t) * (n_ang + 1),
                       cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(&g->lost, g->d_lost, sizeof(int), cudaMemcpyDeviceToHost, g->st));
    RCK(sync(g));
    g->geom_trace_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    dfree(g, d_aro);
    // angle blocks sized so one block's per-segment results stay in L2
    double avg = (double)g->n_seg / n_ang;
    int ablk = g->ablk;
    if (ablk <= 0) ablk = (int)std::max(1.0, std::min((double)BLOCK_SEG_TARGET / std::max(avg, 1.0), (double)MAX_BLOCK_ANGLES));
    ablk = std::min(ablk, n_ang);
    g->ablk = ablk;
    g->blk_w0.clear();
    g->blk_nw.clear();
    g->max_blk_seg = 0;
    for (int w0 = 0; w0 < n_ang; w0 += ablk) {
        int nw = std::min(ablk, n_ang - w0);
        g->blk_w0.push_back(w0);
        g->blk_nw.push_back(nw);
        int64_t ns = g->h_ang_seg_off[w0 + nw] - g->h_ang_seg_off[w0];
        if (ns >= ((int64_t)1 << 31)) return fail(RT_EINVAL, "angle block %d holds too many segments; lower angle_block", w0);
        g->max_blk_seg = std::max(g->max_blk_seg, ns);
    }
    g->nblk = (int)g->blk_w0.size();
    // ownership (CSR) lists and inverse path lengths per (angle, voxel)
    RCK(dalloc(g, &g->d_csr_off, (size_t)g->nblk * (nvox + 1)));
    RCK(dalloc(g, &g->d_perm, g->n_seg));
    RCK(dalloc(g, &g->d_invL, (size_t)n_ang * nvox));
    int32_t *cnt = nullptr;
    int64_t *ctmp = nullptr;
    RCK(dalloc(g, &cnt, nvox));
    RCK(dalloc(g, &ctmp, (nvox + 1) + scan_tmp_elems(nvox)));
    // radix-sort scratch, freed once the lists are built
    RadixScratch rs{};
    rs.cap = std::max<int64_t>(1, g->max_blk_seg);
    const int64_t nhist = 256 * radix_tiles(rs.cap);
    std::vector<void *> rtmp;
    auto talloc = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMalloc(&q, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        rtmp.push_back(q);
        return q;
    };
    rs.kA = (uint32_t *)talloc(4 * (size_t)rs.cap);
    rs.kB = (uint32_t *)talloc(4 * (size_t)rs.cap);
    rs.vA = (int32_t *)talloc(4 * (size_t)rs.cap);
    rs.vB = (int32_t *)talloc(4 * (size_t)rs.cap);
    rs.hist = (int32_t *)talloc(4 * (size_t)nhist);
    rs.off = (int64_t *)talloc(8 * (size_t)(nhist + 1));
    rs.tmp = (int64_t *)talloc(8 * (size_t)scan_tmp_elems(nhist));
    struct Free {
        std::vector<void *> &v;
        ~Free()
        {
            for (void *q : v) cudaFree(q);
        }
    } free_rtmp{rtmp};
    if (!rs.kA || !rs.kB || !rs.vA || !rs.vB || !rs.hist || !rs.off || !rs.tmp)
        return fail(RT_ENOMEM, "ownership-list sort scratch could not be allocated");
    RCK(dalloc(g, &g->d_ufirst, (size_t)g->nblk * (nvox + 1)));
    g->h_ubase.assign(g->nblk + 1, 0);
    g->h_nunits.assign(g->nblk, 0);
    for (int b = 0; b < g->nblk; ++b) {
        int w0 = g->blk_w0[b], nw = g->blk_nw[b];
        int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
        int32_t *off = g->d_csr_off + (size_t)b * (nvox + 1);
        CK(csr_build(nvox, g->d_vox + lo, ns, cnt, off, g->d_perm + lo, ctmp, rs, g->st));
        CK(csr_invL(nvox, off, g->d_perm + lo, g->d_len64 + lo, g->d_ang_seg_off, w0, nw, lo, g->d_invL, g->st));
        int64_t *uf = g->d_ufirst + (size_t)b * (nvox + 1);
        CK(gather_units_build(nvox, off, cnt, uf, ctmp, g->st));
        CK(cudaMemcpyAsync(&g->h_nunits[b], uf + nvox, sizeof(int64_t), cudaMemcpyDeviceToHost, g->st));
    }
    RCK(sync(g));
    g->geom_lists_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() -
                       g->geom_trace_ms;
    int64_t max_units = 0;
    for (int b = 0; b < g->nblk; ++b) {
        g->h_ubase[b + 1] = g->h_ubase[b] + g->h_nunits[b];
        max_units = std::max(max_units, g->h_nunits[b]);
    }
    // voxels whose ownership list spans several units, per block
    {
        int32_t *flag = nullptr;
        int64_t *pos = nullptr, *stmp = nullptr;
        RCK(dalloc(g, &flag, nvox));
        RCK(dalloc(g, &pos, (size_t)g->nblk * (nvox + 1)));
        RCK(dalloc(g, &stmp, scan_tmp_elems(nvox)));
        std::vector<int64_t> nm(g->nblk);
        for (int b = 0; b < g->nblk; ++b) {
            int64_t *pb = pos + (size_t)b * (nvox + 1);
            CK(gather_multi_rows(nvox, g->d_ufirst + (size_t)b * (nvox + 1), flag, pb, stmp, nullptr, g->st));
            CK(cudaMemcpyAsync(&nm[b], pb + nvox, sizeof(int64_t), cudaMemcpyDeviceToHost, g->st));
        }
        RCK(sync(g));
        g->h_mbase.assign(g->nblk + 1, 0);
        for (int b = 0; b < g->nblk; ++b) g->h_mbase[b + 1] = g->h_mbase[b] + nm[b];
        RCK(dalloc(g, &g->d_multi, std::max<int64_t>(1, g->h_mbase[g->nblk])));
        for (int b = 0; b < g->nblk; ++b)
            CK(gather_multi_rows(nvox, g->d_ufirst + (size_t)b * (nvox + 1), flag, pos + (size_t)b * (nvox + 1), stmp,
                                 g->d_multi + g->h_mbase[b], g->st));
        RCK(sync(g));
        dfree(g, flag);
        dfree(g, pos);
        dfree(g, stmp);
    }
    RCK(dalloc(g, &g->d_wL32, (size_t)n_ang * nvox));
    CK(make_wL32(n_ang, nvox, g->d_invL, g->d_wt, g->d_wL32, g->st));
    RCK(dalloc(g, &g->d_urow, g->h_ubase[g->nblk]));
    RCK(dalloc(g, &g->d_ubeg, g->h_ubase[g->nblk]));
    RCK(dalloc(g, &g->d_part, 5 * (size_t)max_units));
    for (int b = 0; b < g->nblk; ++b) {
        const int32_t *off = g->d_csr_off + (size_t)b * (nvox + 1);
        CK(gather_units_fill(nvox, off, g->d_ufirst + (size_t)b * (nvox + 1), g->d_urow + g->h_ubase[b],
                             g->d_ubeg + g->h_ubase[b], g->st));
    }
    RCK(sync(g));
    // sliced-ELL layout of every block's work units
    {
        const int64_t U = g->h_ubase[g->nblk];
        RCK(dalloc(g, &g->d_ulen, std::max<int64_t>(1, U)));
        RCK(dalloc(g, &g->d_order, std::max<int64_t>(1, U)));
        g->h_goff.assign(g->nblk + 1, 0);
        int64_t maxg = 0;
        for (int b = 0; b < g->nblk; ++b) {
            int64_t ng = (g->h_nunits[b] + 31) / 32;
            g->h_goff[b + 1] = g->h_goff[b] + ng + 1;
            maxg = std::max(maxg, ng);
        }
        RCK(dalloc(g, &g->d_gbase, g->h_goff[g->nblk]));
        int32_t *hist = nullptr, *gw = nullptr;
        int64_t *stmp = nullptr;
        RCK(dalloc(g, &hist, 64));
        RCK(dalloc(g, &gw, std::max<int64_t>(1, maxg)));
        RCK(dalloc(g, &stmp, scan_tmp_elems(std::max<int64_t>(1, maxg))));
        std::vector<int64_t> tot(g->nblk, 0);
        for (int b = 0; b < g->nblk; ++b) {
            const int64_t u0 = g->h_ubase[b], nu = g->h_nunits[b], ng = (nu + 31) / 32;
            const int32_t *off = g->d_csr_off + (size_t)b * (nvox + 1);
            CK(sell_order(nu, g->d_urow + u0, g->d_ubeg + u0, off, g->d_ulen + u0, hist, g->d_order + u0, gw, g->st));
            CK(scan_i32(gw, g->d_gbase + g->h_goff[b], ng, stmp, g->st));
            CK(cudaMemcpyAsync(&tot[b], g->d_gbase + g->h_goff[b] + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, g->st));
        }
        RCK(sync(g));
        g->h_soff.assign(g->nblk + 1, 0);
        for (int b = 0; b < g->nblk; ++b) g->h_soff[b + 1] = g->h_soff[b] + tot[b];
        RCK(dalloc(g, &g->d_sell, std::max<int64_t>(1, g->h_soff[g->nblk])));
        for (int b = 0; b < g->nblk; ++b) {
            const int w0 = g->blk_w0[b];
            const int64_t u0 = g->h_ubase[b], lo = g->h_ang_seg_off[w0];
            CK(sell_fill(g->h_nunits[b], g->d_order + u0, g->d_ulen + u0, g->d_ubeg + u0, g->d_perm + lo,
                         g->d_gbase + g->h_goff[b], g->d_sell + g->h_soff[b], g->st));
        }
        RCK(sync(g));
        dfree(g, hist);
        dfree(g, gw);
        dfree(g, stmp);
    }
    // J-only gather tables: short lists in a sliced-ELL copy, long lists in chunks
    {
        int32_t *hist = nullptr, *lflag = nullptr, *nch = nullptr, *gw = nullptr;
        int64_t *lpos = nullptr, *cpos = nullptr, *stmp = nullptr;
        RCK(dalloc(g, &hist, 128));
        RCK(dalloc(g, &lflag, nvox));
        RCK(dalloc(g, &nch, nvox));
        RCK(dalloc(g, &gw, (nvox + 31) / 32 + 1));
        RCK(dalloc(g, &lpos, nvox + 1));
        RCK(dalloc(g, &cpos, nvox + 1));
        RCK(dalloc(g, &stmp, scan_tmp_elems(nvox + 1)));
        g->jt.assign(g->nblk, GatherJTables());
        int64_t max_chunks = 1;
        for (int b = 0; b < g->nblk; ++b) {
            const int w0 = g->blk_w0[b];
            const int64_t lo = g->h_ang_seg_off[w0];
            const int32_t *off = g->d_csr_off + (size_t)b * (nvox + 1);
            GatherJTables &t = g->jt[b];
            CK(gatherJ_classify(nvox, off, hist, lflag, nch, g->st));
            std::vector<int32_t> hh(65);
            CK(cudaMemcpyAsync(hh.data(), hist, sizeof(int32_t) * 65, cudaMemcpyDeviceToHost, g->st));
            RCK(sync(g));
            int64_t nshort = 0;
            for (int q = 0; q < 65; ++q) nshort += hh[q];
            t.nshort = nshort;
            int32_t *jorder = nullptr, *jsell = nullptr;
            int64_t *jgbase = nullptr;
            const int64_t ng = (nshort + 31) / 32;
            RCK(dalloc(g, &jorder, std::max<int64_t>(1, nshort)));
            RCK(dalloc(g, &jgbase, ng + 1));
            CK(gatherJ_short(nvox, off, hist, jorder, nshort, gw, g->st));
            CK(scan_i32(gw, jgbase, ng, stmp, g->st));
            int64_t nsell = 0;
            CK(cudaMemcpyAsync(&nsell, jgbase + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, g->st));
            RCK(sync(g));
            RCK(dalloc(g, &jsell, std::max<int64_t>(1, nsell)));
            CK(gatherJ_sell(nshort, off, jorder, g->d_perm + lo, jgbase, jsell, g->st));
            t.jorder = jorder;
            t.jgbase = jgbase;
            t.jsell = jsell;
            // long lists
            CK(scan_i32(lflag, lpos, nvox, stmp, g->st));
            CK(scan_i32(nch, cpos, nvox, stmp, g->st));
            int64_t tots[2] = {0, 0};
            CK(cudaMemcpyAsync(&tots[0], lpos + nvox, sizeof(int64_t), cudaMemcpyDeviceToHost, g->st));
            CK(cudaMemcpyAsync(&tots[1], cpos + nvox, sizeof(int64_t), cudaMemcpyDeviceToHost, g->st));
            RCK(sync(g));
            t.nlong = (int)tots[0];
            t.nchunks = tots[1];
            int32_t *lrows = nullptr, *lfirst = nullptr, *crow = nullptr, *cbeg = nullptr, *clr = nullptr;
            int *cnt = nullptr;
            RCK(dalloc(g, &lrows, std::max<int64_t>(1, tots[0])));
            RCK(dalloc(g, &lfirst, std::max<int64_t>(1, tots[0])));
            RCK(dalloc(g, &cnt, std::max<int64_t>(1, tots[0])));
            RCK(dalloc(g, &crow, std::max<int64_t>(1, tots[1])));
            RCK(dalloc(g, &cbeg, std::max<int64_t>(1, tots[1])));
            RCK(dalloc(g, &clr, std::max<int64_t>(1, tots[1])));
            CK(cudaMemsetAsync(cnt, 0, sizeof(int) * std::max<int64_t>(1, tots[0]), g->st));
            CK(gatherJ_long(nvox, off, lflag, lpos, cpos, lrows, lfirst, crow, cbeg, clr, g->st));
            t.lfirst = lfirst;
            t.crow = crow;
            t.cbeg = cbeg;
            t.clr = clr;
            t.cnt = cnt;
            max_chunks = std::max(max_chunks, tots[1]);
        }
        RCK(dalloc(g, &g->d_partJ, max_chunks));
        RCK(sync(g));
        dfree(g, hist);
        dfree(g, lflag);
        dfree(g, nch);
        dfree(g, gw);
        dfree(g, lpos);
        dfree(g, cpos);
        dfree(g, stmp);
    }
    dfree(g, cnt);
    dfree(g, ctmp);
    g->geom_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return RT_OK;
}

int alloc_fields(rt_grid *g)
{
    const int n = g->nvox;
    RCK(dalloc(g, &g->d_chi, n));
    RCK(dalloc(g, &g->d_eps, n));
    RCK(dalloc(g, &g->d_B, n));
    RCK(dalloc(g, &g->d_S, n));
    RCK(dalloc(g, &g->d_J, n));
    RCK(dalloc(g, &g->d_L, n));
    RCK(dalloc(g, &g->d_Fc, 3 * (size_t)n));
    RCK(dalloc(g, &g->d_F, 3 * (size_t)n));
    RCK(dalloc(g, &g->d_cs64, n));
    RCK(dalloc(g, &g->d_cs32, n));
    if (g->use_lstar == RT_LSTAR_NN) {
        RCK(dalloc(g, &g->d_L27, 27 * (size_t)n));
        RCK(dalloc(g, &g->d_nnx, (size_t)nn_os_work_elems(n)));  // OS-step solve work space
        RCK(dalloc(g, &g->d_nny, n));
        RCK(dalloc(g, &g->d_nnmx, 2));
    }
    RCK(dalloc(g, &g->d_B32, n));
    RCK(dalloc(g, &g->d_S32, n));
    RCK(dalloc(g, &g->d_H, 4 * (size_t)n));
    RCK(dalloc(g, &g->d_ng_part, ng_partial_elems(n)));
    RCK(dalloc(g, &g->d_ng_coef, 4));
    RCK(dalloc(g, &g->d_maxrel, 1));
    RCK(dalloc(g, &g->d_err, 1));
    CK(cudaMemsetAsync(g->d_err, 0, sizeof(int), g->st));
    RCK(dalloc(g, &g->d_r, n));
    RCK(dalloc(g, &g->d_delta, n));
    RCK(dalloc(g, &g->d_Jd, n));
    RCK(dalloc(g, &g->d_Ld, n));
    RCK(dalloc(g, &g->d_Fcd, 3 * (size_t)n));
    RCK(dalloc(g, &g->d_Lkeep, n));
    void *seg = nullptr;
    cudaError_t e = cudaMalloc(&seg, sizeof(double2) * (size_t)std::max<int64_t>(1, g->max_blk_seg));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RT_ENOMEM, "segment buffer allocation failed");
    }
    g->allocs.push_back(seg);
    g->bytes += (int64_t)(sizeof(double2) * (size_t)std::max<int64_t>(1, g->max_blk_seg));
    g->d_segbuf = seg;
    CK(cudaMallocHost((void **)&g->h_pin, 8 * sizeof(double)));
    CK(fill_const(n, g->d_chi, 1.0, g->st));
    CK(fill_const(n, g->d_eps, 1.0, g->st));
    CK(fill_const(n, g->d_B, 0.0, g->st));
    CK(fill_const(n, g->d_S, 0.0, g->st));
    CK(fill_const(n, g->d_J, 0.0, g->st));
    CK(fill_const(n, g->d_L, 0.0, g->st));
    CK(fill_const(3 * n, g->d_F, 0.0, g->st));
    CK(mark_parabola(g->d_vox, g->d_len64, g->d_chi, g->n_seg, g->interp == RT_PARABOLIC, g->st));
    return RT_OK;
}

// Formal solution of every angle block with the FP64 or FP32 march.
int run_fs(rt_grid *g, int prec, int homog, const double *S_src, double *J, double *L, double *Fc, double *F)
{
    const int n = g->nvox;
    const int para = g->interp == RT_PARABOLIC;
    if (prec == RT_FP64) CK(pack_chiS64(n, g->d_chi, S_src, g->d_cs64, g->st));
    else CK(pack_chiS32(n, g->d_chi, S_src, g->d_B, g->d_cs32, g->d_B32, g->d_S32, g->st));
    g->launches++;
    for (int b = 0; b < g->nblk; ++b) {
        int w0 = g->blk_w0[b], nw = g->blk_nw[b];
        int64_t r_lo = g->h_ang_ray_off[w0], r_hi = g->h_ang_ray_off[w0 + nw];
        int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
        const int32_t *off = g->d_csr_off + (size_t)b * (n + 1);
        int t0, t1;
        if (prec == RT_FP64) {
            double2 *buf = (double2 *)g->d_segbuf;
            t0 = tstart(g, 0);
            CK(march_block<double, double2>(g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs64, g->d_B,
                                            g->I_outer, homog, para, buf, g->march_chunk, g->st));
            tstop(g, t0, 0, ns, 12 * ns);
            t1 = tstart(g, 1);
            CK(gather_block<double2>(n, off, g->d_perm + lo, buf, g->d_ang_seg_off, w0, nw, lo, g->d_invL, g->d_wL32,
                                     g->d_wt, g->d_dirs, g->d_urow + g->h_ubase[b], g->d_ubeg + g->h_ubase[b],
                                     g->d_ufirst + (size_t)b * (n + 1), g->h_nunits[b], g->d_multi + g->h_mbase[b],
                                     (int)(g->h_mbase[b + 1] - g->h_mbase[b]), g->d_order + g->h_ubase[b],
                                     g->d_ulen + g->h_ubase[b], g->d_gbase + g->h_goff[b], g->d_sell + g->h_soff[b],
                                     g->d_part, J, L, Fc, b == 0, g->st));
            tstop(g, t1, 1, ns);
        } else {
            float2 *buf = (float2 *)g->d_segbuf;
            t0 = tstart(g, 0);
            CK(march_block<float, float2>(g->d_vox, g->d_len32, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs32, g->d_B32,
                                          (float)g->I_outer, homog, para, buf, g->march_chunk, g->st));
            tstop(g, t0, 0, ns, 8 * ns);
            t1 = tstart(g, 1);
            CK(gather_block<float2>(n, off, g->d_perm + lo, buf, g->d_ang_seg_off, w0, nw, lo, g->d_invL, g->d_wL32,
                                    g->d_wt, g->d_dirs, g->d_urow + g->h_ubase[b], g->d_ubeg + g->h_ubase[b],
                                     g->d_ufirst + (size_t)b * (n + 1), g->h_nunits[b], g->d_multi + g->h_mbase[b],
                                     (int)(g->h_mbase[b + 1] - g->h_mbase[b]), g->d_order + g->h_ubase[b],
                                     g->d_ulen + g->h_ubase[b], g->d_gbase + g->h_goff[b], g->d_sell + g->h_soff[b],
                                     g->d_part, J, L, Fc, b == 0, g->st));
            tstop(g, t1, 1, ns);
        }
        g->launches += 3;
    }
    if (F) {
        CK(flux_local(g->G, Fc, F, g->st));
        g->launches++;
    }
    return RT_OK;
}

// Streamed-weight march: allocate its per-segment arrays on first use (w l / L
// computed then, from the geometry) and refresh (E, alpha, beta, gamma) after
// chi changed.  Returns false when disabled or when the arrays do not fit; the
// FP32 march then evaluates the weights itself.
// Streamed-weight march, parts shared by both precisions: list positions
// (optional; without them the gather reads through perm) and the bundle bounds
// of the current chunk.  Returns false when they cannot be set up.
bool sw_common(rt_grid *g)
{
    if (g->pos_state == 0) {
        void *c = nullptr;
        if (cudaMalloc(&c, sizeof(int32_t) * (size_t)(g->n_seg + 4)) == cudaSuccess) {
            g->allocs.push_back(c);
            g->bytes += (int64_t)(4 * g->n_seg);
            g->d_pos = (int32_t *)c;
            for (int b = 0; b < g->nblk; ++b) {
                const int64_t lo = g->h_ang_seg_off[g->blk_w0[b]];
                const int64_t ns = g->h_ang_seg_off[g->blk_w0[b] + g->blk_nw[b]] - lo;
                if (inv_perm(g->d_perm + lo, ns, g->d_pos + lo, g->st) != cudaSuccess) return false;
                g->launches++;
            }
            g->pos_state = 1;
        } else {
            cudaGetLastError();
            g->pos_state = -1;
        }
    }
    if (g->bnd_chunk != g->march_chunk) {  // bundle bounds for the current chunk
        std::vector<int64_t> off(g->nblk + 1, 0);
        for (int b = 0; b < g->nblk; ++b) {
            const int w0 = g->blk_w0[b], nw = g->blk_nw[b];
            const int64_t ns = g->h_ang_seg_off[w0 + nw] - g->h_ang_seg_off[w0];
            off[b + 1] = off[b] + (ns + g->march_chunk - 1) / g->march_chunk;
        }
        if (g->d_bnd) {
            cudaFree(g->d_bnd);
            for (auto &q : g->allocs)
                if (q == (void *)g->d_bnd) q = nullptr;
            g->d_bnd = nullptr;
        }
        void *q = nullptr;
        if (cudaMalloc(&q, sizeof(int2) * (size_t)std::max<int64_t>(1, off[g->nblk])) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        g->allocs.push_back(q);
        g->d_bnd = (int2 *)q;
        for (int b = 0; b < g->nblk; ++b) {
            const int w0 = g->blk_w0[b], nw = g->blk_nw[b];
            const int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
            if (sw_bundles(g->d_ray_off, g->h_ang_ray_off[w0], g->h_ang_ray_off[w0 + nw], lo, ns, g->march_chunk,
                           g->d_bnd + off[b], g->st) != cudaSuccess)
                return false;
            g->launches++;
        }
        g->h_bnd_off = off;
        g->bnd_chunk = g->march_chunk;
    }
    return true;
}

// FP32 streamed weights: allocated on first use (w l / L computed then, from the
// geometry), (E, alpha, beta, gamma) refreshed after chi changed.  false when
// disabled or out of memory (the FP32 march then evaluates the weights itself).
bool use_sw(rt_grid *g)
{
    if (!g->sw_enabled || g->sw_state < 0) return false;
    const int fold = g->sw_fold && g->sw_stages == 0;
    if (g->sw_state == 0) {
        void *a = nullptr;
        if (cudaMalloc(&a, sizeof(float4) * (size_t)g->n_seg) != cudaSuccess) {
            cudaGetLastError();
            g->sw_state = -1;
            return false;
        }
        g->allocs.push_back(a);
        g->bytes += (int64_t)(16 * g->n_seg);
        g->d_cw4 = (float4 *)a;
        g->sw_state = 1;
        g->cw_ok = false;
    }
    if (!fold && !g->d_cg) {  // the separate gather-weight stream of the unfolded march
        void *b = nullptr;
        if (cudaMalloc(&b, sizeof(float) * (size_t)(g->n_seg + 4)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        g->allocs.push_back(b);
        g->bytes += (int64_t)(4 * g->n_seg);
        g->d_cg = (float *)b;
        if (seg_weight(g->d_vox, g->d_len64, g->d_ang_seg_off, g->n_ang, g->d_wt, g->d_invL, g->nvox, g->n_seg, g->d_cg,
                       g->st) != cudaSuccess)
            return false;
        g->launches++;
    }
    if (!g->cw_ok || g->cw_fold != fold) {
        cudaError_t e = fold ? coef_stream_fold(g->d_vox, g->d_len64, g->d_chi, g->d_ang_seg_off, g->n_ang, g->d_wt,
                                                g->d_invL, g->nvox, g->n_seg, g->d_cw4, g->st)
                             : coef_stream(g->d_vox, g->d_len64, g->d_chi, g->n_seg, g->d_cw4, g->st);
        if (e != cudaSuccess) return false;
        g->launches++;
        g->cw_ok = true;
        g->cw_fold = fold;
    }
    return sw_common(g);
}

// FP64 streamed weights (40 bytes per segment), the same life cycle.
bool use_sw64(rt_grid *g)
{
    if (!g->sw_enabled || g->sw64_state < 0) return false;
    if (g->sw64_state == 0) {
        void *a = nullptr, *b = nullptr;
        if (cudaMalloc(&a, sizeof(Wd4) * (size_t)g->n_seg) != cudaSuccess ||
            cudaMalloc(&b, sizeof(double) * (size_t)(g->n_seg + 4)) != cudaSuccess) {
            cudaGetLastError();
            if (a) cudaFree(a);
            g->sw64_state = -1;
            return false;
        }
        g->allocs.push_back(a);
        g->allocs.push_back(b);
        g->bytes += (int64_t)(40 * g->n_seg);
        g->d_cw64 = (Wd4 *)a;
        g->d_cg64 = (double *)b;
        if (seg_weight64(g->d_vox, g->d_len64, g->d_ang_seg_off, g->n_ang, g->d_wt, g->d_invL, g->nvox, g->n_seg,
                         g->d_cg64, g->st) != cudaSuccess) {
            g->sw64_state = -1;
            return false;
        }
        g->launches++;
        g->sw64_state = 1;
        g->cw64_ok = false;
    }
    if (!g->cw64_ok) {
        if (coef_stream64(g->d_vox, g->d_len64, g->d_chi, g->n_seg, g->d_cw64, g->st) != cudaSuccess) return false;
        g->launches++;
        g->cw64_ok = true;
    }
    return sw_common(g);
}

// Blocked voxel order for the FP32 march's S lookups (once per grid): slots of
// 4 x 2 x 4 index blocks, 32 voxels (one 128-byte line of FP32 S) each.
bool build_sblk(rt_grid *g)
{
    if (g->sblk_state != 0) return g->sblk_state > 0;
    g->sblk_state = -1;
    const int n1 = g->n1, n2 = g->n2, n3 = g->n3;
    const int nbj = (n2 + 1) / 2, nbk = (n3 + 3) / 4, nbi = (n1 + 3) / 4;
    const int64_t nslot = (int64_t)nbi * nbj * nbk * 32;
    if (nslot > (int64_t)RTK_VOXMASK) return false;
    std::vector<int32_t> h(g->nvox);
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j)
            for (int k = 0; k < n3; ++k) {
                const int64_t blk = ((int64_t)(i / 4) * nbj + j / 2) * nbk + k / 4;
                h[((int64_t)i * n2 + j) * n3 + k] = (int32_t)(blk * 32 + ((i % 4) * 2 + j % 2) * 4 + k % 4);
            }
    void *a = nullptr, *b = nullptr, *c = nullptr, *d = nullptr;
    auto al = [&](void **q, size_t bytes) {
        if (cudaMalloc(q, bytes) != cudaSuccess) {
            cudaGetLastError();
            *q = nullptr;
            return false;
        }
        g->allocs.push_back(*q);
        g->bytes += (int64_t)bytes;
        return true;
    };
    if (!al(&a, sizeof(int32_t) * g->nvox) || !al(&b, sizeof(uint32_t) * (size_t)(g->n_seg + 4)) ||
        !al(&c, sizeof(float) * (size_t)nslot) || !al(&d, sizeof(float) * (size_t)nslot))
        return false;
    g->d_vblk = (int32_t *)a;
    g->d_voxb = (uint32_t *)b;
    g->d_S32b = (float *)c;
    g->d_B32b = (float *)d;
    if (cudaMemsetAsync(g->d_S32b, 0, sizeof(float) * nslot, g->st) != cudaSuccess ||
        cudaMemsetAsync(g->d_B32b, 0, sizeof(float) * nslot, g->st) != cudaSuccess ||
        cudaMemcpyAsync(g->d_vblk, h.data(), sizeof(int32_t) * g->nvox, cudaMemcpyHostToDevice, g->st) != cudaSuccess ||
        make_voxb(g->d_vox, g->n_seg, g->d_vblk, g->d_voxb, g->st) != cudaSuccess ||
        cudaStreamSynchronize(g->st) != cudaSuccess)  // h goes out of scope
        return false;
    g->launches++;
    g->sblk_state = 1;
    return true;
}

SwMarch sw_march(rt_grid *g, int b, int homog, float *out)
{
    SwMarch m{};
    if (b < 0 || b >= g->nblk) return m;  // nbundles = 0: no march part
    const int w0 = g->blk_w0[b];
    m.vox = g->d_vox;
    m.cw = g->d_cw4;
    m.cg = g->d_cg;
    m.bnd = g->d_bnd + g->h_bnd_off[b];
    m.pos = (g->sw_scatter && g->d_pos) ? g->d_pos : nullptr;
    m.stages = g->sw_stages;
    m.bulk = g->sw_bulk;
    m.lookahead = g->sw_lookahead;
    m.fold = g->sw_fold && g->sw_stages == 0;
    m.err = g->d_err;
    m.seg_lo = g->h_ang_seg_off[w0];
    m.nbundles = g->h_bnd_off[b + 1] - g->h_bnd_off[b];
    m.S = g->d_S32;
    m.B = g->d_B32;
    if (g->sblk && g->sblk_state == 1) {  // S lookups in the blocked order
        m.vox = g->d_voxb;
        m.S = g->d_S32b;
        m.B = g->d_B32b;
    }
    m.I_outer = (float)g->I_outer;
    m.homog = homog;
    m.out = out;
    return m;
}

SwMarch64 sw_march64(rt_grid *g, int b, int homog, double *out)
{
    SwMarch64 m{};
    const int w0 = g->blk_w0[b];
    m.vox = g->d_vox;
    m.cw = g->d_cw64;
    m.cg = g->d_cg64;
    m.bnd = g->d_bnd + g->h_bnd_off[b];
    m.pos = (g->sw_scatter && g->d_pos) ? g->d_pos : nullptr;
    m.seg_lo = g->h_ang_seg_off[w0];
    m.nbundles = g->h_bnd_off[b + 1] - g->h_bnd_off[b];
    m.S = nullptr;  // set by the caller (the S of this formal solution)
    m.B = g->d_B;
    m.I_outer = g->I_outer;
    m.homog = homog;
    m.out = out;
    return m;
}

SwGather sw_gather(rt_grid *g, int b, const float *buf, double *J)
{
    SwGather t{};
    if (b < 0 || b >= g->nblk) return t;  // nshort = nchunks = 0: no gather part
    const GatherJTables &jt = g->jt[b];
    t.off = g->d_csr_off + (size_t)b * (g->nvox + 1);
    t.jorder = jt.jorder;
    t.jsell = jt.jsell;
    t.jgbase = jt.jgbase;
    t.crow = jt.crow;
    t.cbeg = jt.cbeg;
    t.clr = jt.clr;
    t.lfirst = jt.lfirst;
    t.cnt = jt.cnt;
    t.perm = g->d_perm + g->h_ang_seg_off[g->blk_w0[b]];
    t.part = g->d_partJ;
    t.buf = buf;
    t.J = J;
    t.nshort = jt.nshort;
    t.nchunks = jt.nchunks;
    t.nbs = (jt.nshort + 255) / 256;
    t.nlong = jt.nlong;
    t.first = b == 0;
    return t;
}

// Streamed-weight J.  Overlapped: the march of block b writes buffer
// b % nbuf (nbuf = max(2, march streams)) and waits only for the gather of
// block b - nbuf, which read that buffer; the gathers run in block order on
// the second stream, each after its march, so J accumulates in the same order
// as without overlap.  With several march streams block b is marched on
// stream b % nms (the grid's stream first), so a march may begin while the
// previous one drains.
int run_fs_J_sw_streams(rt_grid *g, int prec, int homog, const double *S_src, double *J, cudaStream_t base);

int run_fs_J_sw(rt_grid *g, int prec, int homog, const double *S_src, double *J)
{
    const bool f64 = prec == RT_FP64;
    const bool scatter = g->sw_scatter && g->d_pos;
    // double (FP64) or up to triple (FP32) buffer of per-segment values: the
    // segment buffer holds 16 bytes per segment of the largest block
    float *b32[3] = {(float *)g->d_segbuf, (float *)g->d_segbuf + g->max_blk_seg,
                     (float *)g->d_segbuf + 2 * g->max_blk_seg};
    double *b64[2] = {(double *)g->d_segbuf, (double *)g->d_segbuf + g->max_blk_seg};
    const bool fold = !f64 && g->sw_fold && g->sw_stages == 0;  // no separate gather-weight stream
    const int64_t bps = (f64 ? (scatter ? 48 : 44) : (scatter ? 28 : 24)) - (fold ? 4 : 0);  // streamed bytes per segment
    auto segs = [&](int b) -> int64_t {
        return g->h_ang_seg_off[g->blk_w0[b] + g->blk_nw[b]] - g->h_ang_seg_off[g->blk_w0[b]];
    };
    auto march = [&](int b, int q, cudaStream_t st) -> cudaError_t {
        if (!f64) return march_sw_launch(sw_march(g, b, homog, b32[q]), g->sw_coarsen, st);
        SwMarch64 m = sw_march64(g, b, homog, b64[q]);
        m.S = S_src;
        return march_sw64_launch(m, g->sw64_coarsen, st);
    };
    auto gather = [&](int b, int q, cudaStream_t st) -> cudaError_t {
        SwGather t = sw_gather(g, b, b32[q], J);
        if (f64) {
            t.buf = nullptr;
            t.buf64 = b64[q];
        }
        return scatter ? gather_rows_sw_launch(t, g->nvox, st) : gather_sw_launch(t, st);
    };
    if (!g->sw_overlap) {
        if (!f64 && g->sblk && build_sblk(g)) {  // this step's FP32 S and B in the blocked order
            CK(blk_scatter(g->nvox, g->d_vblk, g->d_S32, g->d_B32, g->d_S32b, g->d_B32b, g->st));
            g->launches++;
        }
        for (int b = 0; b < g->nblk; ++b) {
            int t0 = tstart(g, 0);
            CK(march(b, 0, g->st));
            tstop(g, t0, 0, segs(b), bps * segs(b));
            t0 = tstart(g, 1);
            CK(gather(b, 0, g->st));
            tstop(g, t0, 1, segs(b));
            g->launches += 2;
        }
        return RT_OK;
    }
    if (!g->st2) {
        CK(cudaStreamCreateWithFlags(&g->st2, cudaStreamNonBlocking));
        for (cudaEvent_t &e : g->sev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (g->sw_graph && !g->timing) {
        rt_grid::FsGraph *f = nullptr;
        for (rt_grid::FsGraph &c : g->fsg)
            if (c.prec == prec && c.homog == homog && c.S == (const void *)S_src && c.J == (const void *)J) f = &c;
        if (!f) {  // take the least recently used entry for these arguments
            f = g->fsg[0].used <= g->fsg[1].used ? &g->fsg[0] : &g->fsg[1];
            if (f->exec) cudaGraphExecDestroy(f->exec);
            *f = rt_grid::FsGraph{};
            f->prec = prec;
            f->homog = homog;
            f->S = S_src;
            f->J = J;
        }
        f->used = ++g->fsg_tick;
        if (!f->exec && f->calls >= 1) {  // the first call ran directly: lazy set-up is done
            if (!g->stc) CK(cudaStreamCreateWithFlags(&g->stc, cudaStreamNonBlocking));
            const int64_t l0 = g->launches;
            cudaError_t ec = cudaStreamBeginCapture(g->stc, cudaStreamCaptureModeRelaxed);
            if (ec == cudaSuccess) {
                const int rc = run_fs_J_sw_streams(g, prec, homog, S_src, J, g->stc);
                cudaGraph_t graph = nullptr;
                ec = cudaStreamEndCapture(g->stc, &graph);
                f->launches = g->launches - l0;
                g->launches = l0;
                if (rc != RT_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return rc;
                }
                if (ec == cudaSuccess) ec = cudaGraphInstantiate(&f->exec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
            }
            if (ec != cudaSuccess) {  // no graph on this grid: the same launches, one by one
                cudaGetLastError();
                f->exec = nullptr;
                g->sw_graph = 0;
            }
        }
        f->calls++;
        if (f->exec) {
            CK(cudaGraphLaunch(f->exec, g->st));
            g->launches += f->launches;
            return RT_OK;
        }
    }
    return run_fs_J_sw_streams(g, prec, homog, S_src, J, g->st);
}

// The overlapped streamed-weight J on base stream `base` (the grid's stream, or
// the private stream the graph is captured on).
int run_fs_J_sw_streams(rt_grid *g, int prec, int homog, const double *S_src, double *J, cudaStream_t base)
{
    const bool f64 = prec == RT_FP64;
    const bool scatter = g->sw_scatter && g->d_pos;
    float *b32[3] = {(float *)g->d_segbuf, (float *)g->d_segbuf + g->max_blk_seg,
                     (float *)g->d_segbuf + 2 * g->max_blk_seg};
    double *b64[2] = {(double *)g->d_segbuf, (double *)g->d_segbuf + g->max_blk_seg};
    const bool fold = !f64 && g->sw_fold && g->sw_stages == 0;  // no separate gather-weight stream
    const int64_t bps = (f64 ? (scatter ? 48 : 44) : (scatter ? 28 : 24)) - (fold ? 4 : 0);  // streamed bytes per segment
    auto segs = [&](int b) -> int64_t {
        return g->h_ang_seg_off[g->blk_w0[b] + g->blk_nw[b]] - g->h_ang_seg_off[g->blk_w0[b]];
    };
    if (!f64 && g->sblk && build_sblk(g)) {  // this step's FP32 S and B in the blocked order
        CK(blk_scatter(g->nvox, g->d_vblk, g->d_S32, g->d_B32, g->d_S32b, g->d_B32b, base));
        g->launches++;
    }
    auto march = [&](int b, int q, cudaStream_t st) -> cudaError_t {
        if (!f64) return march_sw_launch(sw_march(g, b, homog, b32[q]), g->sw_coarsen, st);
        SwMarch64 m = sw_march64(g, b, homog, b64[q]);
        m.S = S_src;
        return march_sw64_launch(m, g->sw64_coarsen, st);
    };
    auto gather = [&](int b, int q, cudaStream_t st) -> cudaError_t {
        SwGather t = sw_gather(g, b, b32[q], J);
        if (f64) {
            t.buf = nullptr;
            t.buf64 = b64[q];
        }
        return scatter ? gather_rows_sw_launch(t, g->nvox, st) : gather_sw_launch(t, st);
    };
    // events: fork, join, march done and gather done per buffer, join of each extra march stream
    cudaEvent_t fork = g->sev[0], join = g->sev[1], *mdone = g->sev + 2, *gdone = g->sev + 5, *mjoin = g->sev + 8;
    const int nms = std::min(g->nblk, f64 ? std::min(g->sw_mstreams, 2) : g->sw_mstreams);
    const int nbuf = std::max(2, nms);  // a buffer per march that may run at once
    cudaStream_t ms[3] = {base, g->st3, g->st4};
    for (int q = 1; q < nms; ++q) {
        cudaStream_t &sq = q == 1 ? g->st3 : g->st4;
        if (!sq) CK(cudaStreamCreateWithFlags(&sq, cudaStreamNonBlocking));
        ms[q] = sq;
    }
    CK(cudaEventRecord(fork, base));
    CK(cudaStreamWaitEvent(g->st2, fork, 0));
    for (int q = 1; q < nms; ++q) CK(cudaStreamWaitEvent(ms[q], fork, 0));
    for (int b = 0; b < g->nblk; ++b) {
        const int q = b % nbuf;
        cudaStream_t s = ms[b % nms];
        if (b >= nbuf) CK(cudaStreamWaitEvent(s, gdone[q], 0));  // the gather that read buffer q
        int t0 = tstart(g, 0, s);
        CK(march(b, q, s));
        tstop(g, t0, 0, segs(b), bps * segs(b), s);
        CK(cudaEventRecord(mdone[q], s));
        CK(cudaStreamWaitEvent(g->st2, mdone[q], 0));
        t0 = tstart(g, 1, g->st2);
        CK(gather(b, q, g->st2));
        tstop(g, t0, 1, segs(b), 0, g->st2);
        CK(cudaEventRecord(gdone[q], g->st2));
        g->launches += 2;
    }
    CK(cudaEventRecord(join, g->st2));
    CK(cudaStreamWaitEvent(base, join, 0));
    for (int q = 1; q < nms; ++q) {
        CK(cudaEventRecord(mjoin[q - 1], ms[q]));
        CK(cudaStreamWaitEvent(base, mjoin[q - 1], 0));
    }
    return RT_OK;
}

// J-only formal solution (the ALI iteration reuses Lambda*, which depends on
// chi and the lengths but not on S).
int run_fs_J(rt_grid *g, int prec, int homog, const double *S_src, double *J)
{
    const int n = g->nvox;
    if (prec == RT_FP64) CK(pack_chiS64(n, g->d_chi, S_src, g->d_cs64, g->st));
    else CK(pack_chiS32(n, g->d_chi, S_src, g->d_B, g->d_cs32, g->d_B32, g->d_S32, g->st));
    g->launches++;
    if (prec == RT_MIXED && use_sw(g)) return run_fs_J_sw(g, prec, homog, S_src, J);
    if (prec == RT_FP64 && use_sw64(g)) return run_fs_J_sw(g, prec, homog, S_src, J);
    CK(cudaGetLastError());
    for (int b = 0; b < g->nblk; ++b) {
        int w0 = g->blk_w0[b], nw = g->blk_nw[b];
        int64_t r_lo = g->h_ang_ray_off[w0], r_hi = g->h_ang_ray_off[w0 + nw];
        int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
        const int32_t *off = g->d_csr_off + (size_t)b * (n + 1);
        int t0, t1;
        if (prec == RT_FP64) {
            double *buf = (double *)g->d_segbuf;
            t0 = tstart(g, 0);
            CK(march_block_J<double, double2>(g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs64, g->d_B,
                                              g->I_outer, homog, buf, g->march_chunk, g->st));
            tstop(g, t0, 0, ns, 12 * ns);
            t1 = tstart(g, 1);
            CK(gather_J<double>(n, off, g->jt[b], g->d_perm + lo, buf, g->d_ang_seg_off, w0, nw, lo, g->d_wL32,
                                g->d_invL, g->d_wt, g->d_partJ, J, b == 0, g->st));
            tstop(g, t1, 1, ns);
        } else {
            float *buf = (float *)g->d_segbuf;
            t0 = tstart(g, 0);
            CK(march_block_J<float, float2>(g->d_vox, g->d_len32, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs32,
                                            g->d_B32, (float)g->I_outer, homog, buf, g->march_chunk, g->st));
            tstop(g, t0, 0, ns, 8 * ns);
            t1 = tstart(g, 1);
            CK(gather_J<float>(n, off, g->jt[b], g->d_perm + lo, buf, g->d_ang_seg_off, w0, nw, lo, g->d_wL32,
                               g->d_invL, g->d_wt, g->d_partJ, J, b == 0, g->st));
            tstop(g, t1, 1, ns);
        }
        g->launches += 2;
    }
    return RT_OK;
}

// J of S for an ALI iteration: a full FS (J, Lambda*, flux) when Lambda* is not
// yet known for this chi at this precision, else the J-only FS.
int fs_iteration(rt_grid *g, int prec, const double *S_src, double *J)
{
    const bool lstar_ok = g->lstar_prec == RT_FP64 || (g->lstar_prec == RT_MIXED && prec == RT_MIXED);
    if (!g->use_lstar || lstar_ok) return run_fs_J(g, prec, 0, S_src, J);
    RCK(run_fs(g, prec, 0, S_src, J, g->d_L, g->d_Fc, g->d_F));
    g->lstar_prec = prec;
    return RT_OK;
}

int read_maxrel(rt_grid *g, double *rel)
{
    CK(cudaMemcpyAsync(g->h_pin, g->d_maxrel, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(g->h_pin + 2, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->st));
    RCK(sync(g));
    *rel = g->h_pin[0];  // the device word holds the bits of a non-negative double
    int err = 0;
    std::memcpy(&err, g->h_pin + 2, sizeof(int));
    if (err) {
        CK(cudaMemsetAsync(g->d_err, 0, sizeof(int), g->st));
        return fail(RT_ETIMEOUT, "a bounded wait in the staged ray march gave up; results of this step are invalid");
    }
    return RT_OK;
}

void reset_ng(rt_grid *g)
{
    for (int q = 0; q < 4; ++q) g->hs[q] = q;
    g->nh = 0;
}

double *ng_append_slot(rt_grid *g)
{
    if (g->nh == 4) {
        int t = g->hs[0];
        g->hs[0] = g->hs[1];
        g->hs[1] = g->hs[2];
        g->hs[2] = g->hs[3];
        g->hs[3] = t;
        g->nh = 3;
    }
    return g->d_H + (size_t)g->hs[g->nh] * g->nvox;
}

// After an iterate was written to the slot from ng_append_slot: extrapolate
// into `out` once four iterates are stored; clears the history if applied.
int ng_maybe(rt_grid *g, double *out, const double *wref)
{
    g->nh++;
    if (g->nh < 4) return RT_OK;
    const size_t n = g->nvox;
    CK(ng_extrapolate(g->nvox, g->d_H + g->hs[3] * n, g->d_H + g->hs[2] * n, g->d_H + g->hs[1] * n,
                      g->d_H + g->hs[0] * n, wref, g->d_ng_part, g->d_ng_coef, out, g->st));
    g->launches += 3;
    CK(cudaMemcpyAsync(g->h_pin + 1, g->d_ng_coef + 2, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    RCK(sync(g));
    if (g->h_pin[1] != 0.0) g->nh = 0;
    return RT_OK;
}

// Nearest-neighbour Lambda* of the current chi (FP64, once per chi): per
// angle block, a walker thread per characteristic and a per-voxel sum in list
// order; the diagonal is copied to d_L.
// The exact nearest-neighbour Lambda* of opacity chi (device, n_vox) with the
// parabola choices pbits (NULL: those marked in the crossing words for the
// grid's own chi) into L27 (device, 27 n_vox), on stream st; returns after the
// stream has drained.
int nn_lstar_into(rt_grid *g, const double *chi, const uint32_t *pbits, double *L27, cudaStream_t st)
{
    const int n = g->nvox;
    int8_t *slot = nullptr;
    double *val = nullptr, *part = nullptr;
    int64_t max_units = 1;
    for (int b = 0; b < g->nblk; ++b) max_units = std::max(max_units, g->h_nunits[b]);
    if (cudaMalloc(&slot, (size_t)RTK_NNW * std::max<int64_t>(1, g->max_blk_seg)) != cudaSuccess ||
        cudaMalloc(&val, sizeof(double) * RTK_NNW * std::max<int64_t>(1, g->max_blk_seg)) != cudaSuccess ||
        cudaMalloc(&part, sizeof(double) * 27 * (size_t)max_units) != cudaSuccess) {
        cudaGetLastError();
        if (slot) cudaFree(slot);
        if (val) cudaFree(val);
        return fail(RT_ENOMEM, "NN Lambda* work arrays could not be allocated");
    }
    struct Free {
        void *a, *b, *c;
        cudaStream_t st;
        ~Free()
        {
            cudaStreamSynchronize(st);  // no launch may still use them
            cudaFree(a);
            cudaFree(b);
            cudaFree(c);
        }
    } fr{slot, val, part, st};
    for (int b = 0; b < g->nblk; ++b) {
        const int w0 = g->blk_w0[b], nw = g->blk_nw[b];
        NnWalk a{};
        a.vox = g->d_vox;
        a.len64 = g->d_len64;
        a.ray_off = g->d_ray_off;
        a.ray_angle = g->d_ray_angle;
        a.r_lo = g->h_ang_ray_off[w0];
        a.r_hi = g->h_ang_ray_off[w0 + nw];
        a.seg_lo = g->h_ang_seg_off[w0];
        a.chi = chi;
        a.pbits = pbits;
        a.wt = g->d_wt;
        a.invL = g->d_invL;
        a.nvox = n;
        a.n2 = g->n2;
        a.n3 = g->n3;
        a.sph = g->coord == RT_SPHERICAL;
        a.slot = slot;
        a.val = val;
        CK(nn_walk(a, st));
        NnUnits un{};
        un.urow = g->d_urow + g->h_ubase[b];
        un.ubeg = g->d_ubeg + g->h_ubase[b];
        un.ufirst = g->d_ufirst + (size_t)b * (n + 1);
        un.nunits = g->h_nunits[b];
        un.multi = g->d_multi + g->h_mbase[b];
        un.nmulti = g->h_mbase[b + 1] - g->h_mbase[b];
        CK(nn_gather(n, g->d_csr_off + (size_t)b * (n + 1), g->d_perm + a.seg_lo, slot, val, un, part, L27, b == 0, st));
        g->launches += 3;
    }
    CK(cudaStreamSynchronize(st));
    return RT_OK;
}

int build_nn(rt_grid *g)
{
    if (g->nn_ok) return RT_OK;
    RCK(nn_lstar_into(g, g->d_chi, nullptr, g->d_L27, g->st));
    CK(nn_diag(g->nvox, g->d_L27, g->d_L, g->st));
    g->launches++;
    RCK(sync(g));
    g->nn_ok = true;
    g->lstar_prec = RT_FP64;
    return RT_OK;
}

// x = (I - (1-eps) L*_NN)^-1 y: BiCGSTAB on the Jacobi-preconditioned system
// (unless RT_TUNE_NN_KRYLOV is 0), then Jacobi sweeps until one changes x by
// <= jtol max |x| (jtol <= 0: the grid's nn_jtol), in one cooperative launch;
// returns the result's buffer in *x_out.
constexpr double kCorrOsJtol = 1e-8;  // OS-step bound inside the FP32 correction sweeps of rt_solve

int nn_solve(rt_grid *g, const double *y, double **x_out, double jtol = 0.0)
{
    NnOs o{};
    o.nvox = g->nvox;
    o.sph = g->coord == RT_SPHERICAL;
    o.n1 = g->n1;
    o.n2 = g->n2;
    o.n3 = g->n3;
    o.L27 = g->d_L27;
    o.eps = g->d_eps;
    o.y = y;
    o.work = g->d_nnx;
    o.jtol = jtol > 0.0 ? jtol : g->nn_jtol;
    o.jmax = g->nn_jmax;
    o.krylov = g->nn_krylov;
    o.kmax = 1000;
    o.stall = g->nn_stall;
    g->nn_stall = 0;
    int its = 0, sweeps = 0, status = 0;
    const int t = tstart(g, 2);
    CK(nn_os_solve(o, g->st, x_out, &its, &sweeps, &status));
    tstop(g, t, 2, 0);
    g->launches += 1;
    g->nn_sweeps = sweeps;
    g->nn_krylov_its = its;
    g->os_solves += 1;
    g->os_its += its;
    g->os_sweeps += sweeps;
    if (status == 3) return fail(RT_ETIMEOUT, "NN Lambda* OS step: a grid-barrier wait gave up; S not updated by this step");
    if (status == 2) return fail(RT_EDEVICE, "NN Lambda* OS step diverged");
    if (status == 1) return fail(RT_ENOTCONVERGED, "NN Lambda* OS step: no convergence in %d sweeps", sweeps);
    return RT_OK;
}

int ali_step_impl(rt_grid *g, int prec, double *rel_out)
{
    if (g->use_lstar == RT_LSTAR_NN) {
        RCK(build_nn(g));
        RCK(run_fs_J(g, prec, 0, g->d_S, g->d_J));
        CK(nn_rhs(g->nvox, g->d_S, g->d_J, g->d_eps, g->d_B, g->d_nny, g->st));
        double *x = nullptr;
        RCK(nn_solve(g, g->d_nny, &x));
        CK(cudaMemsetAsync(g->d_maxrel, 0, sizeof(unsigned long long), g->st));
        double *slot = g->ng ? ng_append_slot(g) : nullptr;
        CK(nn_apply(g->nvox, g->d_S, x, nullptr, slot, g->d_maxrel, g->st));
        g->launches += 2;
        double rel = 0.0;
        RCK(read_maxrel(g, &rel));
        *rel_out = rel;
        g->history.push_back(rel);
        return RT_OK;
    }
    RCK(fs_iteration(g, prec, g->d_S, g->d_J));
    CK(cudaMemsetAsync(g->d_maxrel, 0, sizeof(unsigned long long), g->st));
    double *slot = g->ng ? ng_append_slot(g) : nullptr;
    CK(ali_update(g->nvox, g->d_S, g->d_J, g->d_L, g->d_eps, g->d_B, g->use_lstar, slot, g->d_maxrel, g->st));
    g->launches++;
    double rel = 0.0;
    RCK(read_maxrel(g, &rel));
    *rel_out = rel;
    g->history.push_back(rel);
    return RT_OK;
}

int copy_out(rt_grid *g, const double *src, double *out, size_t n, int where)
{
    if (!out) return fail(RT_EINVAL, "output pointer is NULL");
    if (where != RT_HOST && where != RT_DEVICE) return fail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    CK(cudaMemcpyAsync(out, src, sizeof(double) * n, where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       g->st));
    if (where == RT_HOST) RCK(sync(g));
    return RT_OK;
}

int check_lost(rt_grid *g)
{
    if (g->lost) return fail(RT_EDEVICE, "%d characteristics could not be tracked", g->lost);
    return RT_OK;
}

}  // namespace

int rt_grid_nn_lstar(rt_grid *g, const double *chi, const uint32_t *pbits, double *L27, cudaStream_t st)
{
    if (g->nphi < 3) return fail(RT_EINVAL, "the nearest-neighbour Lambda* needs n_phi >= 3");
    if (!pbits) return fail(RT_EINVAL, "parabola choices of chi required");
    return nn_lstar_into(g, chi, pbits, L27, st);
}

int rt_grid_member_fs(rt_grid *g, const float2 *cs, const float *B32, const uint32_t *pbits, double *J, double *L,
                      double *Fc, cudaStream_t st)
{
    const int n = g->nvox;
    for (int b = 0; b < g->nblk; ++b) {
        int w0 = g->blk_w0[b], nw = g->blk_nw[b];
        int64_t r_lo = g->h_ang_ray_off[w0], r_hi = g->h_ang_ray_off[w0 + nw];
        int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
        const int32_t *off = g->d_csr_off + (size_t)b * (n + 1);
        float2 *buf = (float2 *)g->d_segbuf;
        CK(march_block_bits(g->d_vox, g->d_len32, g->d_ray_off, r_lo, r_hi, lo, ns, cs, B32, (float)g->I_outer, buf,
                            g->march_chunk, pbits, st));
        CK(gather_block<float2>(n, off, g->d_perm + lo, buf, g->d_ang_seg_off, w0, nw, lo, g->d_invL, g->d_wL32,
                                g->d_wt, g->d_dirs, g->d_urow + g->h_ubase[b], g->d_ubeg + g->h_ubase[b],
                                g->d_ufirst + (size_t)b * (n + 1), g->h_nunits[b], g->d_multi + g->h_mbase[b],
                                (int)(g->h_mbase[b + 1] - g->h_mbase[b]), g->d_order + g->h_ubase[b],
                                g->d_ulen + g->h_ubase[b], g->d_gbase + g->h_goff[b], g->d_sell + g->h_soff[b],
                                g->d_part, J, L, Fc, b == 0, st));
    }
    return RT_OK;
}

int rt_grid_build_nn(rt_grid *g) { return build_nn(g); }

int rt_grid_member_fs64J(rt_grid *g, const double2 *cs64, const double *B64, const uint32_t *pbits, double *J,
                         cudaStream_t st)
{
    const int n = g->nvox;
    for (int b = 0; b < g->nblk; ++b) {
        int w0 = g->blk_w0[b], nw = g->blk_nw[b];
        int64_t r_lo = g->h_ang_ray_off[w0], r_hi = g->h_ang_ray_off[w0 + nw];
        int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
        const int32_t *off = g->d_csr_off + (size_t)b * (n + 1);
        double *buf = (double *)g->d_segbuf;
        CK(march_block_bits64J(g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, lo, ns, cs64, B64, g->I_outer, 0, buf,
                               g->march_chunk, pbits, st));
        CK(gather_J<double>(n, off, g->jt[b], g->d_perm + lo, buf, g->d_ang_seg_off, w0, nw, lo, g->d_wL32,
                            g->d_invL, g->d_wt, g->d_partJ, J, b == 0, st));
    }
    return RT_OK;
}

extern "C" {

const char *rt_last_error(void) { return g_err.c_str(); }

int rt_grid_create(rt_grid **out, const rt_grid_desc *d)
{
    if (!out) return fail(RT_EINVAL, "out is NULL");
    RCK(check_desc(d));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(RT_ECUDA, "no CUDA device available");
    }
    if (d->device < 0 || d->device >= ndev) return fail(RT_EINVAL, "device %d out of range", d->device);
    CK(cudaSetDevice(d->device));
    rt_grid *g = new rt_grid();
    g->device = d->device;
    g->st = (cudaStream_t)d->stream;
    g->coord = d->coord;
    g->n1 = d->n[0];
    g->n2 = d->n[1];
    g->n3 = d->n[2];
    g->nvox = g->n1 * g->n2 * g->n3;
    g->n_ang = d->n_angles;
    g->nphi = (d->coord == RT_SPHERICAL) ? g->n3 : g->n2;
    g->inner_bc = d->inner_bc;
    g->interp = d->interp;
    g->precision = d->precision;
    g->use_lstar = d->use_lstar;
    g->ng = d->ng ? 1 : 0;
    g->refine_every = d->refine_every > 0 ? d->refine_every : 32;
    g->I_outer = d->I_outer;
    g->ablk = d->angle_block;
    for (int a = 0; a < 3; ++a) g->h_e[a].assign(d->edges[a], d->edges[a] + d->n[a] + 1);
    g->h_dirs.assign(d->dirs, d->dirs + 3 * (size_t)d->n_angles);
    g->h_wt.assign(d->weights, d->weights + d->n_angles);
    int rc = noalloc_prepare(g->device);
    if (rc == RT_OK) rc = upload_tables(g);
    if (rc == RT_OK) rc = build_geometry(g);
    if (rc == RT_OK) rc = alloc_fields(g);
    if (rc == RT_OK) rc = sync(g);
    if (rc != RT_OK) {
        std::string keep = g_err;
        cudaStreamSynchronize(g->st);
        release(g);
        delete g;
        g_err = keep;
        return rc;
    }
    *out = g;
    return RT_OK;
}

int rt_grid_destroy(rt_grid *g)
{
    if (!g) return RT_OK;
    cudaSetDevice(g->device);
    cudaStreamSynchronize(g->st);
    release(g);
    delete g;
    return RT_OK;
}

int rt_get_info(const rt_grid *g, rt_info *info)
{
    if (!g || !info) return fail(RT_EINVAL, "NULL argument");
    info->n_vox = g->nvox;
    info->n_angles = g->n_ang;
    info->n_rays = g->n_rays;
    info->n_segments = g->n_seg;
    info->device_bytes = g->bytes;
    info->n_blocks = g->nblk;
    info->angle_block = g->ablk;
    info->lost_rays = g->lost;
    info->precision = g->precision;
    info->geometry_ms = g->geom_ms;
    info->geometry_trace_ms = g->geom_trace_ms;
    info->geometry_lists_ms = g->geom_lists_ms;
    return RT_OK;
}

int rt_set_opacity(rt_grid *g, const double *chi, const double *eps, const double *B, int where)
{
    if (!g || !chi || !eps || !B) return fail(RT_EINVAL, "NULL argument");
    if (where != RT_HOST && where != RT_DEVICE) return fail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    CK(cudaSetDevice(g->device));
    const size_t n = g->nvox;
    if (where == RT_HOST) {
        for (size_t v = 0; v < n; ++v) {
            if (!(chi[v] > 0.0) || !std::isfinite(chi[v])) return fail(RT_EINVAL, "chi[%zu] must be > 0 and finite", v);
            if (!(eps[v] > 0.0 && eps[v] <= 1.0)) return fail(RT_EINVAL, "eps[%zu] must be in (0, 1]", v);
            if (!(B[v] >= 0.0) || !std::isfinite(B[v])) return fail(RT_EINVAL, "B[%zu] must be >= 0 and finite", v);
        }
    } else {  // device input: checked on the device before anything is copied (one wait)
        CK(check_opacity(g->nvox, chi, eps, B, g->d_maxrel, g->st));
        g->launches++;
        CK(cudaMemcpyAsync(g->h_pin, g->d_maxrel, sizeof(unsigned long long), cudaMemcpyDeviceToHost, g->st));
        RCK(sync(g));
        unsigned long long bad = 0;
        std::memcpy(&bad, g->h_pin, sizeof(bad));
        if (bad != ~0ull) {
            const unsigned long long v = bad >> 2;
            const int c = (int)(bad & 3ull);
            if (c == 0) return fail(RT_EINVAL, "chi[%llu] must be > 0 and finite", v);
            if (c == 1) return fail(RT_EINVAL, "eps[%llu] must be in (0, 1]", v);
            return fail(RT_EINVAL, "B[%llu] must be >= 0 and finite", v);
        }
    }
    drop_graph(g);
    cudaMemcpyKind kind = where == RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(g->d_chi, chi, sizeof(double) * n, kind, g->st));
    CK(cudaMemcpyAsync(g->d_eps, eps, sizeof(double) * n, kind, g->st));
    CK(cudaMemcpyAsync(g->d_B, B, sizeof(double) * n, kind, g->st));
    CK(cudaMemcpyAsync(g->d_S, g->d_B, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->st));
    CK(mark_parabola(g->d_vox, g->d_len64, g->d_chi, g->n_seg, g->interp == RT_PARABOLIC, g->st));
    g->launches++;
    g->lstar_prec = -1;
    g->cw_ok = false;
    g->cw64_ok = false;
    g->nn_ok = false;
    if (where == RT_HOST) RCK(sync(g));
    reset_ng(g);
    g->history.clear();
    return RT_OK;
}

int rt_set_S(rt_grid *g, const double *S, int where)
{
    if (!g || !S) return fail(RT_EINVAL, "NULL argument");
    if (where != RT_HOST && where != RT_DEVICE) return fail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    CK(cudaSetDevice(g->device));
    CK(cudaMemcpyAsync(g->d_S, S, sizeof(double) * g->nvox,
                       where == RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->st));
    if (where == RT_HOST) RCK(sync(g));
    reset_ng(g);
    g->history.clear();
    return RT_OK;
}

int rt_tune(rt_grid *g, int knob, int value)
{
    if (!g && knob == RT_TUNE_GEOM_PREDICT) {  // library-wide, for grids created afterwards
        if (value != 0 && value != 1) return fail(RT_EINVAL, "guided completion: 0 or 1");
        g_geom_predict = value;
        return RT_OK;
    }
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    if (knob == RT_TUNE_GEOM_PREDICT) return fail(RT_EINVAL, "RT_TUNE_GEOM_PREDICT is set on the library (grid NULL)");
    drop_graph(g);  // a captured formal solution holds the old settings
    if (knob == RT_TUNE_GRAPH) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "graph: 0 or 1");
        g->sw_graph = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_MARCH_CHUNK) {
        if (value < 64 || value > 16384) return fail(RT_EINVAL, "march chunk must be in [64, 16384]");
        g->march_chunk = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_STREAMED_WEIGHTS) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "streamed weights: 0 or 1");
        g->sw_enabled = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_MARCH64_COARSEN) {
        if (value != 1 && value != 2) return fail(RT_EINVAL, "FP64 march coarsening must be 1 or 2");
        g->sw64_coarsen = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_MARCH_STAGES) {
        if (value != 0 && (value < 2 || value > 4)) return fail(RT_EINVAL, "march stages: 0 or 2..4");
        g->sw_stages = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_MARCH_BULK) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "march bulk copies: 0 or 1");
        g->sw_bulk = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_NN_JTOL) {
        if (value < 1 || value > 15) return fail(RT_EINVAL, "NN Jacobi tolerance exponent must be in [1, 15]");
        g->nn_jtol = std::pow(10.0, -value);
        return RT_OK;
    }
    if (knob == RT_TUNE_SCATTER) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "scatter: 0 or 1");
        g->sw_scatter = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_OVERLAP) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "overlap: 0 or 1");
        g->sw_overlap = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_MARCH_COARSEN) {
        if (value != 1 && value != 2 && value != 4) return fail(RT_EINVAL, "march coarsening must be 1, 2 or 4");
        g->sw_coarsen = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_NN_KRYLOV) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "NN Krylov OS solve: 0 or 1");
        g->nn_krylov = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_S_BLOCKED) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "blocked S order: 0 or 1");
        g->sblk = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_MARCH_STREAMS) {
        if (value < 1 || value > 3) return fail(RT_EINVAL, "march streams: 1, 2 or 3");
        g->sw_mstreams = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_FOLD_WEIGHT) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "fold weight: 0 or 1");
        g->sw_fold = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_MARCH_LOOKAHEAD) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "march lookahead: 0 or 1");
        g->sw_lookahead = value;
        return RT_OK;
    }
    if (knob == RT_TUNE_NN_TEST_STALL) {
        if (value != 0 && value != 1) return fail(RT_EINVAL, "NN OS-step stall test: 0 or 1");
        g->nn_stall = value;
        return RT_OK;
    }
    return fail(RT_EINVAL, "unknown tuning knob %d", knob);
}

int rt_set_precision(rt_grid *g, int precision)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    if (precision != RT_FP64 && precision != RT_MIXED) return fail(RT_EINVAL, "bad precision");
    g->precision = precision;
    reset_ng(g);
    return RT_OK;
}

int rt_formal_solution_ex(rt_grid *g, int precision, int homog)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    if (precision != RT_FP64 && precision != RT_MIXED) return fail(RT_EINVAL, "bad precision");
    RCK(check_lost(g));
    CK(cudaSetDevice(g->device));
    RCK(run_fs(g, precision, homog ? 1 : 0, g->d_S, g->d_J, g->d_L, g->d_Fc, g->d_F));
    CK(cudaGetLastError());
    g->lstar_prec = precision;
    return RT_OK;
}

int rt_formal_solution(rt_grid *g)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    return rt_formal_solution_ex(g, g->precision, 0);
}

int rt_ali_step(rt_grid *g, double *max_rel_dS)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    RCK(check_lost(g));
    CK(cudaSetDevice(g->device));
    double rel = 0.0;
    RCK(ali_step_impl(g, g->precision, &rel));
    if (g->ng) RCK(ng_maybe(g, g->d_S, nullptr));
    if (max_rel_dS) *max_rel_dS = rel;
    return RT_OK;
}

int rt_solve(rt_grid *g, double tol, int max_iter, int *iters)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    if (!(tol > 0.0) || max_iter < 1) return fail(RT_EINVAL, "need tol > 0 and max_iter >= 1");
    RCK(check_lost(g));
    CK(cudaSetDevice(g->device));
    reset_ng(g);
    g->history.clear();
    if (iters) *iters = 0;
    if (g->precision == RT_FP64) {
        for (int it = 1; it <= max_iter; ++it) {
            double rel = 0.0;
            RCK(ali_step_impl(g, RT_FP64, &rel));
            if (iters) *iters = it;
            if (rel < tol) return RT_OK;
            if (g->ng) RCK(ng_maybe(g, g->d_S, nullptr));
        }
        return fail(RT_ENOTCONVERGED, "no convergence to %g in %d iterations", tol, max_iter);
    }
    // mixed precision: FP64 residual, FP32 correction sweeps, FP64 update
    const int n = g->nvox;
    if (g->use_lstar == RT_LSTAR_NN) RCK(build_nn(g));
    int total = 0;
    while (total < max_iter) {
        RCK(fs_iteration(g, RT_FP64, g->d_S, g->d_J));
        total++;
        CK(cudaMemsetAsync(g->d_maxrel, 0, sizeof(unsigned long long), g->st));
        if (g->use_lstar == RT_LSTAR_NN) {  // residual and its NN-preconditioned step
            CK(nn_rhs(n, g->d_S, g->d_J, g->d_eps, g->d_B, g->d_r, g->st));
            double *x = nullptr;
            RCK(nn_solve(g, g->d_r, &x));
            CK(cudaMemsetAsync(g->d_maxrel, 0, sizeof(unsigned long long), g->st));
            CK(nn_apply(n, nullptr, x, g->d_S, nullptr, g->d_maxrel, g->st));
        } else {
            CK(residual(n, g->d_S, g->d_J, g->d_L, g->d_eps, g->d_B, g->use_lstar, g->d_r, g->d_maxrel, g->st));
        }
        g->launches++;
        double rel = 0.0;
        RCK(read_maxrel(g, &rel));
        g->history.push_back(rel);
        if (iters) *iters = total;
        if (rel < tol) return RT_OK;
        CK(cudaMemcpyAsync(g->d_Lkeep, g->d_L, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->st));
        CK(cudaMemsetAsync(g->d_delta, 0, sizeof(double) * n, g->st));
        reset_ng(g);
        // the correction sweeps stop early only when the update is far below the
        // outer tolerance; a small per-sweep change alone says little when ALI
        // converges slowly (thick media, small eps)
        const double inner_tol = 0.01 * tol;
        for (int k = 0; k < g->refine_every && total < max_iter; ++k) {
            RCK(run_fs_J(g, RT_MIXED, 1, g->d_delta, g->d_Jd));
            total++;
            CK(cudaMemsetAsync(g->d_maxrel, 0, sizeof(unsigned long long), g->st));
            double *slot = g->ng ? ng_append_slot(g) : nullptr;
            if (g->use_lstar == RT_LSTAR_NN) {
                CK(nn_rhs_corr(n, g->d_delta, g->d_Jd, g->d_r, g->d_eps, g->d_nny, g->st));
                // the right-hand side carries the FP32 rounding of the correction's
                // formal solution (~1e-7 of it): its OS step needs no more than 1e-8
                double *x = nullptr;
                RCK(nn_solve(g, g->d_nny, &x, std::max(g->nn_jtol, kCorrOsJtol)));
                CK(cudaMemsetAsync(g->d_maxrel, 0, sizeof(unsigned long long), g->st));
                CK(nn_apply(n, g->d_delta, x, g->d_S, slot, g->d_maxrel, g->st));
            } else {
                CK(ali_correction(n, g->d_delta, g->d_Jd, g->d_r, g->d_Lkeep, g->d_eps, g->d_S, g->use_lstar, slot,
                                  g->d_maxrel, g->st));
            }
            g->launches++;
            double rd = 0.0;
            RCK(read_maxrel(g, &rd));
            if (rd < inner_tol) break;
            if (g->ng) RCK(ng_maybe(g, g->d_delta, g->d_S));
        }
        CK(add_inplace(n, g->d_S, g->d_delta, g->st));
        g->launches++;
    }
    if (iters) *iters = total;
    return fail(RT_ENOTCONVERGED, "no convergence to %g in %d formal solutions", tol, max_iter);
}

int rt_get_J(const rt_grid *g, double *out, int where)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    return copy_out((rt_grid *)g, g->d_J, out, g->nvox, where);
}

int rt_get_S(const rt_grid *g, double *out, int where)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    return copy_out((rt_grid *)g, g->d_S, out, g->nvox, where);
}

int rt_get_Lstar(const rt_grid *g, double *out, int where)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    return copy_out((rt_grid *)g, g->d_L, out, g->nvox, where);
}

int rt_get_Lstar_nn(rt_grid *g, double *out27, int where)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    if (g->use_lstar != RT_LSTAR_NN) return fail(RT_EINVAL, "the grid was not created with use_lstar = RT_LSTAR_NN");
    RCK(check_lost(g));
    CK(cudaSetDevice(g->device));
    RCK(build_nn(g));
    if (!out27) return fail(RT_EINVAL, "out is NULL");
    if (where == RT_DEVICE) {  // slot planes to rows of 27
        CK(nn_rows(g->nvox, g->d_L27, out27, g->st));
        RCK(sync(g));
        return RT_OK;
    }
    if (where != RT_HOST) return fail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    double *tmp = nullptr;
    if (cudaMalloc(&tmp, sizeof(double) * 27 * (size_t)g->nvox) != cudaSuccess) {
        cudaGetLastError();
        return fail(RT_ENOMEM, "no device memory for the row layout of the NN Lambda*");
    }
    cudaError_t e = nn_rows(g->nvox, g->d_L27, tmp, g->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out27, tmp, sizeof(double) * 27 * (size_t)g->nvox, cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    cudaFree(tmp);
    CK(e);
    return RT_OK;
}

int rt_get_flux(const rt_grid *g, double *out3, int where)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    return copy_out((rt_grid *)g, g->d_F, out3, 3 * (size_t)g->nvox, where);
}

int rt_get_history(const rt_grid *g, double *hist, int max, int *n)
{
    if (!g || !n) return fail(RT_EINVAL, "NULL argument");
    int c = (int)std::min<size_t>(g->history.size(), max > 0 ? (size_t)max : 0);
    if (hist)
        for (int q = 0; q < c; ++q) hist[q] = g->history[q];
    *n = hist ? c : (int)g->history.size();
    return RT_OK;
}

int rt_get_crossings(const rt_grid *g, int omega, int64_t *n_rays, int64_t *n_seg, int32_t *ray_off,
                     int32_t *ray_origin, int32_t *ray_core, int32_t *vox, double *len, uint8_t *restart)
{
    if (!g || !n_rays || !n_seg) return fail(RT_EINVAL, "NULL argument");
    if (omega < 0 || omega >= g->n_ang) return fail(RT_EINVAL, "omega %d out of range", omega);
    rt_grid *gg = (rt_grid *)g;
    CK(cudaSetDevice(g->device));
    int64_t r0 = g->h_ang_ray_off[omega], r1 = g->h_ang_ray_off[omega + 1];
    int64_t s0 = g->h_ang_seg_off[omega], s1 = g->h_ang_seg_off[omega + 1];
    *n_rays = r1 - r0;
    *n_seg = s1 - s0;
    if (!ray_off && !ray_origin && !ray_core && !vox && !len && !restart) return RT_OK;
    if (!ray_off || !ray_origin || !ray_core || !vox || !len || !restart) return fail(RT_EINVAL, "all buffers are needed");
    std::vector<int64_t> ro(r1 - r0 + 1);
    std::vector<uint32_t> vw(s1 - s0);
    CK(cudaMemcpyAsync(ro.data(), g->d_ray_off + r0, sizeof(int64_t) * ro.size(), cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(ray_origin, g->d_ray_origin + r0, sizeof(int32_t) * (r1 - r0), cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(vw.data(), g->d_vox + s0, sizeof(uint32_t) * vw.size(), cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(len, g->d_len64 + s0, sizeof(double) * vw.size(), cudaMemcpyDeviceToHost, g->st));
    RCK(sync(gg));
    for (size_t r = 0; r < ro.size(); ++r) ray_off[r] = (int32_t)(ro[r] - s0);
    for (size_t s = 0; s < vw.size(); ++s) {
        vox[s] = (int32_t)(vw[s] & RTK_VOXMASK);
        restart[s] = (vw[s] & RTK_RESTART) ? 1 : 0;
    }
    for (int64_t r = 0; r < r1 - r0; ++r) ray_core[r] = (vw[ro[r] - s0] & RTK_CORE) ? 1 : 0;
    return RT_OK;
}

int rt_fs_angles(rt_grid *g, const int32_t *omegas, int n, int precision, double *Ibar, double *Lbar, int where)
{
    if (!g || (!omegas && n > 0) || !Ibar || !Lbar) return fail(RT_EINVAL, "NULL argument");
    if (precision != RT_FP64 && precision != RT_MIXED) return fail(RT_EINVAL, "bad precision");
    if (where != RT_HOST && where != RT_DEVICE) return fail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    for (int q = 0; q < n; ++q)
        if (omegas[q] < 0 || omegas[q] >= g->n_ang) return fail(RT_EINVAL, "omega %d out of range", omegas[q]);
    RCK(check_lost(g));
    CK(cudaSetDevice(g->device));
    const int nv = g->nvox;
    const int para = g->interp == RT_PARABOLIC;
    if (precision == RT_FP64) CK(pack_chiS64(nv, g->d_chi, g->d_S, g->d_cs64, g->st));
    else CK(pack_chiS32(nv, g->d_chi, g->d_S, g->d_B, g->d_cs32, g->d_B32, nullptr, g->st));
    double *tI = g->d_Jd, *tL = g->d_Ld;  // scratch vectors of the correction sweep
    int marched = -1;  // block whose per-segment results are in the buffer
    for (int q = 0; q < n; ++q) {
        int w = omegas[q];
        int b = w / g->ablk;
        int w0 = g->blk_w0[b], nw = g->blk_nw[b];
        int64_t r_lo = g->h_ang_ray_off[w0], r_hi = g->h_ang_ray_off[w0 + nw];
        int64_t lo = g->h_ang_seg_off[w0], ns = g->h_ang_seg_off[w0 + nw] - lo;
        const int32_t *off = g->d_csr_off + (size_t)b * (nv + 1);
        if (b == marched) {
            // results of this block are still in the buffer
        } else if (precision == RT_FP64)
            CK(march_block<double, double2>(g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs64, g->d_B,
                                            g->I_outer, 0, para, (double2 *)g->d_segbuf, g->march_chunk, g->st));
        else
            CK(march_block<float, float2>(g->d_vox, g->d_len32, g->d_ray_off, r_lo, r_hi, lo, ns, g->d_cs32, g->d_B32,
                                          (float)g->I_outer, 0, para, (float2 *)g->d_segbuf, g->march_chunk, g->st));
        marched = b;
        CK(gather_angle_range(nv, off, g->d_perm + lo, g->d_segbuf, 0, precision == RT_MIXED,
                              g->h_ang_seg_off[w] - lo, g->h_ang_seg_off[w + 1] - lo, g->d_invL + (size_t)w * nv, tI,
                              tL, g->st));
        cudaMemcpyKind kind = where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(Ibar + (size_t)q * nv, tI, sizeof(double) * nv, kind, g->st));
        CK(cudaMemcpyAsync(Lbar + (size_t)q * nv, tL, sizeof(double) * nv, kind, g->st));
    }
    RCK(sync(g));
    return RT_OK;
}

int rt_set_timing(rt_grid *g, int enable)
{
    if (!g) return fail(RT_EINVAL, "grid is NULL");
    if (enable < 0) return fail(RT_EINVAL, "timing: 0 (off), 1 (every launch) or N > 1 (every N-th march launch)");
    CK(cudaSetDevice(g->device));
    if (enable) {
        RCK(sync(g));
        g->ev_used = 0;
        g->ev_kind.clear();
        g->ev_segs.clear();
        g->ev_bytes.clear();
        g->launches = 0;
        g->os_solves = g->os_its = g->os_sweeps = 0;
        g->timing_count = 0;
        g->timing_every = enable;
    }
    g->timing = enable != 0;
    return RT_OK;
}

int rt_get_timing(rt_grid *g, rt_timing *t)
{
    if (!g || !t) return fail(RT_EINVAL, "NULL argument");
    CK(cudaSetDevice(g->device));
    RCK(sync(g));
    std::memset(t, 0, sizeof(*t));
    for (size_t q = 0; q < g->ev_kind.size(); ++q) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, g->ev[2 * q], g->ev[2 * q + 1]));
        if (g->ev_kind[q] == 0) {
            t->march_ms += ms;
            t->march_launches++;
            t->march_segments += g->ev_segs[q];
            t->march_bytes += g->ev_bytes[q];
        } else if (g->ev_kind[q] == 1) {
            t->gather_ms += ms;
            t->gather_launches++;
        } else {
            t->os_ms += ms;
        }
    }
    t->kernel_launches = g->launches;
    t->os_solves = g->os_solves;
    t->os_krylov_its = g->os_its;
    t->os_sweeps = g->os_sweeps;
    return RT_OK;
}

}  // extern "C"
