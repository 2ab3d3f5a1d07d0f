// sweep.cu -- formal solution over a solid-angle set too large to hold its
// crossing lists at once (the angle-resolution study of Sect. 3.1-3.2: flux
// vectors of the outermost voxels with up to 512^2 solid angles).  The angles
// are processed in chunks: each chunk is a grid of its own (geometry,
// parabola choices, formal solution), whose J and flux, taken with the chunk's
// weights renormalised to 1, enter the sums with the chunk's share of the
// total weight; the chunk's memory is released before the next one.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "grid.h"
#include "rt_internal.h"

using namespace rtk;

namespace {

int sfail(int code, const std::string &m)
{
    set_last_error(m.c_str());
    return code;
}

#define SCK(...)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (__VA_ARGS__);                                                                  \
        if (e_ != cudaSuccess) return sfail(RT_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// acc (+)= a x
__global__ void k_sweep_axpy(int64_t n, double a, const double *x, double *acc, int first)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[i] = first ? a * x[i] : acc[i] + a * x[i];
}

struct DevBuf {
    double *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

struct GridGuard {
    rt_grid *g = nullptr;
    ~GridGuard() { rt_grid_destroy(g); }
};

}  // namespace

extern "C" {

int rt_fs_sweep(const rt_grid_desc *d, int angles_per_chunk, const double *chi, const double *S, const double *B,
                int precision, double *J, double *F, int where)
{
    if (!d || !chi || !S || !B || !J || !F) return sfail(RT_EINVAL, "NULL argument");
    if (angles_per_chunk < 1) return sfail(RT_EINVAL, "angles_per_chunk must be >= 1");
    if (precision != RT_FP64 && precision != RT_MIXED) return sfail(RT_EINVAL, "precision must be RT_FP64 or RT_MIXED");
    if (where != RT_HOST && where != RT_DEVICE) return sfail(RT_EINVAL, "where must be RT_HOST or RT_DEVICE");
    if (d->n_angles < 1 || !d->dirs || !d->weights) return sfail(RT_EINVAL, "need n_angles >= 1, dirs and weights");
    double wsum = 0.0;
    for (int w = 0; w < d->n_angles; ++w) {
        if (!(d->weights[w] > 0.0) || !std::isfinite(d->weights[w])) return sfail(RT_EINVAL, "weights must be > 0");
        wsum += d->weights[w];
    }
    if (!(std::fabs(wsum - 1.0) < 1e-10)) return sfail(RT_EINVAL, "weights must sum to 1");
    if (d->n[0] < 1 || d->n[1] < 1 || d->n[2] < 1) return sfail(RT_EINVAL, "need n[a] >= 1");
    const int64_t nvox = (int64_t)d->n[0] * d->n[1] * d->n[2];
    SCK(cudaSetDevice(d->device));
    cudaStream_t st = (cudaStream_t)d->stream;
    DevBuf accJ, accF, tmp, ones;
    SCK(cudaMalloc(&accJ.p, sizeof(double) * nvox));
    SCK(cudaMalloc(&accF.p, sizeof(double) * 3 * nvox));
    SCK(cudaMalloc(&tmp.p, sizeof(double) * 3 * nvox));
    SCK(cudaMalloc(&ones.p, sizeof(double) * nvox));
    SCK(fill_const((int)nvox, ones.p, 1.0, st));
    std::vector<double> h_ones(where == RT_HOST ? nvox : 0, 1.0);  // eps = 1: only the formal solution is used
    int first = 1;
    for (int w0 = 0; w0 < d->n_angles; w0 += angles_per_chunk) {
        const int nw = std::min(angles_per_chunk, d->n_angles - w0);
        double wc = 0.0;
        for (int w = w0; w < w0 + nw; ++w) wc += d->weights[w];
        std::vector<double> wn(nw);
        for (int w = 0; w < nw; ++w) wn[w] = d->weights[w0 + w] / wc;
        double wn_sum = 0.0;  // renormalised to 1 within the grid's check
        for (double x : wn) wn_sum += x;
        if (!(std::fabs(wn_sum - 1.0) < 1e-10)) return sfail(RT_EINVAL, "chunk weights cannot be renormalised");
        rt_grid_desc c = *d;
        c.n_angles = nw;
        c.dirs = d->dirs + 3 * (size_t)w0;
        c.weights = wn.data();
        c.precision = precision;
        c.use_lstar = RT_LSTAR_DIAG;
        c.ng = 0;
        GridGuard gg;
        int rc = rt_grid_create(&gg.g, &c);
        if (rc != RT_OK) return rc;
        if ((rc = rt_set_opacity(gg.g, chi, where == RT_HOST ? h_ones.data() : ones.p, B, where)) != RT_OK) return rc;
        if ((rc = rt_set_S(gg.g, S, where)) != RT_OK) return rc;
        if ((rc = rt_formal_solution_ex(gg.g, precision, 0)) != RT_OK) return rc;
        if ((rc = rt_get_J(gg.g, tmp.p, RT_DEVICE)) != RT_OK) return rc;
        k_sweep_axpy<<<152 * 4, 256, 0, st>>>(nvox, wc, tmp.p, accJ.p, first);
        SCK(cudaGetLastError());
        if ((rc = rt_get_flux(gg.g, tmp.p, RT_DEVICE)) != RT_OK) return rc;
        k_sweep_axpy<<<152 * 4, 256, 0, st>>>(3 * nvox, wc, tmp.p, accF.p, first);
        SCK(cudaGetLastError());
        SCK(cudaStreamSynchronize(st));
        first = 0;
    }
    const cudaMemcpyKind kind = where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    SCK(cudaMemcpyAsync(J, accJ.p, sizeof(double) * nvox, kind, st));
    SCK(cudaMemcpyAsync(F, accF.p, sizeof(double) * 3 * nvox, kind, st));
    SCK(cudaStreamSynchronize(st));
    return RT_OK;
}

}  // extern "C"
