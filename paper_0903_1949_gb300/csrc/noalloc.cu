// noalloc.cu -- formal solution of one solid angle without any allocation.
//
// Some callers cannot call cudaMalloc at the moment they need a result: code
// that runs inside another framework's stream-ordered memory pool or under a
// hard device-memory budget that was fully handed out up front, or host code
// that must not take the allocator's global locks (a real-time or signal
// context).  rt_fs_angle_noalloc serves them: it reuses the grid built
// earlier by rt_grid_create and keeps its per-segment scratch in the
// file-scope device array below instead of any allocated buffer.  The caller
// passes the output buffers.
#include <cuda_runtime.h>

#include <mutex>

#include "grid.h"
#include "rt_internal.h"

namespace {

// Per-segment scratch (l I, l lambda) of one solid angle: 16 MiB, i.e. up to
// 1 Mi segments in FP64 or 2 Mi in FP32.  Every GPU that loads the library
// holds this array until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side shadow, not device memory:
// the device address is looked up once per device and cached here.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_scratch_addr[MAX_DEVICES] = {};

int scratch_for(int dev, void **out, char *msg, size_t msglen)
{
    if (dev < 0 || dev >= MAX_DEVICES) {
        snprintf(msg, msglen, "device %d outside the supported range", dev);
        return RT_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // the device current is `dev`
        if (e != cudaSuccess || !p) {
            snprintf(msg, msglen, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return RT_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RT_OK;
}

// Ibar / Lbar of one solid angle: the angle's segments occupy entries
// [a0, a1) of its block's ownership lists and [0, a1 - a0) of the scratch.
template <typename P>
__global__ void k_noalloc_gather(int nvox, const int32_t *off, const int32_t *perm, const P *buf, int32_t a0, int32_t a1,
                                 const double *invL_w, double *Ibar, double *Lbar)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    double aI = 0.0, aL = 0.0;
    for (int e = off[v]; e < off[v + 1]; ++e) {
        int s = perm[e];
        if (s < a0 || s >= a1) continue;
        P val = buf[s - a0];
        aI += (double)val.x;
        aL += (double)val.y;
    }
    Ibar[v] = aI * invL_w[v];
    Lbar[v] = aL * invL_w[v];
}

int nofail(int code, const char *m)
{
    rtk::set_last_error(m);
    return code;
}

}  // namespace

extern "C" {

int rt_fs_angle_noalloc(rt_grid *g, int omega, int precision, double *Ibar, double *Lbar)
{
    if (!g || !Ibar || !Lbar) return nofail(RT_EINVAL, "NULL argument");
    if (omega < 0 || omega >= g->n_ang) return nofail(RT_EINVAL, "omega out of range");
    if (precision != RT_FP64 && precision != RT_MIXED) return nofail(RT_EINVAL, "bad precision");
    if (g->lost) return nofail(RT_EDEVICE, "the grid has characteristics that could not be tracked");
    if (cudaSetDevice(g->device) != cudaSuccess) return nofail(RT_ECUDA, "cudaSetDevice failed");
    const int64_t s_lo = g->h_ang_seg_off[omega], nseg = g->h_ang_seg_off[omega + 1] - s_lo;
    const size_t pair = precision == RT_FP64 ? sizeof(double2) : sizeof(float2);
    if ((size_t)nseg * pair > NOALLOC_SCRATCH_BYTES) {
        char m[200];
        snprintf(m, sizeof(m), "solid angle %d has %lld segments; the static scratch holds %zu in this precision",
                 omega, (long long)nseg, NOALLOC_SCRATCH_BYTES / pair);
        return nofail(RT_EINVAL, m);
    }
    void *scratch = nullptr;
    char m[200];
    int rc = scratch_for(g->device, &scratch, m, sizeof(m));
    if (rc != RT_OK) return nofail(rc, m);
    const int n = g->nvox;
    const int para = g->interp == RT_PARABOLIC;
    const int b = omega / g->ablk;
    const int64_t b_lo = g->h_ang_seg_off[g->blk_w0[b]];
    const int32_t a0 = (int32_t)(s_lo - b_lo), a1 = (int32_t)(s_lo + nseg - b_lo);
    const int32_t *off = g->d_csr_off + (size_t)b * (n + 1);
    const int64_t r_lo = g->h_ang_ray_off[omega], r_hi = g->h_ang_ray_off[omega + 1];
    cudaError_t e;
    if (precision == RT_FP64) {
        if ((e = rtk::pack_chiS64(n, g->d_chi, g->d_S, g->d_cs64, g->st)) != cudaSuccess) return nofail(RT_ECUDA, cudaGetErrorString(e));
        e = rtk::march_block<double, double2>(g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, s_lo, nseg, g->d_cs64,
                                              g->d_B, g->I_outer, 0, para, (double2 *)scratch, 512, g->st);
        if (e != cudaSuccess) return nofail(RT_ECUDA, cudaGetErrorString(e));
        k_noalloc_gather<double2><<<(n + 255) / 256, 256, 0, g->st>>>(n, off, g->d_perm + b_lo, (const double2 *)scratch,
                                                                     a0, a1, g->d_invL + (size_t)omega * n, Ibar, Lbar);
    } else {
        if ((e = rtk::pack_chiS32(n, g->d_chi, g->d_S, g->d_B, g->d_cs32, g->d_B32, nullptr, g->st)) != cudaSuccess)
            return nofail(RT_ECUDA, cudaGetErrorString(e));
        e = rtk::march_block<float, float2>(g->d_vox, g->d_len32, g->d_ray_off, r_lo, r_hi, s_lo, nseg, g->d_cs32,
                                            g->d_B32, (float)g->I_outer, 0, para, (float2 *)scratch, 512, g->st);
        if (e != cudaSuccess) return nofail(RT_ECUDA, cudaGetErrorString(e));
        k_noalloc_gather<float2><<<(n + 255) / 256, 256, 0, g->st>>>(n, off, g->d_perm + b_lo, (const float2 *)scratch,
                                                                    a0, a1, g->d_invL + (size_t)omega * n, Ibar, Lbar);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return nofail(RT_ECUDA, cudaGetErrorString(e));
    return RT_OK;
}

}  // extern "C"
