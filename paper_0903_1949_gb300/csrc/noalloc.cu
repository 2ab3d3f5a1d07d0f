// noalloc.cu -- formal solution of one solid angle without any allocation.
//
// Some callers cannot call cudaMalloc at the moment they need a result: code
// that runs inside another framework's stream-ordered memory pool or under a
// hard device-memory budget that was fully handed out up front, or host code
// that must not take the CUDA allocator's locks.  rt_fs_angle_noalloc serves
// them: it reuses the grid built earlier by rt_grid_create and keeps its
// per-segment scratch in the file-scope device array below instead of any
// allocated buffer.  The caller passes the output buffers.  The call is not
// async-signal-safe (it enters the CUDA runtime): never make it from a signal
// handler.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <mutex>

#include "grid.h"
#include "rt_internal.h"

namespace {

// Per-segment scratch (l I, l lambda) of one solid angle: 16 MiB, i.e. up to
// 1 Mi segments in FP64 or 2 Mi in FP32.  Every GPU on which a grid has been
// created holds this array until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side shadow, not device memory:
// the device address is looked up once per device (by rt_grid_create, which
// allocates anyway) and cached here; the allocation-free call only reads it.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
std::atomic<void *> g_scratch_addr[MAX_DEVICES];

int resolve_scratch(int dev, void **out, char *msg, size_t msglen)
{
    if (dev < 0 || dev >= MAX_DEVICES) {
        snprintf(msg, msglen, "device %d outside the supported range", dev);
        return RT_EINVAL;
    }
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lk(g_mu);
        p = g_scratch_addr[dev].load(std::memory_order_relaxed);
        if (!p) {
            // loads this file's module on the current device (dev), which places the array
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(msg, msglen, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
                return RT_ECUDA;
            }
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return RT_OK;
}

int nofail(int code, const char *m)
{
    rtk::set_last_error(m);
    return code;
}

}  // namespace

namespace rtk {

int noalloc_prepare(int dev)
{
    void *p = nullptr;
    char m[200];
    int rc = resolve_scratch(dev, &p, m, sizeof(m));
    if (rc != RT_OK) return nofail(rc, m);
    cudaError_t e = march_block_preload();
    if (e == cudaSuccess) e = gather_angle_preload();
    if (e == cudaSuccess) e = pack_preload();
    if (e != cudaSuccess) return nofail(RT_ECUDA, cudaGetErrorString(e));
    return RT_OK;
}

}  // namespace rtk

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
    char m[200];
    if ((size_t)nseg * pair > NOALLOC_SCRATCH_BYTES) {
        snprintf(m, sizeof(m), "solid angle %d has %lld segments; the static scratch holds %zu in this precision",
                 omega, (long long)nseg, NOALLOC_SCRATCH_BYTES / pair);
        return nofail(RT_EINVAL, m);
    }
    void *scratch = nullptr;
    int rc = resolve_scratch(g->device, &scratch, m, sizeof(m));  // cached by rt_grid_create
    if (rc != RT_OK) return nofail(rc, m);
    const int n = g->nvox;
    const int para = g->interp == RT_PARABOLIC;
    const int b = omega / g->ablk;
    const int64_t b_lo = g->h_ang_seg_off[g->blk_w0[b]];
    const int64_t a0 = s_lo - b_lo, a1 = s_lo + nseg - b_lo;  // the angle's entries of its block's lists
    const int32_t *off = g->d_csr_off + (size_t)b * (n + 1);
    const int64_t r_lo = g->h_ang_ray_off[omega], r_hi = g->h_ang_ray_off[omega + 1];
    cudaError_t e;
    if (precision == RT_FP64) {
        if ((e = rtk::pack_chiS64(n, g->d_chi, g->d_S, g->d_cs64, g->st)) != cudaSuccess)
            return nofail(RT_ECUDA, cudaGetErrorString(e));
        e = rtk::march_block<double, double2>(g->d_vox, g->d_len64, g->d_ray_off, r_lo, r_hi, s_lo, nseg, g->d_cs64,
                                              g->d_B, g->I_outer, 0, para, (double2 *)scratch, g->march_chunk, g->st);
    } else {
        if ((e = rtk::pack_chiS32(n, g->d_chi, g->d_S, g->d_B, g->d_cs32, g->d_B32, nullptr, g->st)) != cudaSuccess)
            return nofail(RT_ECUDA, cudaGetErrorString(e));
        e = rtk::march_block<float, float2>(g->d_vox, g->d_len32, g->d_ray_off, r_lo, r_hi, s_lo, nseg, g->d_cs32,
                                            g->d_B32, (float)g->I_outer, 0, para, (float2 *)scratch, g->march_chunk,
                                            g->st);
    }
    if (e != cudaSuccess) return nofail(RT_ECUDA, cudaGetErrorString(e));
    // the scratch holds block segments [a0, a1) from its start: base a0
    e = rtk::gather_angle_range(n, off, g->d_perm + b_lo, scratch, a0, precision == RT_MIXED, a0, a1,
                                g->d_invL + (size_t)omega * n, Ibar, Lbar, g->st);
    if (e != cudaSuccess) return nofail(RT_ECUDA, cudaGetErrorString(e));
    return RT_OK;
}

}  // extern "C"
