// scan.cu -- exclusive prefix sums of per-item counts into int64 offsets
// (ray lists, segment offsets, ownership lists) and a small gather helper.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.h"

namespace rtk {
namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_PER_THREAD = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

// Inclusive block scan of one value per thread (512 threads).
__device__ int64_t block_inclusive(int64_t x, int64_t *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t s = (lane < SCAN_THREADS / 32) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) sh[lane] = s;
    }
    __syncthreads();
    if (wid > 0) x += sh[wid - 1];
    __syncthreads();
    return x;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sums(const int32_t *in, int64_t n, int64_t *tile_sum)
{
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    int64_t s = 0;
    for (int q = 0; q < SCAN_PER_THREAD; ++q)
        if (base + q < n) s += in[base + q];
    int64_t incl = block_inclusive(s, sh);
    if (threadIdx.x == SCAN_THREADS - 1) tile_sum[blockIdx.x] = incl;
}

// Exclusive scan of the tile sums in place, one block, sequential over chunks.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(int64_t *tile_sum, int64_t ntiles)
{
    __shared__ int64_t sh[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < ntiles; c0 += SCAN_THREADS) {
        int64_t i = c0 + threadIdx.x;
        int64_t x = (i < ntiles) ? tile_sum[i] : 0;
        int64_t incl = block_inclusive(x, sh);
        int64_t c = carry;
        if (i < ntiles) tile_sum[i] = c + incl - x;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = c + incl;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_write(const int32_t *in, int64_t n, const int64_t *tile_off,
                                                             int64_t *out)
{
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    int64_t v[SCAN_PER_THREAD];
    int64_t s = 0;
    for (int q = 0; q < SCAN_PER_THREAD; ++q) {
        v[q] = (base + q < n) ? in[base + q] : 0;
        s += v[q];
    }
    int64_t incl = block_inclusive(s, sh);
    int64_t run = tile_off[blockIdx.x] + incl - s;
    for (int q = 0; q < SCAN_PER_THREAD; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
    if (base + SCAN_PER_THREAD >= n && base < n) out[n] = run;  // thread holding the last element
}

__global__ void k_gather_i64(const int64_t *src, const int64_t *idx, int64_t *dst, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_zero_end(int64_t *out) { out[0] = 0; }

}  // namespace

int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

cudaError_t scan_i32(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st)
{
    if (n <= 0) {
        k_zero_end<<<1, 1, 0, st>>>(out);
        return cudaGetLastError();
    }
    int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_tile_sums<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(in, n, tmp);
    k_scan_tiles<<<1, SCAN_THREADS, 0, st>>>(tmp, ntiles);
    k_tile_write<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(in, n, tmp, out);
    return cudaGetLastError();
}

cudaError_t gather_i64(const int64_t *src, const int64_t *idx, int64_t *dst, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_gather_i64<<<(n + 255) / 256, 256, 0, st>>>(src, idx, dst, n);
    return cudaGetLastError();
}

}  // namespace rtk
