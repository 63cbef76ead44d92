// Exclusive prefix sums of int32 arrays on the device, used to compact
// selected events, to place the buckets of the counting sorts of the LRF fit
// and to number its work items.  Integer sums: the result does not depend on
// the launch shape.
//
// Three launches over tiles of kTile = 4096 values (1024 threads x 4):
//   1. each tile's total
//   2. one block scans the tile totals in chunks of kTile, carrying the
//      running sum (the number of tiles is at most 2^31 / 4096)
//   3. each tile's exclusive scan plus its tile offset
#include "internal.cuh"

namespace ants {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kPer = 4;
constexpr int kTile = kScanThreads * kPer;

// exclusive scan of one value per thread over the block; returns the block
// total through *total (every thread)
__device__ __forceinline__ int block_exclusive(int v, int *s_warp, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const int before = (wid > 0 ? s_warp[wid - 1] : 0) + x - v;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();  // s_warp is reused by the caller's next round
    return before;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_totals(const int *in, long n, int *tile_sum)
{
    __shared__ int s_warp[32];
    const long base = (long)blockIdx.x * kTile + (long)threadIdx.x * kPer;
    int v = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k)
        if (base + k < n) v += in[base + k];
    int total;
    block_exclusive(v, s_warp, &total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_offsets(int *tile_sum, long n_tiles, int *grand_total)
{
    __shared__ int s_warp[32];
    int carry = 0;
    for (long c0 = 0; c0 < n_tiles; c0 += kTile) {
        const long base = c0 + (long)threadIdx.x * kPer;
        int v[kPer], t = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            v[k] = base + k < n_tiles ? tile_sum[base + k] : 0;
            t += v[k];
        }
        int total;
        int run = carry + block_exclusive(t, s_warp, &total);
#pragma unroll
        for (int k = 0; k < kPer; ++k)
            if (base + k < n_tiles) {
                tile_sum[base + k] = run;
                run += v[k];
            }
        carry += total;
    }
    if (threadIdx.x == 0 && grand_total) *grand_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles(const int *in, long n, const int *tile_off, int *out)
{
    __shared__ int s_warp[32];
    const long base = (long)blockIdx.x * kTile + (long)threadIdx.x * kPer;
    int v[kPer], t = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        t += v[k];
    }
    int total;
    int run = tile_off[blockIdx.x] + block_exclusive(t, s_warp, &total);
#pragma unroll
    for (int k = 0; k < kPer; ++k)
        if (base + k < n) {
            out[base + k] = run;
            run += v[k];
        }
}

}  // namespace

size_t exclusive_scan_tmp_bytes(long n)
{
    const long tiles = (n + kTile - 1) / kTile;
    return (size_t)(tiles > 0 ? tiles : 1) * sizeof(int);
}

int exclusive_scan(const int *in, int *out, long n, int *total_dev, void *tmp, cudaStream_t s)
{
    if (n <= 0) {
        if (total_dev) ANTS_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(int), s), "scan: memset");
        return ANTS_OK;
    }
    const long tiles = (n + kTile - 1) / kTile;
    int *tile_sum = (int *)tmp;
    scan_tile_totals<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, tile_sum);
    scan_tile_offsets<<<1, kScanThreads, 0, s>>>(tile_sum, tiles, total_dev);
    scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, tile_sum, out);
    ANTS_CUDA_TRY(cudaGetLastError(), "scan launch");
    count_launch(3);
    return ANTS_OK;
}

}  // namespace ants
