// sbr_scan.cu -- exclusive prefix sums used by the radix sort (digit histograms)
// and by the valid-hit compaction (popcount of the per-tile hit masks).
#include "sbr_internal.h"

namespace sbr {

namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned load_item(const unsigned* in, long long i, long long n, bool popc)
{
    if (i >= n) return 0u;
    unsigned v = in[i];
    return popc ? (unsigned)__popc(v) : v;
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ unsigned block_exclusive(unsigned v, unsigned* excl)
{
    __shared__ unsigned s_warp[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned s = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        s_warp[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    unsigned warp_excl = (w == 0) ? 0u : s_warp[w - 1];
    unsigned total = s_warp[(blockDim.x >> 5) - 1];
    *excl = warp_excl + x - v;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_up(const unsigned* in, long long n, bool popc, unsigned* bsum)
{
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += load_item(in, base + k, n, popc);
    unsigned ex;
    unsigned tot = block_exclusive(s, &ex);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_mid(unsigned* bsum, int nb, unsigned* total)
{
    // one block; thread t owns the contiguous slice [t*per, (t+1)*per)
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int lo = threadIdx.x * per;
    unsigned s = 0;
    for (int i = lo; i < lo + per && i < nb; ++i) s += bsum[i];
    unsigned ex;
    unsigned tot = block_exclusive(s, &ex);
    unsigned run = ex;
    for (int i = lo; i < lo + per && i < nb; ++i) {
        unsigned v = bsum[i];
        bsum[i] = run;
        run += v;
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const unsigned* in, long long n, bool popc,
                                                            const unsigned* bsum, unsigned* out)
{
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    unsigned v[kScanItems];
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = load_item(in, base + k, n, popc);
        s += v[k];
    }
    unsigned ex;
    block_exclusive(s, &ex);
    unsigned run = ex + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}
}  // namespace

size_t scan_scratch_bytes(long long n)
{
    long long nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)((nb + 1) * sizeof(unsigned) + 256);
}

// in and out may alias (each block reads its tile before writing it)
cudaError_t scan_exclusive_u32(const unsigned* in, unsigned* out, long long n, bool popc, unsigned* total,
                               void* scratch, cudaStream_t st)
{
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(unsigned), st);
        return cudaSuccess;
    }
    long long nb = (n + kScanTile - 1) / kScanTile;
    unsigned* bsum = (unsigned*)scratch;
    k_scan_up<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, popc, bsum);
    k_scan_mid<<<1, kScanThreads, 0, st>>>(bsum, (int)nb, total);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, popc, bsum, out);
    return cudaGetLastError();
}

cudaError_t scan_popc(const unsigned* mask, unsigned* tile_base, long long n, unsigned* total, void* scratch,
                      cudaStream_t st)
{
    return scan_exclusive_u32(mask, tile_base, n, true, total, scratch, st);
}

}  // namespace sbr
