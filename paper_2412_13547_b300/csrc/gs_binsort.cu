// gs_binsort.cu -- tile/depth binning of the projected Gaussians (the
// tile-Gaussian pair generation and pair sort of the tile-based rasterizer,
// Sec. 3 and the profile of Sec. 3.1), without any host synchronisation.
//
// The result equals sorting the pairs (tile_id << 32 | depth bits, id) by
// (key, id). It is computed in two stages that move fewer bytes than one
// 64-bit key sort:
//   1. the Gaussians are sorted by (depth bits, id) with a stable LSD radix
//      sort of 32-bit keys (N items);
//   2. the pairs are emitted in that order with a 32-bit tile key, and a stable
//      LSD radix sort on the ceil(log2(#tiles)) tile bits orders them by tile;
//      stability keeps the depth order (and id order among equal depths).
// Per-tile ranges are read off the sorted tile keys. The pair count K stays on
// the device; every kernel clamps to the caller's capacity.
#include <cstdio>
#include <mutex>

#include "gs_common.cuh"

// Scratch of gs_bin_sort_static: one array per device, held while the library
// is loaded. Only device code may name it directly; host code must use the
// address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_bin_sort_scratch[GS_BIN_SORT_STATIC_SCRATCH_BYTES];

namespace gs {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItemsPerThread = 16;
constexpr int kTileItems = kSortThreads * kItemsPerThread;  // 4096
constexpr int kRadixBins = 256;
constexpr int kMaxSortBlocks = 148 * 4;
constexpr int kScanItems = 2048;  // items per block of the offsets scan

__device__ __forceinline__ int64_t sort_count(const int64_t* d_num, int64_t cap)
{
    if (d_num == nullptr) return cap;
    int64_t k = *d_num;
    return k < cap ? k : cap;
}

__device__ __forceinline__ void block_segment(int64_t count, int G, int b, int64_t& begin, int64_t& end)
{
    int64_t per = (count + G - 1) / G;
    int64_t seg = ((per + kTileItems - 1) / kTileItems) * kTileItems;
    begin = (int64_t)b * seg;
    end = begin + seg;
    if (begin > count) begin = count;
    if (end > count) end = count;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t x, uint32_t* s_tmp, uint32_t& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kSortWarps ? s_tmp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kSortWarps) s_tmp[lane] = wi - w;
        if (lane == kSortWarps - 1) s_tmp[kSortWarps] = wi;
    }
    __syncthreads();
    uint32_t res = s_tmp[warp] + inc - x;
    total = s_tmp[kSortWarps];
    __syncthreads();
    return res;
}

// ---------------------------------------------------------------------------
// LSD radix sort pass: upsweep (per-block digit histograms), scan (per digit
// over blocks), downsweep (stable rank + scatter, staged in shared memory).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads)
k_radix_upsweep(const uint32_t* __restrict__ keys, const int64_t* __restrict__ d_num, int64_t cap, int shift,
                uint32_t mask, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t s_hist[kSortWarps][kRadixBins];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadixBins; i += kSortThreads) (&s_hist[0][0])[i] = 0u;
    __syncthreads();
    int64_t begin, end;
    block_segment(sort_count(d_num, cap), gridDim.x, blockIdx.x, begin, end);
    // begin is a multiple of 4 items (16 bytes); vector loads for the body
    int64_t body_end = begin + ((end - begin) & ~int64_t(3));
    const uint4* k4 = reinterpret_cast<const uint4*>(keys);
    for (int64_t i = begin / 4 + threadIdx.x; i < body_end / 4; i += kSortThreads) {
        uint4 v = k4[i];
        atomicAdd(&s_hist[warp][(v.x >> shift) & mask], 1u);
        atomicAdd(&s_hist[warp][(v.y >> shift) & mask], 1u);
        atomicAdd(&s_hist[warp][(v.z >> shift) & mask], 1u);
        atomicAdd(&s_hist[warp][(v.w >> shift) & mask], 1u);
    }
    for (int64_t i = body_end + threadIdx.x; i < end; i += kSortThreads)
        atomicAdd(&s_hist[warp][(keys[i] >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBins; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s += s_hist[w][d];
        hist[(int64_t)d * gridDim.x + blockIdx.x] = s;
    }
}

// One block per digit: exclusive scan of hist[d][0..G) in place, total -> totals[d].
__global__ void __launch_bounds__(kSortThreads)
k_radix_scan(uint32_t* __restrict__ hist, int G, uint32_t* __restrict__ totals)
{
    __shared__ uint32_t s_tmp[kSortWarps + 1];
    uint32_t* row = hist + (int64_t)blockIdx.x * G;
    const int per = (G + kSortThreads - 1) / kSortThreads;
    const int i0 = threadIdx.x * per;
    uint32_t local[8];
    uint32_t sum = 0;
    for (int j = 0; j < per; ++j) {
        uint32_t v = (i0 + j < G) ? row[i0 + j] : 0u;
        local[j] = v;
        sum += v;
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan_256(sum, s_tmp, total);
    for (int j = 0; j < per; ++j) {
        if (i0 + j < G) row[i0 + j] = run;
        run += local[j];
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kSortThreads)
k_radix_downsweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                  uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                  const int64_t* __restrict__ d_num, int64_t cap, int shift, uint32_t mask,
                  const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals)
{
    __shared__ uint32_t s_base[kRadixBins];
    __shared__ uint32_t s_warp[kSortWarps][kRadixBins];
    __shared__ uint32_t s_start[kRadixBins];
    __shared__ uint32_t s_count[kRadixBins];
    __shared__ uint32_t s_tmp[kSortWarps + 1];
    __shared__ uint32_t s_keys[kTileItems];
    __shared__ uint32_t s_vals[kTileItems];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int G = gridDim.x;

    int64_t begin, end;
    block_segment(sort_count(d_num, cap), G, blockIdx.x, begin, end);
    {
        uint32_t tot = totals[threadIdx.x];
        uint32_t all;
        uint32_t pre = block_exclusive_scan_256(tot, s_tmp, all);
        s_base[threadIdx.x] = pre + hist[(int64_t)threadIdx.x * G + blockIdx.x];
    }
    __syncthreads();

    for (int64_t tile = begin; tile < end; tile += kTileItems) {
        for (int i = threadIdx.x; i < kSortWarps * kRadixBins; i += kSortThreads) (&s_warp[0][0])[i] = 0u;
        __syncthreads();
        uint32_t k[kItemsPerThread], v[kItemsPerThread], dg[kItemsPerThread], rk[kItemsPerThread];
        const int64_t wbase = tile + warp * (32 * kItemsPerThread);
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            int64_t idx = wbase + j * 32 + lane;
            bool ok = idx < end;
            k[j] = ok ? keys_in[idx] : 0u;
            v[j] = ok ? vals_in[idx] : 0u;
            dg[j] = ok ? ((k[j] >> shift) & mask) : 0xffffffffu;
        }
        // stable rank within the warp: rounds in order, lanes in order
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            uint32_t peers = __match_any_sync(0xffffffffu, dg[j]);
            uint32_t pre = __popc(peers & lt_mask);
            int leader = __ffs(peers) - 1;
            uint32_t basec = (dg[j] != 0xffffffffu) ? s_warp[warp][dg[j]] : 0u;
            rk[j] = basec + pre;
            __syncwarp();
            if (lane == leader && dg[j] != 0xffffffffu) s_warp[warp][dg[j]] = basec + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, tile count, tile-local start
        {
            const int d = threadIdx.x;
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t c = s_warp[w][d];
                s_warp[w][d] = run;
                run += c;
            }
            s_count[d] = run;
            uint32_t all;
            uint32_t st = block_exclusive_scan_256(run, s_tmp, all);
            s_start[d] = st;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            if (dg[j] == 0xffffffffu) continue;
            uint32_t lp = s_start[dg[j]] + s_warp[warp][dg[j]] + rk[j];
            s_keys[lp] = k[j];
            s_vals[lp] = v[j];
        }
        __syncthreads();
        const int n_tile = (int)((end - tile) < kTileItems ? (end - tile) : kTileItems);
        for (int lp = threadIdx.x; lp < n_tile; lp += kSortThreads) {
            uint32_t key = s_keys[lp];
            uint32_t d = (key >> shift) & mask;
            uint32_t gpos = s_base[d] + (uint32_t)lp - s_start[d];
            keys_out[gpos] = key;
            vals_out[gpos] = s_vals[lp];
        }
        __syncthreads();
        s_base[threadIdx.x] += s_count[threadIdx.x];
        __syncthreads();
    }
}

struct SortBufs {
    uint32_t *keys0, *vals0, *keys1, *vals1;
};

// Sorts (keys0, vals0) by bits [0, bits) of the keys; the result lands in
// buffer set (passes % 2 == 0 ? 0 : 1). Returns the number of passes.
int radix_sort(SortBufs b, const int64_t* d_num, int64_t cap, int bits, int G, uint32_t* hist, uint32_t* totals,
               cudaStream_t st)
{
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    int per = (bits + passes - 1) / passes;
    int shift = 0;
    uint32_t *ki = b.keys0, *vi = b.vals0, *ko = b.keys1, *vo = b.vals1;
    for (int p = 0; p < passes; ++p) {
        int nb = (bits - shift) < per ? (bits - shift) : per;
        uint32_t mask = (nb >= 32) ? 0xffffffffu : ((1u << nb) - 1u);
        k_radix_upsweep<<<G, kSortThreads, 0, st>>>(ki, d_num, cap, shift, mask, hist);
        k_radix_scan<<<kRadixBins, kSortThreads, 0, st>>>(hist, G, totals);
        k_radix_downsweep<<<G, kSortThreads, 0, st>>>(ki, vi, ko, vo, d_num, cap, shift, mask, hist, totals);
        uint32_t* t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
        shift += nb;
    }
    return passes;
}

int sort_blocks(int64_t cap)
{
    int64_t tiles = (cap + kTileItems - 1) / kTileItems;
    if (tiles < 1) tiles = 1;
    return (int)(tiles < kMaxSortBlocks ? tiles : kMaxSortBlocks);
}

// ---------------------------------------------------------------------------
// Depth keys, offsets scan, pair emission, tile ranges
// ---------------------------------------------------------------------------
__global__ void k_depth_keys(int n, const float4* __restrict__ splats, const int* __restrict__ tiles_touched,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ ids)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    float depth = splats[3 * (int64_t)g + 2].y;
    // depth > z_near > 0 for visible Gaussians: the float bits order like the value
    keys[g] = tiles_touched[g] > 0 ? __float_as_uint(depth) : 0xffffffffu;
    ids[g] = (uint32_t)g;
}

// Block sums of tiles_touched gathered in depth order.
__global__ void __launch_bounds__(kSortThreads)
k_scan_reduce(int n, const uint32_t* __restrict__ perm, const int* __restrict__ tiles_touched,
              unsigned long long* __restrict__ partials)
{
    __shared__ uint32_t s_tmp[kSortWarps + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanItems;
    unsigned long long sum = 0;
    for (int j = threadIdx.x; j < kScanItems; j += kSortThreads) {
        int64_t k = base + j;
        if (k < n) sum += (unsigned)tiles_touched[perm[k]];
    }
    // 64-bit block reduction via warp shuffles
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    __shared__ unsigned long long s_sum[kSortWarps];
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kSortWarps; ++w) t += s_sum[w];
        partials[blockIdx.x] = t;
    }
    (void)s_tmp;
}

// Single block: exclusive scan of the block sums (nb values) in place; total -> *d_total.
__global__ void __launch_bounds__(1024) k_scan_partials(int nb, unsigned long long* __restrict__ partials,
                                                        int64_t* __restrict__ d_total)
{
    __shared__ unsigned long long s_w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        unsigned long long x = i < nb ? partials[i] : 0ull;
        unsigned long long inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_w[lane];
            unsigned long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            s_w[lane] = wi - w;
        }
        __syncthreads();
        unsigned long long excl = carry + s_w[warp] + inc - x;
        if (i < nb) partials[i] = excl;
        __syncthreads();
        // carry of this chunk = exclusive prefix of the last thread + its value
        __shared__ unsigned long long s_carry;
        if (threadIdx.x == 1023) s_carry = excl + x;
        __syncthreads();
        carry = s_carry;
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_total = (int64_t)carry;
}

// offsets[k] = sum of tiles_touched[perm[j]] for j < k (64-bit).
__global__ void __launch_bounds__(kSortThreads)
k_scan_down(int n, const uint32_t* __restrict__ perm, const int* __restrict__ tiles_touched,
            const unsigned long long* __restrict__ partials, unsigned long long* __restrict__ offsets)
{
    __shared__ uint32_t s_tmp[kSortWarps + 1];
    constexpr int per = kScanItems / kSortThreads;  // 8 consecutive items per thread
    const int64_t base = (int64_t)blockIdx.x * kScanItems + threadIdx.x * per;
    uint32_t c[per];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < per; ++j) {
        int64_t k = base + j;
        c[j] = k < n ? (uint32_t)tiles_touched[perm[k]] : 0u;
        sum += c[j];
    }
    // per-block sums fit in 32 bits: at most 2048 * 2^15 tiles
    uint32_t total;
    uint32_t pre = block_exclusive_scan_256(sum, s_tmp, total);
    unsigned long long run = partials[blockIdx.x] + pre;
#pragma unroll
    for (int j = 0; j < per; ++j) {
        int64_t k = base + j;
        if (k < n) offsets[k] = run;
        run += c[j];
    }
}

// Warp-cooperative pair emission: a warp takes 32 consecutive Gaussians of the
// depth order and writes their pairs with consecutive lanes on consecutive
// output slots (coalesced), each lane finding its owner by a shuffle search.
__global__ void __launch_bounds__(kSortThreads)
k_emit(int n, const uint32_t* __restrict__ perm, const unsigned long long* __restrict__ offsets,
       const int64_t* __restrict__ d_total, const int4* __restrict__ rects, int tiles_x, int64_t cap,
       uint32_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * kSortThreads + threadIdx.x - lane);
    if (w0 >= n) return;
    const int64_t total = *d_total;
    const int64_t k = w0 + lane;
    const bool in = k < n;
    const unsigned long long my_off = in ? offsets[k] : (unsigned long long)total;
    const unsigned long long base = __shfl_sync(0xffffffffu, my_off, 0);
    const int64_t wend = (w0 + 32 < n) ? (int64_t)offsets[w0 + 32] : total;
    uint32_t g = in ? perm[k] : 0u;
    int4 rc = in ? rects[g] : make_int4(0, 0, -1, -1);
    const uint32_t rel_start = (uint32_t)(my_off - base);
    const int width = rc.z - rc.x + 1;
    for (int64_t c0 = (int64_t)base; c0 < wend; c0 += 32) {
        const int64_t j = c0 + lane;
        const uint32_t rel = (uint32_t)(j - (int64_t)base);
        int lo = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            uint32_t s = __shfl_sync(0xffffffffu, rel_start, lo + step);
            if (s <= rel) lo += step;
        }
        const uint32_t o_start = __shfl_sync(0xffffffffu, rel_start, lo);
        const int o_x0 = __shfl_sync(0xffffffffu, rc.x, lo);
        const int o_y0 = __shfl_sync(0xffffffffu, rc.y, lo);
        const int o_w = __shfl_sync(0xffffffffu, width, lo);
        const uint32_t o_g = __shfl_sync(0xffffffffu, g, lo);
        if (j < wend && j < cap) {
            const uint32_t local = rel - o_start;
            const uint32_t ly = local / (uint32_t)o_w;
            const uint32_t lx = local - ly * (uint32_t)o_w;
            keys[j] = (uint32_t)(o_y0 + (int)ly) * (uint32_t)tiles_x + (uint32_t)(o_x0 + (int)lx);
            vals[j] = o_g;
        }
    }
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, const int64_t* __restrict__ d_total, int64_t cap,
                         uint2* __restrict__ ranges)
{
    const int64_t K = *d_total;
    if (K > cap) return;  // overflow: ranges stay empty
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t t = keys[i];
        if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
        if (i == K - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

// Workspace layout (each region 256-byte aligned)
struct Ws {
    uint32_t *dkeys0, *dkeys1, *perm0, *perm1;
    unsigned long long *offsets, *partials;
    uint32_t *tkeys0, *tkeys1, *tvals;
    uint32_t *hist, *totals;
    size_t bytes;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Ws carve(void* base, int n, int64_t cap)
{
    Ws w{};
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = static_cast<char*>(base) + off;
        off += align256(bytes);
        return p;
    };
    size_t nn = (size_t)(n > 0 ? n : 1);
    size_t cc = (size_t)(cap > 0 ? cap : 1);
    int nb = (int)((nn + kScanItems - 1) / kScanItems);
    int G = sort_blocks(cap > n ? cap : n);
    w.dkeys0 = (uint32_t*)take(nn * 4);
    w.dkeys1 = (uint32_t*)take(nn * 4);
    w.perm0 = (uint32_t*)take(nn * 4);
    w.perm1 = (uint32_t*)take(nn * 4);
    w.offsets = (unsigned long long*)take((nn + 1) * 8);
    w.partials = (unsigned long long*)take(((size_t)nb + 1) * 8);
    w.tkeys0 = (uint32_t*)take(cc * 4);
    w.tkeys1 = (uint32_t*)take(cc * 4);
    w.tvals = (uint32_t*)take(cc * 4);
    w.hist = (uint32_t*)take((size_t)kRadixBins * G * 4);
    w.totals = (uint32_t*)take(kRadixBins * 4);
    w.bytes = off;
    return w;
}

}  // namespace
}  // namespace gs

extern "C" {

size_t gs_bin_sort_workspace_size(int32_t n, int64_t capacity, int32_t num_tiles)
{
    (void)num_tiles;
    if (n < 0 || capacity < 0) return 0;
    return gs::carve(nullptr, n, capacity).bytes + 256;
}

int32_t gs_bin_sort(int32_t n, const int32_t* rects, const int32_t* tiles_touched, const float* splats,
                    int32_t tiles_x, int32_t tiles_y, void* workspace, size_t workspace_bytes, int64_t capacity,
                    uint32_t* sorted_ids, uint32_t* ranges, int64_t* num_pairs, gs_stream_t stream)
{
    using namespace gs;
    if (n < 0 || capacity < 0 || capacity > 0x7fffffffLL || tiles_x <= 0 || tiles_y <= 0) {
        gs_host::set_error("gs_bin_sort: bad sizes (n >= 0, 0 <= capacity < 2^31, tiles > 0)");
        return GS_ERR_ARG;
    }
    if ((int64_t)tiles_x * tiles_y > (1LL << 30)) {
        gs_host::set_error("gs_bin_sort: too many tiles");
        return GS_ERR_ARG;
    }
    if (!ranges || !num_pairs || (n > 0 && (!rects || !tiles_touched || !splats || !workspace)) ||
        (capacity > 0 && !sorted_ids)) {
        gs_host::set_error("gs_bin_sort: null pointer");
        return GS_ERR_ARG;
    }
    uintptr_t base = reinterpret_cast<uintptr_t>(workspace);
    void* ws_al = reinterpret_cast<void*>((base + 255) & ~uintptr_t(255));
    size_t slack = reinterpret_cast<uintptr_t>(ws_al) - base;
    Ws w = carve(ws_al, n, capacity);
    if (n > 0 && workspace_bytes < w.bytes + slack) {
        gs_host::set_error("gs_bin_sort: workspace too small");
        return GS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t num_tiles = (int64_t)tiles_x * tiles_y;
    cudaMemsetAsync(ranges, 0, (size_t)num_tiles * 2 * sizeof(uint32_t), st);
    if (n == 0) {
        cudaMemsetAsync(num_pairs, 0, sizeof(int64_t), st);
        return gs_host::check_launch("gs_bin_sort");
    }
    // 1. sort Gaussians by (depth bits, id)
    k_depth_keys<<<(n + 255) / 256, 256, 0, st>>>(n, reinterpret_cast<const float4*>(splats), tiles_touched,
                                                  w.dkeys0, w.perm0);
    int Gd = sort_blocks(n);
    radix_sort(SortBufs{w.dkeys0, w.perm0, w.dkeys1, w.perm1}, nullptr, n, 32, Gd, w.hist, w.totals, st);
    // 4 passes: the result is back in (dkeys0, perm0)
    // 2. offsets of each Gaussian's pairs in depth order, and K
    int nb = (n + kScanItems - 1) / kScanItems;
    k_scan_reduce<<<nb, kSortThreads, 0, st>>>(n, w.perm0, tiles_touched, w.partials);
    k_scan_partials<<<1, 1024, 0, st>>>(nb, w.partials, num_pairs);
    k_scan_down<<<nb, kSortThreads, 0, st>>>(n, w.perm0, tiles_touched, w.partials, w.offsets);
    // 3. emit (tile key, id) in depth order, then stable sort by tile bits
    int bits = 1;
    while ((1LL << bits) < num_tiles) ++bits;
    int passes = (bits + 7) / 8;
    uint32_t* v_emit = (passes % 2 == 0) ? sorted_ids : w.tvals;
    uint32_t* v_other = (passes % 2 == 0) ? w.tvals : sorted_ids;
    if (capacity > 0) {
        k_emit<<<(n + kSortThreads - 1) / kSortThreads, kSortThreads, 0, st>>>(
            n, w.perm0, w.offsets, num_pairs, reinterpret_cast<const int4*>(rects), tiles_x, capacity, w.tkeys0,
            v_emit);
        int Gt = sort_blocks(capacity);
        radix_sort(SortBufs{w.tkeys0, v_emit, w.tkeys1, v_other}, num_pairs, capacity, bits, Gt, w.hist, w.totals,
                   st);
        uint32_t* kfinal = (passes % 2 == 0) ? w.tkeys0 : w.tkeys1;
        k_ranges<<<148 * 8, 256, 0, st>>>(kfinal, num_pairs, capacity, reinterpret_cast<uint2*>(ranges));
    }
    return gs_host::check_launch("gs_bin_sort");
}

// Device address of g_bin_sort_scratch, looked up once per device with that
// device current.
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};
}  // namespace

int32_t gs_bin_sort_static(int32_t n, const int32_t* rects, const int32_t* tiles_touched, const float* splats,
                           int32_t tiles_x, int32_t tiles_y, int64_t capacity, uint32_t* sorted_ids,
                           uint32_t* ranges, int64_t* num_pairs, gs_stream_t stream)
{
    if (n < 0 || capacity < 0 || tiles_x <= 0 || tiles_y <= 0) {
        gs_host::set_error("gs_bin_sort_static: bad sizes (n >= 0, capacity >= 0, tiles > 0)");
        return GS_ERR_ARG;
    }
    const size_t need = gs_bin_sort_workspace_size(n, capacity, tiles_x * tiles_y);
    if (need > (size_t)GS_BIN_SORT_STATIC_SCRATCH_BYTES) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "gs_bin_sort_static: n=%d, capacity=%lld need %zu bytes of scratch; the static array holds "
                      "%u (use gs_bin_sort with a caller workspace)",
                      n, (long long)capacity, need, (unsigned)GS_BIN_SORT_STATIC_SCRATCH_BYTES);
        gs_host::set_error(msg);
        return GS_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        gs_host::set_error(e != cudaSuccess ? cudaGetErrorString(e) : "gs_bin_sort_static: device index too large");
        return GS_ERR_CUDA;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (g_static_ptr[dev] == nullptr) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_bin_sort_scratch);
            if (e != cudaSuccess || p == nullptr) {
                char msg[256];
                std::snprintf(msg, sizeof(msg), "gs_bin_sort_static: cudaGetSymbolAddress failed: %s",
                              cudaGetErrorString(e));
                gs_host::set_error(msg);
                return GS_ERR_CUDA;
            }
            g_static_ptr[dev] = p;
        }
        scratch = g_static_ptr[dev];
    }
    return gs_bin_sort(n, rects, tiles_touched, splats, tiles_x, tiles_y, scratch,
                       (size_t)GS_BIN_SORT_STATIC_SCRATCH_BYTES, capacity, sorted_ids, ranges, num_pairs, stream);
}

}  // extern "C"
