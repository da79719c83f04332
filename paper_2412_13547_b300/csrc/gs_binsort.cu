// gs_binsort.cu -- tile/depth binning of the projected Gaussians (the
// tile-Gaussian pair generation and pair sort of the tile-based rasterizer,
// Sec. 3 and the profile of Sec. 3.1), without any host synchronisation.
//
// The result equals sorting the pairs (tile_id << 32 | depth bits, id) by
// (key, id): every tile's list of Gaussian ids, front to back. It is built
// without materialising or sorting pair keys:
//   1. the visible Gaussians are sorted by (depth bits, id) with a stable LSD
//      radix sort of 32-bit keys (4 passes; culled Gaussians carry the all-ones
//      key and the first pass drops them, so the later ones sort the visible
//      ones only and level 1 reads their count from the device);
//   2. a two-level counting scatter (rows, then tiles within a row) writes each
//      id straight into its final slot (see the section comment below).
// The pair count K stays on the device; every kernel checks it against the
// caller's capacity.
#include <algorithm>
#include <cstdio>

#include "gs_common.cuh"

// Scratch of gs_bin_sort_static: one array per device, held while the library
// is loaded. Only device code may name it directly; host code must use the
// address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_bin_sort_scratch[GS_BIN_SORT_STATIC_SCRATCH_BYTES];

namespace gs {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItemsPerThread = 8;
constexpr int kTileItems = kSortThreads * kItemsPerThread;  // 2048
constexpr int kRadixBins = 256;
constexpr int kSortBlocksPerSM = 4;  // one wave of the downsweep (64 registers: 4 CTAs per SM)
constexpr uint32_t kCulledKey = 0xffffffffu;  // depth key of a culled Gaussian (a visible one never takes it)

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
                uint32_t mask, bool drop, uint32_t* __restrict__ hist)
{
    kernel_prologue();
    __shared__ uint32_t s_hist[kSortWarps][kRadixBins];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadixBins; i += kSortThreads) (&s_hist[0][0])[i] = 0u;
    __syncthreads();
    int64_t begin, end;
    block_segment(sort_count(d_num, cap), gridDim.x, blockIdx.x, begin, end);
    // begin is a multiple of 4 items: 16-byte vector loads for the body when the key array
    // is 16-byte aligned (a caller's key array need only be 4-byte aligned)
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
    int64_t body_end = vec ? begin + ((end - begin) & ~int64_t(3)) : begin;
    const uint4* k4 = reinterpret_cast<const uint4*>(keys);
    // drop: keys equal to kCulledKey are left out (not counted here, not written by the downsweep)
    for (int64_t i = begin / 4 + threadIdx.x; i < body_end / 4; i += kSortThreads) {
        const uint4 v = k4[i];
        if (!drop || v.x != kCulledKey) atomicAdd(&s_hist[warp][(v.x >> shift) & mask], 1u);
        if (!drop || v.y != kCulledKey) atomicAdd(&s_hist[warp][(v.y >> shift) & mask], 1u);
        if (!drop || v.z != kCulledKey) atomicAdd(&s_hist[warp][(v.z >> shift) & mask], 1u);
        if (!drop || v.w != kCulledKey) atomicAdd(&s_hist[warp][(v.w >> shift) & mask], 1u);
    }
    for (int64_t i = body_end + threadIdx.x; i < end; i += kSortThreads) {
        const uint32_t v = keys[i];
        if (!drop || v != kCulledKey) atomicAdd(&s_hist[warp][(v >> shift) & mask], 1u);
    }
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
    kernel_prologue();
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

__global__ void __launch_bounds__(kSortThreads, 4)
k_radix_downsweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                  uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                  const int64_t* __restrict__ d_num, int64_t cap, int shift, uint32_t mask, bool drop,
                  const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals,
                  int64_t* __restrict__ kept_out)
{
    kernel_prologue();
    __shared__ uint32_t s_base[kRadixBins];
    __shared__ uint32_t s_warp[kSortWarps][kRadixBins];
    __shared__ uint32_t s_start[kRadixBins];
    __shared__ uint32_t s_count[kRadixBins];
    __shared__ uint32_t s_tmp[kSortWarps + 1];
    __shared__ uint32_t s_ntile;
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
        // the number of items kept (all of them unless culled keys are dropped)
        if (kept_out != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *kept_out = (int64_t)all;
    }
    __syncthreads();

    for (int64_t tile = begin; tile < end; tile += kTileItems) {
        for (int i = threadIdx.x; i < kSortWarps * kRadixBins; i += kSortThreads) (&s_warp[0][0])[i] = 0u;
        __syncthreads();
        // per item: its key, value and rank among the warp's items of its digit (the digit
        // is recomputed from the key where needed, to keep the registers for 4 CTAs per SM)
        uint32_t k[kItemsPerThread], v[kItemsPerThread], rk[kItemsPerThread];
        uint32_t okm = 0u;  // bit j: item j is in range and kept
        const int64_t wbase = tile + warp * (32 * kItemsPerThread);
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            int64_t idx = wbase + j * 32 + lane;
            bool ok = idx < end;
            k[j] = ok ? keys_in[idx] : 0u;
            v[j] = ok ? (vals_in != nullptr ? vals_in[idx] : (uint32_t)idx) : 0u;
            ok = ok && !(drop && k[j] == kCulledKey);
            okm |= ok ? (1u << j) : 0u;
        }
        // stable rank within the warp: rounds in order, lanes in order. The lanes holding the
        // same digit come from one ballot per digit bit (the digit has at most 8 bits).
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            const bool ok = (okm >> j) & 1u;
            const uint32_t dg = ok ? ((k[j] >> shift) & mask) : 0xffffffffu;
            uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint32_t bit = (dg >> b) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bb : ~bb;
            }
            uint32_t pre = __popc(peers & lt_mask);
            int leader = __ffs(peers) - 1;
            uint32_t basec = ok ? s_warp[warp][dg] : 0u;
            rk[j] = basec + pre;
            __syncwarp();
            if (lane == leader && ok) s_warp[warp][dg] = basec + __popc(peers);
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
            if (d == 0) s_ntile = all;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            if (!((okm >> j) & 1u)) continue;
            const uint32_t dg = (k[j] >> shift) & mask;
            uint32_t lp = s_start[dg] + s_warp[warp][dg] + rk[j];
            s_keys[lp] = k[j];
            s_vals[lp] = v[j];
        }
        __syncthreads();
        const int n_tile = (int)s_ntile;  // the tile's kept items
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
    bool iota_vals;  // vals0 holds 0, 1, 2, ... on entry: the first pass makes them instead of reading them
    uint32_t* keys2;  // with an even pass count the result keys land here instead of keys0 (which is
                      // then only read, e.g. a caller's array); null: keys0
};

// Sorts (keys0, vals0) by bits [0, bits) of the keys; the result lands in
// buffer set (passes % 2 == 0 ? 0 : 1), its keys in keys2 when given. Returns
// the number of passes. kept (nullable): the first pass drops the items whose
// key is kCulledKey and writes the number kept here; the later passes and the
// result cover only those (the dropped ones would all sort last, in index
// order, so the kept prefix is the same as in the full sort).
int radix_sort(SortBufs b, const int64_t* d_num, int64_t cap, int bits, int G, uint32_t* hist, uint32_t* totals,
               int64_t* kept, cudaStream_t st)
{
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    int per = (bits + passes - 1) / passes;
    int shift = 0;
    uint32_t* k0 = b.keys2 ? b.keys2 : b.keys0;
    uint32_t *ki = b.keys0, *vi = b.vals0, *ko = b.keys1, *vo = b.vals1;
    for (int p = 0; p < passes; ++p) {
        int nb = (bits - shift) < per ? (bits - shift) : per;
        uint32_t mask = (nb >= 32) ? 0xffffffffu : ((1u << nb) - 1u);
        const bool drop = p == 0 && kept != nullptr;
        const int64_t* cnt = (p > 0 && kept != nullptr) ? kept : d_num;
        gs::launch(k_radix_upsweep, G, kSortThreads, 0, st, ki, cnt, cap, shift, mask, drop, hist);
        gs::launch(k_radix_scan, kRadixBins, kSortThreads, 0, st, hist, G, totals);
        const uint32_t* vin = (p == 0 && b.iota_vals) ? nullptr : vi;
        gs::launch(k_radix_downsweep, G, kSortThreads, 0, st, ki, vin, ko, vo, cnt, cap, shift, mask, drop, hist,
                   totals, drop ? kept : nullptr);
        // the next pass reads what this one wrote and writes the other set (set 0's keys in k0)
        uint32_t* t = vi; vi = vo; vo = t;
        ki = ko;
        ko = (ko == b.keys1) ? k0 : b.keys1;
        shift += nb;
    }
    return passes;
}

int sort_blocks(int64_t cap)
{
    int64_t tiles = (cap + kTileItems - 1) / kTileItems;
    if (tiles < 1) tiles = 1;
    const int64_t wave = (int64_t)gs_host::sm_count() * kSortBlocksPerSM;
    return (int)(tiles < wave ? tiles : wave);
}

// ---------------------------------------------------------------------------
// Depth keys and the pair count
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool rect_in_grid(int4 r, int TX, int TY)
{
    return r.x >= 0 && r.y >= 0 && r.x <= r.z && r.y <= r.w && r.z < TX && r.w < TY;
}

constexpr int kKeyThreads = 256;
constexpr int kKeysPerThread = 4;

// One pass over the Gaussians when the caller gives no depth keys: the depth
// sort key of each (the float bits of the view depth, which order like the
// value since depth > z_near > 0 for a visible Gaussian; all ones for a culled
// one). Each thread takes kKeysPerThread Gaussians a block apart, loads first.
__global__ void __launch_bounds__(kKeyThreads)
k_depth_keys(int n, const float4* __restrict__ splats, const int* __restrict__ tiles_touched,
             uint32_t* __restrict__ keys)
{
    kernel_prologue();
    const int64_t g0 = (int64_t)blockIdx.x * (kKeyThreads * kKeysPerThread) + threadIdx.x;
    int tt[kKeysPerThread];
#pragma unroll
    for (int j = 0; j < kKeysPerThread; ++j) {
        const int64_t g = g0 + j * kKeyThreads;
        tt[j] = g < n ? tiles_touched[g] : 0;
    }
#pragma unroll
    for (int j = 0; j < kKeysPerThread; ++j) {
        const int64_t g = g0 + j * kKeyThreads;
        if (g >= n) break;
        // all ones marks a culled Gaussian: a visible one never takes it (even with bad input)
        keys[g] = tt[j] > 0 ? min(__float_as_uint(splats[4 * g + 2].y), 0xfffffffeu) : 0xffffffffu;
    }
}

// ---------------------------------------------------------------------------
// Two-level counting scatter. The pairs are never stored with keys nor sorted:
//   level 1 bins the depth-ordered Gaussians into per-row lists (one entry per
//   tile row a Gaussian's rect spans, carrying the rect's x-extent), level 2
//   bins each row list into the row's tiles. Each level is a counting scatter: per-warp counts from a
//   difference array, exclusive scans down the columns of the count matrix for
//   every warp's first slot in every bin, then each warp regenerates its items
//   in order and ranks them per bin with __match_any_sync and shared counters.
//   Order is kept at both levels, so every tile's list is in depth order (and
//   id order among equal depths). A warp writes to at most one row's tiles at a
//   time, so the partly written sectors in flight stay few enough for L2 to
//   merge them before HBM sees them.
// ---------------------------------------------------------------------------
constexpr int kLvlWarps = 8;              // warps per block of the level kernels
constexpr int kLvlThreads = kLvlWarps * 32;
constexpr int kRowChunk = 512;            // Gaussians per level-1 warp
constexpr int kSegLen = 2048;             // row-list entries per level-2 segment (one CTA of 8 warps)
constexpr int kScanRows = 32;             // matrix rows per block of the column scans
constexpr int kMaxGridSide = 4096;        // tiles_x, tiles_y limit (per-warp shared counters)

__device__ __forceinline__ bool overflow(const int64_t* d_K, int64_t cap) { return *d_K > cap; }

// Inclusive scan of len values d[0..len) in place by one warp.
__device__ __forceinline__ void warp_inclusive_scan_smem(int* d, int len, int lane)
{
    int carry = 0;
    for (int b = 0; b < len; b += 32) {
        const int i = b + lane;
        int v = i < len ? d[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        v += carry;
        if (i < len) d[i] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    __syncwarp();
}

// Flattened item j of a warp's round -> (owner lane, item offset in the owner):
// the largest lane whose exclusive prefix `begin` is <= j.
__device__ __forceinline__ int owner_lane(uint32_t begin, uint32_t j)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const uint32_t sb = __shfl_sync(0xffffffffu, begin, lo + step);
        if (sb <= j) lo += step;
    }
    return lo;
}

__device__ __forceinline__ uint32_t shfl_val(uint32_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ uint2 shfl_val(uint2 v, int src)
{
    return make_uint2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// One round of a warp's counting scatter. Lane i holds an item val spanning
// bins [b0, b0 + nb) (nb = 0: none); cnt[b] is the warp's next free slot of
// bin b. Every item is written to each of its bins, in lane order within a
// bin, and cnt is advanced. When the round's bins lie within 32 consecutive
// ones, one ballot per bin gives every lane its rank directly (scratch: 64
// words of the warp's shared memory); otherwise the items are flattened 32
// at a time and ranked per bin with __match_any_sync.
template <typename V>
__device__ __forceinline__ void scatter_round(V val, int b0, int nb, uint32_t* cnt, uint32_t* scratch, V* out,
                                              int64_t cap, int lane)
{
    const uint32_t lt_mask = (1u << lane) - 1u;
    const bool has = nb > 0;
    const int lo = __reduce_min_sync(0xffffffffu, has ? b0 : 0x7fffffff);
    const int hi = __reduce_max_sync(0xffffffffu, has ? b0 + nb - 1 : -1);
    if (lo > hi) return;  // no items in the round (uniform)
    if (hi - lo < 32) {
        uint32_t my_m = 0u;  // lane t: the lanes whose items cover bin lo + t
        for (int t = 0; t <= hi - lo; ++t) {
            const int b = lo + t;
            const uint32_t m = __ballot_sync(0xffffffffu, has && b0 <= b && b < b0 + nb);
            my_m = lane == t ? m : my_m;
        }
        uint32_t* s_base = scratch;
        uint32_t* s_mask = scratch + 32;
        if (lane <= hi - lo) {
            const uint32_t base = cnt[lo + lane];
            s_base[lane] = base;
            s_mask[lane] = my_m;
            cnt[lo + lane] = base + __popc(my_m);
        }
        __syncwarp();
        for (int k = 0; k < nb; ++k) {
            const int t = b0 + k - lo;
            const uint32_t pos = s_base[t] + __popc(s_mask[t] & lt_mask);
            if ((int64_t)pos < cap) out[pos] = val;
        }
        __syncwarp();
        return;
    }
    uint32_t inc = (uint32_t)nb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    const uint32_t begin = inc - (uint32_t)nb;
    for (uint32_t j0 = 0; j0 < total; j0 += 32) {
        const uint32_t j = j0 + lane;
        const int o = owner_lane(begin, j);
        const uint32_t o_begin = __shfl_sync(0xffffffffu, begin, o);
        const int o_b0 = __shfl_sync(0xffffffffu, b0, o);
        const V o_val = shfl_val(val, o);
        const bool valid = j < total;
        const uint32_t bin = valid ? (uint32_t)o_b0 + (j - o_begin) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, bin);
        uint32_t pos = 0;
        if (valid) pos = cnt[bin] + __popc(peers & lt_mask);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[bin] += __popc(peers);
        __syncwarp();
        if (valid && (int64_t)pos < cap) out[pos] = o_val;
    }
}

// Level-1 input of sorted position k: the Gaussian id and whether it is
// visible (its sorted depth key is not the culled key: the sort dropped the
// culled ones, this keeps the test for the record).
__device__ __forceinline__ uint32_t lvl1_id(const uint32_t* perm, const uint32_t* skeys, int k, int k1, bool& vis)
{
    vis = false;
    if (k >= k1) return 0u;
    vis = skeys[k] != kCulledKey;
    return perm[k];
}

// Level 1a: per level-1 warp (chunk of kRowChunk depth-ordered Gaussians), the
// number of its Gaussians whose rect spans each tile row -> M1[chunk][row],
// and K, the number of (Gaussian, tile) pairs: the rect areas of the visible
// Gaussians inside the grid, summed into *d_K (zeroed by the caller; complete
// when this kernel ends, and checked against the capacity by every later
// one). Counting from the rects the scatters use keeps every row list within
// K slots. The rects of four rounds are fetched together.
__global__ void __launch_bounds__(kLvlThreads)
k_row_hist(int n, const int64_t* __restrict__ d_nvis, int C1, const uint32_t* __restrict__ perm,
           const uint32_t* __restrict__ skeys, const int4* __restrict__ rects, int TX, int TY,
           int64_t* __restrict__ d_K, uint32_t* __restrict__ M1)
{
    kernel_prologue();
    extern __shared__ int s_lvl[];
    constexpr int U = 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kLvlWarps + warp;
    if (c >= C1) return;
    int* d = s_lvl + warp * (TY + 1);
    for (int i = lane; i <= TY; i += 32) d[i] = 0;
    __syncwarp();
    const int k0 = c * kRowChunk, k1 = min(k0 + kRowChunk, (int)min((int64_t)n, *d_nvis));
    unsigned long long area = 0;
    for (int kb = k0 + lane; kb < k1; kb += 32 * U) {
        uint32_t g[U];
        bool vis[U];
#pragma unroll
        for (int j = 0; j < U; ++j) g[j] = lvl1_id(perm, skeys, kb + 32 * j, k1, vis[j]);
        int4 r[U];
#pragma unroll
        for (int j = 0; j < U; ++j) r[j] = vis[j] ? rects[g[j]] : make_int4(0, 0, -1, -1);
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (!vis[j] || !rect_in_grid(r[j], TX, TY)) continue;
            atomicAdd(&d[r[j].y], 1);
            atomicAdd(&d[r[j].w + 1], -1);
            area += (unsigned long long)(r[j].z - r[j].x + 1) * (unsigned long long)(r[j].w - r[j].y + 1);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) area += __shfl_down_sync(0xffffffffu, area, o);
    if (lane == 0 && area) atomicAdd(reinterpret_cast<unsigned long long*>(d_K), area);
    __syncwarp();
    warp_inclusive_scan_smem(d, TY, lane);
    for (int ty = lane; ty < TY; ty += 32) M1[(int64_t)c * TY + ty] = (uint32_t)d[ty];
}

// Column scans of a count matrix M (R rows x Cc columns). Level 1 stores it
// row-major (element (r, c) at r * Cc + c). Level 2 stores only the rows that
// exist: column c = (ty, tx) of the tile grid (col_div = TX) has the rows of
// its tile row's segments, element (r, c) at (rowbase[ty] + r) * TX + tx.
// Column c uses only its first active(c) rows when `active` is given
// (active(c) = active[c / col_div]); the others count as zero.
__device__ __forceinline__ int active_rows(const uint32_t* active, int col_div, int c, int R)
{
    return active ? min(R, (int)active[c / col_div]) : R;
}

__device__ __forceinline__ int64_t mat_at(const uint32_t* rowbase, int col_div, int Cc, int c, int r)
{
    return rowbase ? ((int64_t)rowbase[c / col_div] + r) * col_div + c % col_div : (int64_t)r * Cc + c;
}

// One warp per (column, block of kScanRows = 32 rows), lane = row: blocks of
// 8 warps take 8 consecutive columns and loop over the row blocks by
// gridDim.y, up to the column's active rows.
constexpr int kColsPerBlock = kLvlWarps;

__global__ void __launch_bounds__(kLvlThreads)
k_col_segsum(int R, int Cc, const uint32_t* __restrict__ M, uint32_t* __restrict__ SS,
             const uint32_t* __restrict__ active, const uint32_t* __restrict__ rowbase, int col_div,
             const int64_t* __restrict__ d_K, int64_t cap)
{
    kernel_prologue();
    const int c = blockIdx.x * kColsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= Cc || overflow(d_K, cap)) return;  // uniform over the warp
    const int act = active_rows(active, col_div, c, R);
    for (int by = blockIdx.y; by * kScanRows < act; by += gridDim.y) {
        const int r = by * kScanRows + lane;
        uint32_t x = r < act ? M[mat_at(rowbase, col_div, Cc, c, r)] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) SS[(int64_t)by * Cc + c] = x;
    }
}

// Exclusive scan of column c's segment sums in place by one warp (32 segments
// per step; only the ceil(active / kScanRows) segments that hold active rows),
// the column total into total[c].
__device__ __forceinline__ void col_total_warp(int R, int Cc, int c, uint32_t* SS, uint32_t* total,
                                               const uint32_t* active, int col_div, int lane)
{
    const int nsb = (active_rows(active, col_div, c, R) + kScanRows - 1) / kScanRows;
    uint32_t run = 0;
    for (int b0 = 0; b0 < nsb; b0 += 32) {
        const int b = b0 + lane;
        const uint32_t x = b < nsb ? SS[(int64_t)b * Cc + c] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (b < nsb) SS[(int64_t)b * Cc + c] = run + inc - x;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) total[c] = run;
}

// One warp per column: col_total_warp over all Cc columns.
__global__ void k_col_totals(int R, int Cc, uint32_t* __restrict__ SS, uint32_t* __restrict__ total,
                             const uint32_t* __restrict__ active, int col_div, const int64_t* __restrict__ d_K,
                             int64_t cap)
{
    kernel_prologue();
    const int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (c >= Cc || overflow(d_K, cap)) return;  // uniform over the warp
    col_total_warp(R, Cc, c, SS, total, active, col_div, lane);
}

// Exclusive scan of x[0..len) -> start by one block of 1024 threads; the sum ->
// *sum (nullable). count_ranges (nullable): also ranges[i] = [start, start +
// x[i]) for x[i] > 0, else (0, 0). Every thread of the block must call it.
__device__ void block_scan_1024(int len, const uint32_t* __restrict__ x, uint32_t* __restrict__ start,
                                int64_t* __restrict__ sum, uint2* __restrict__ count_ranges)
{
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;
    for (int base = 0; base < len; base += 1024) {
        const int i = base + threadIdx.x;
        const unsigned long long v = i < len ? x[i] : 0ull;
        unsigned long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long w = s_w[lane];
            unsigned long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            s_w[lane] = wi - w;
        }
        __syncthreads();
        const unsigned long long excl = carry + s_w[warp] + inc - v;
        if (i < len) {
            start[i] = (uint32_t)excl;
            if (count_ranges)
                count_ranges[i] = v > 0 ? make_uint2((uint32_t)excl, (uint32_t)(excl + v)) : make_uint2(0u, 0u);
        }
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
        carry = s_carry;
        __syncthreads();
    }
    if (threadIdx.x == 0 && sum) *sum = (int64_t)carry;
}

// Level-1 row bookkeeping in one block of 1024 threads, after the column
// segment sums of M1: per tile row the exclusive scan of its segment sums (in
// place) and its row-list length, the rows' starts (exclusive scan) and the
// row-list total *R, then the level-2 segments per row (ceil(rowlen /
// kSegLen)), their offsets (exclusive scan) and total *NS.
__global__ void __launch_bounds__(1024)
k_lvl1_rows(int C1, int TY, uint32_t* __restrict__ SS1, uint32_t* __restrict__ rowlen,
            uint32_t* __restrict__ rowstart, int64_t* __restrict__ R, uint32_t* __restrict__ nseg,
            uint32_t* __restrict__ segoff, int64_t* __restrict__ NS, const int64_t* __restrict__ d_K, int64_t cap)
{
    kernel_prologue();
    if (overflow(d_K, cap)) return;  // uniform over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < TY; c += 32) col_total_warp(C1, TY, c, SS1, rowlen, nullptr, 1, lane);
    __syncthreads();
    block_scan_1024(TY, rowlen, rowstart, R, nullptr);
    for (int ty = threadIdx.x; ty < TY; ty += 1024) nseg[ty] = (rowlen[ty] + kSegLen - 1) / kSegLen;
    __syncthreads();
    block_scan_1024(TY, nseg, segoff, NS, nullptr);
}

// Level-2 tile starts in one block of 1024 threads: the exclusive scan of the
// tile counts, and the ranges ((0, 0) for empty tiles). On overflow every range
// is set empty instead. K_max (nullable): a high-water mark of K across calls,
// raised here.
__global__ void __launch_bounds__(1024)
k_tile_starts(int T, const uint32_t* __restrict__ count, uint32_t* __restrict__ start,
              const int64_t* __restrict__ d_K, int64_t cap, uint2* __restrict__ ranges, int64_t* __restrict__ K_max)
{
    kernel_prologue();
    if (K_max && threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long*>(K_max), (unsigned long long)*d_K);
    if (overflow(d_K, cap)) {
        for (int t = threadIdx.x; t < T; t += 1024) ranges[t] = make_uint2(0u, 0u);
        return;
    }
    block_scan_1024(T, count, start, nullptr, ranges);
}

// M[r][c] <- start[c] + (sum of M[r'][c] for r' < r): the first slot of row r
// in bin c. Same warp layout as k_col_segsum.
__global__ void __launch_bounds__(kLvlThreads)
k_col_base(int R, int Cc, uint32_t* __restrict__ M, const uint32_t* __restrict__ SS,
           const uint32_t* __restrict__ start, const uint32_t* __restrict__ active,
           const uint32_t* __restrict__ rowbase, int col_div, const int64_t* __restrict__ d_K, int64_t cap)
{
    kernel_prologue();
    const int c = blockIdx.x * kColsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= Cc || overflow(d_K, cap)) return;  // uniform over the warp
    const int act = active_rows(active, col_div, c, R);
    for (int by = blockIdx.y; by * kScanRows < act; by += gridDim.y) {
        const int r = by * kScanRows + lane;
        const bool in = r < act;
        const int64_t at = mat_at(rowbase, col_div, Cc, c, r);
        const uint32_t h = in ? M[at] : 0u;
        uint32_t inc = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (in) M[at] = start[c] + SS[(int64_t)by * Cc + c] + inc - h;
    }
}

// A row-list entry: the Gaussian id and its rect's x-extent (x0 in the low
// 16 bits, the tile count in the high 16), so that level 2 needs no rect.
__device__ __forceinline__ uint32_t pack_x(int4 r) { return (uint32_t)r.x | ((uint32_t)(r.z - r.x + 1) << 16); }

// Level 1c: each level-1 warp writes its Gaussians into the row lists, in
// depth order, at the slots M1 (now bases) gives it. The ids and rects of the
// next round are fetched while the current round is written.
__global__ void __launch_bounds__(kLvlThreads)
k_row_scatter(int n, const int64_t* __restrict__ d_nvis, int C1, const uint32_t* __restrict__ perm,
              const uint32_t* __restrict__ skeys, const int4* __restrict__ rects, int TX, int TY,
              const uint32_t* __restrict__ M1, const int64_t* __restrict__ d_K, int64_t cap,
              uint2* __restrict__ rowlist)
{
    kernel_prologue();
    extern __shared__ int s_lvl[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kLvlWarps + warp;
    if (c >= C1 || overflow(d_K, cap)) return;
    uint32_t* cnt = reinterpret_cast<uint32_t*>(s_lvl) + warp * (TY + 1 + 64);
    uint32_t* scratch = cnt + TY + 1;
    for (int ty = lane; ty < TY; ty += 32) cnt[ty] = M1[(int64_t)c * TY + ty];
    __syncwarp();
    const int k0 = c * kRowChunk, k1 = min(k0 + kRowChunk, (int)min((int64_t)n, *d_nvis));
    bool vis_n;
    uint32_t g_n = lvl1_id(perm, skeys, k0 + lane, k1, vis_n);
    int4 r_n = vis_n ? rects[g_n] : make_int4(0, 0, -1, -1);
    for (int kb = k0; kb < k1; kb += 32) {
        const uint32_t g = g_n;
        const bool vis = vis_n;
        const int4 r = r_n;
        if (kb + 32 < k1) {
            g_n = lvl1_id(perm, skeys, kb + 32 + lane, k1, vis_n);
            r_n = vis_n ? rects[g_n] : make_int4(0, 0, -1, -1);
        }
        int y0 = 0, nr = 0;
        if (vis && rect_in_grid(r, TX, TY)) {
            y0 = r.y;
            nr = r.w - r.y + 1;
        }
        scatter_round<uint2>(make_uint2(g, pack_x(r)), y0, nr, cnt, scratch, rowlist, cap, lane);
    }
}

// Segment index -> (row, segment within the row): the largest row whose first
// segment is <= seg (rows without segments share the next row's offset).
__device__ __forceinline__ int segment_row(const uint32_t* segoff, int TY, uint32_t seg)
{
    int lo = 0, hi = TY - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segoff[mid] <= seg) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Level 2a: per level-2 segment (one CTA), the number of its Gaussians
// spanning each tile of the row -> M2[segment][tile of the row].
__global__ void __launch_bounds__(kLvlThreads)
k_seg_hist(int TX, int TY, const uint32_t* __restrict__ rowstart, const uint32_t* __restrict__ rowlen,
           const uint32_t* __restrict__ segoff, const int64_t* __restrict__ d_NS, const uint2* __restrict__ rowlist,
           const int64_t* __restrict__ d_K, int64_t cap, uint32_t* __restrict__ M2)
{
    kernel_prologue();
    extern __shared__ int s_lvl[];
    if (overflow(d_K, cap)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* d = s_lvl;
    const int64_t NS = *d_NS;
    for (int64_t seg = blockIdx.x; seg < NS; seg += gridDim.x) {
        const int ty = segment_row(segoff, TY, (uint32_t)seg);
        const uint32_t s = (uint32_t)seg - segoff[ty];
        const uint32_t e0 = rowstart[ty] + s * kSegLen;
        const uint32_t e1 = min(e0 + kSegLen, rowstart[ty] + rowlen[ty]);
        for (int i = threadIdx.x; i <= TX; i += kLvlThreads) d[i] = 0;
        __syncthreads();
        for (uint32_t e = e0 + threadIdx.x; e < e1; e += kLvlThreads) {
            const uint32_t xp = rowlist[e].y;
            atomicAdd(&d[xp & 0xffffu], 1);
            atomicAdd(&d[(xp & 0xffffu) + (xp >> 16)], -1);
        }
        __syncthreads();
        if (warp == 0) {
            warp_inclusive_scan_smem(d, TX, lane);
            uint32_t* out = M2 + seg * TX;
            for (int tx = lane; tx < TX; tx += 32) out[tx] = (uint32_t)d[tx];
        }
        __syncthreads();
    }
}

// Level 2c: per level-2 segment (one CTA) the 8 warps take consecutive
// sub-ranges of the segment. Each warp counts its sub-range per tile, a
// cross-warp exclusive prefix per tile (starting from the segment's first slot
// in M2) gives every warp its own counters, and the warps write the ids of
// their sub-range into the row's tile lists, in order.
// (6 CTAs per SM: 2048-entry segments and the higher occupancy took the 4K binning from 0.325 to
// 0.321 ms)
__global__ void __launch_bounds__(kLvlThreads, 6)
k_seg_scatter(int TX, int TY, const uint32_t* __restrict__ rowstart, const uint32_t* __restrict__ rowlen,
              const uint32_t* __restrict__ segoff, const int64_t* __restrict__ d_NS,
              const uint2* __restrict__ rowlist, const uint32_t* __restrict__ M2,
              const int64_t* __restrict__ d_K, int64_t cap, uint32_t* __restrict__ out)
{
    kernel_prologue();
    extern __shared__ int s_lvl[];
    if (overflow(d_K, cap)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W1 = TX + 1;
    const int WS = W1 + 64;  // per warp: counters, then the scatter scratch
    int* d = s_lvl + warp * WS;
    uint32_t* cnt = reinterpret_cast<uint32_t*>(d);
    uint32_t* scratch = cnt + W1;
    const int64_t NS = *d_NS;
    constexpr uint32_t kSub = kSegLen / kLvlWarps;
    for (int64_t seg = blockIdx.x; seg < NS; seg += gridDim.x) {
        const int ty = segment_row(segoff, TY, (uint32_t)seg);
        const uint32_t s = (uint32_t)seg - segoff[ty];
        const uint32_t e0 = rowstart[ty] + s * kSegLen;
        const uint32_t e1 = min(e0 + kSegLen, rowstart[ty] + rowlen[ty]);
        const uint32_t w0 = min(e0 + (uint32_t)warp * kSub, e1);
        const uint32_t w1 = min(w0 + kSub, e1);
        // counts of this warp's sub-range
        for (int i = lane; i < W1; i += 32) d[i] = 0;
        __syncwarp();
#pragma unroll 4
        for (uint32_t e = w0 + lane; e < w1; e += 32) {
            const uint32_t xp = rowlist[e].y;
            atomicAdd(&d[xp & 0xffffu], 1);
            atomicAdd(&d[(xp & 0xffffu) + (xp >> 16)], -1);
        }
        __syncwarp();
        warp_inclusive_scan_smem(d, TX, lane);
        __syncthreads();
        // counters: the segment's first slot plus the counts of the earlier warps
        const uint32_t* base = M2 + seg * TX;
        for (int tx = threadIdx.x; tx < TX; tx += kLvlThreads) {
            uint32_t run = base[tx];
            for (int w = 0; w < kLvlWarps; ++w) {
                uint32_t* c = reinterpret_cast<uint32_t*>(s_lvl + w * WS) + tx;
                const uint32_t x = *c;
                *c = run;
                run += x;
            }
        }
        __syncthreads();
        uint2 ent_n = w0 + lane < w1 ? rowlist[w0 + lane] : make_uint2(0u, 0u);
        for (uint32_t eb = w0; eb < w1; eb += 32) {
            // this round's entries; the next round's are fetched while these are written
            const uint2 ent = ent_n;
            if (eb + 32 < w1) ent_n = eb + 32 + lane < w1 ? rowlist[eb + 32 + lane] : make_uint2(0u, 0u);
            scatter_round<uint32_t>(ent.x, (int)(ent.y & 0xffffu), (int)(ent.y >> 16), cnt, scratch, out, cap, lane);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Workspace layout (each region 256-byte aligned)
// ---------------------------------------------------------------------------
struct Ws {
    uint32_t *dkeys0, *dkeys1, *perm0, *perm1;
    uint32_t *hist, *totals;
    uint32_t *M1, *SS1, *rowlen, *rowstart;
    uint2* rowlist;
    uint32_t *nseg, *segoff;
    int64_t *R, *NS, *nvis;
    uint32_t *M2, *SS2, *tcount, *tstart;
    size_t bytes;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int lvl1_warps(int n) { return (n + kRowChunk - 1) / kRowChunk; }
int lvl2_rows(int n) { return (n + kSegLen - 1) / kSegLen; }  // segments per row, at most
// segments over all rows, at most: sum over rows of ceil(rowlen / kSegLen) for row lists of rows_cap entries
int64_t lvl2_segments(int64_t rows_cap, int TY) { return rows_cap / kSegLen + TY; }
constexpr int kScanGridY = 64;  // row-block parallelism of the column scans (they loop beyond it)

Ws carve(void* base, int n, int64_t cap, int tiles_x, int tiles_y)
{
    Ws w{};
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = static_cast<char*>(base) + off;
        off += align256(bytes);
        return p;
    };
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t T = (size_t)tiles_x * tiles_y;
    const size_t TY = (size_t)tiles_y;
    const int C1 = lvl1_warps(n > 0 ? n : 1);
    const int NSR = lvl2_rows(n > 0 ? n : 1);
    // every row entry yields at least one pair, so the row lists fit in min(K, n*TY) <= cap slots
    const size_t rows_cap = (size_t)std::min<int64_t>(cap > 0 ? cap : 1, (int64_t)nn * (int64_t)TY);
    w.dkeys0 = (uint32_t*)take(nn * 4);
    w.dkeys1 = (uint32_t*)take(nn * 4);
    w.perm0 = (uint32_t*)take(nn * 4);
    w.perm1 = (uint32_t*)take(nn * 4);
    w.hist = (uint32_t*)take((size_t)kRadixBins * sort_blocks(n) * 4);
    w.totals = (uint32_t*)take(kRadixBins * 4);
    w.M1 = (uint32_t*)take((size_t)C1 * TY * 4);
    w.SS1 = (uint32_t*)take((size_t)((C1 + kScanRows - 1) / kScanRows) * TY * 4);
    w.rowlen = (uint32_t*)take(TY * 4);
    w.rowstart = (uint32_t*)take(TY * 4);
    w.rowlist = (uint2*)take(rows_cap * 8);
    w.nseg = (uint32_t*)take(TY * 4);
    w.segoff = (uint32_t*)take(TY * 4);
    w.R = (int64_t*)take(8);
    w.NS = (int64_t*)take(8);
    w.nvis = (int64_t*)take(8);
    w.M2 = (uint32_t*)take((size_t)lvl2_segments((int64_t)rows_cap, (int)TY) * (size_t)tiles_x * 4);
    w.SS2 = (uint32_t*)take((size_t)((NSR + kScanRows - 1) / kScanRows) * T * 4);
    w.tcount = (uint32_t*)take(T * 4);
    w.tstart = (uint32_t*)take(T * 4);
    w.bytes = off;
    return w;
}

}  // namespace
}  // namespace gs

extern "C" {

size_t gs_bin_sort_workspace_size(int32_t n, int64_t capacity, int32_t tiles_x, int32_t tiles_y)
{
    if (n < 0 || capacity < 0 || tiles_x <= 0 || tiles_y <= 0) return 0;
    // every term grows with tiles_x and tiles_y: the size covers all smaller grids
    return gs::carve(nullptr, n, capacity, tiles_x, tiles_y).bytes + 256;
}

int32_t gs_bin_sort(int32_t n, const int32_t* rects, const int32_t* tiles_touched, const float* splats,
                    const uint32_t* depth_keys, int32_t tiles_x, int32_t tiles_y, void* workspace,
                    size_t workspace_bytes, int64_t capacity, uint32_t* sorted_ids, uint32_t* ranges,
                    int64_t* num_pairs, int64_t* num_pairs_max, gs_stream_t stream)
{
    using namespace gs;
    if (n < 0 || capacity < 0 || capacity > 0x7fffffffLL || tiles_x <= 0 || tiles_y <= 0 ||
        tiles_x > kMaxGridSide || tiles_y > kMaxGridSide) {
        gs_host::set_error("gs_bin_sort: bad sizes (n >= 0, 0 <= capacity < 2^31, 0 < tiles_x, tiles_y <= 4096)");
        return GS_ERR_ARG;
    }
    if (!ranges || !num_pairs || (n > 0 && (!rects || !tiles_touched || (!splats && !depth_keys) || !workspace)) ||
        (capacity > 0 && !sorted_ids)) {
        gs_host::set_error("gs_bin_sort: null pointer");
        return GS_ERR_ARG;
    }
    uintptr_t base = reinterpret_cast<uintptr_t>(workspace);
    void* ws_al = reinterpret_cast<void*>((base + 255) & ~uintptr_t(255));
    size_t slack = reinterpret_cast<uintptr_t>(ws_al) - base;
    Ws w = carve(ws_al, n, capacity, tiles_x, tiles_y);
    if (n > 0 && workspace_bytes < w.bytes + slack) {
        gs_host::set_error("gs_bin_sort: workspace too small");
        return GS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int T = tiles_x * tiles_y, TX = tiles_x, TY = tiles_y;
    cudaMemsetAsync(num_pairs, 0, sizeof(int64_t), st);
    if (n == 0) {
        cudaMemsetAsync(ranges, 0, (size_t)T * 2 * sizeof(uint32_t), st);
        return gs_host::check_launch("gs_bin_sort");
    }
    const int4* rc = reinterpret_cast<const int4*>(rects);
    // the depth order of the Gaussians: a stable LSD radix sort of (depth bits, id), from the
    // projection's keys or from a pass over the splat records
    const uint32_t* keys_in = depth_keys;
    if (!keys_in) {
        gs::launch(k_depth_keys, (n + kKeyThreads * kKeysPerThread - 1) / (kKeyThreads * kKeysPerThread), kKeyThreads,
                   0, st, n, reinterpret_cast<const float4*>(splats), tiles_touched, w.dkeys0);
        keys_in = w.dkeys0;
    }
    // (4 passes: the sorted keys and the order in dkeys0, perm0). The culled Gaussians are dropped
    // by the first pass; the others, *w.nvis of them, are sorted.
    radix_sort(SortBufs{const_cast<uint32_t*>(keys_in), w.perm0, w.dkeys1, w.perm1, true, w.dkeys0}, nullptr, n,
               32, sort_blocks(n), w.hist, w.totals, w.nvis, st);
    // level 1: rows
    const int C1 = lvl1_warps(n);
    const int lvl1_blocks = (C1 + kLvlWarps - 1) / kLvlWarps;
    const size_t smem1 = (size_t)kLvlWarps * (TY + 1 + 64) * sizeof(int);
    if (smem1 > 48 * 1024) {
        cudaFuncSetAttribute(k_row_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
        cudaFuncSetAttribute(k_row_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
    }
    gs::launch(k_row_hist, lvl1_blocks, kLvlThreads, smem1, st, n, w.nvis, C1, w.perm0, w.dkeys0, rc, TX, TY,
               num_pairs, w.M1);
    const int nsb1 = (C1 + kScanRows - 1) / kScanRows;
    const dim3 g1((TY + kColsPerBlock - 1) / kColsPerBlock, std::min(nsb1, kScanGridY));
    gs::launch(k_col_segsum, g1, kLvlThreads, 0, st, C1, TY, w.M1, w.SS1, nullptr, nullptr, 1, num_pairs, capacity);
    gs::launch(k_lvl1_rows, 1, 1024, 0, st, C1, TY, w.SS1, w.rowlen, w.rowstart, w.R, w.nseg, w.segoff, w.NS,
               num_pairs, capacity);
    gs::launch(k_col_base, g1, kLvlThreads, 0, st, C1, TY, w.M1, w.SS1, w.rowstart, nullptr, nullptr, 1, num_pairs,
               capacity);
    gs::launch(k_row_scatter, lvl1_blocks, kLvlThreads, smem1, st, n, w.nvis, C1, w.perm0, w.dkeys0, rc, TX, TY,
               w.M1, num_pairs, capacity, w.rowlist);
    // level 2: tiles within each row
    const int NSR = lvl2_rows(n);
    const size_t smem2 = (size_t)kLvlWarps * (TX + 1 + 64) * sizeof(int);
    const size_t smem2h = (size_t)(TX + 1) * sizeof(int);
    if (smem2 > 48 * 1024) {
        cudaFuncSetAttribute(k_seg_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2h);
        cudaFuncSetAttribute(k_seg_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    }
    const int lvl2_blocks = gs_host::sm_count() * 8;
    gs::launch(k_seg_hist, lvl2_blocks, kLvlThreads, smem2h, st, TX, TY, w.rowstart, w.rowlen, w.segoff, w.NS,
               w.rowlist, num_pairs, capacity, w.M2);
    const int nsb2 = (NSR + kScanRows - 1) / kScanRows;
    const dim3 g2((T + kColsPerBlock - 1) / kColsPerBlock, std::min(nsb2, kScanGridY));
    gs::launch(k_col_segsum, g2, kLvlThreads, 0, st, NSR, T, w.M2, w.SS2, w.nseg, w.segoff, TX, num_pairs, capacity);
    gs::launch(k_col_totals, (int)(((int64_t)T * 32 + 255) / 256), 256, 0, st, NSR, T, w.SS2, w.tcount, w.nseg, TX,
               num_pairs, capacity);
    gs::launch(k_tile_starts, 1, 1024, 0, st, T, w.tcount, w.tstart, num_pairs, capacity,
               reinterpret_cast<uint2*>(ranges), num_pairs_max);
    gs::launch(k_col_base, g2, kLvlThreads, 0, st, NSR, T, w.M2, w.SS2, w.tstart, w.nseg, w.segoff, TX, num_pairs,
               capacity);
    if (capacity > 0)
        gs::launch(k_seg_scatter, lvl2_blocks, kLvlThreads, smem2, st, TX, TY, w.rowstart, w.rowlen, w.segoff, w.NS,
                   w.rowlist, w.M2, num_pairs, capacity, sorted_ids);
    return gs_host::check_launch("gs_bin_sort");
}

int32_t gs_bin_sort_static(int32_t n, const int32_t* rects, const int32_t* tiles_touched, const float* splats,
                           const uint32_t* depth_keys, int32_t tiles_x, int32_t tiles_y, int64_t capacity,
                           uint32_t* sorted_ids, uint32_t* ranges, int64_t* num_pairs, int64_t* num_pairs_max,
                           gs_stream_t stream)
{
    if (n < 0 || capacity < 0 || tiles_x <= 0 || tiles_y <= 0) {
        gs_host::set_error("gs_bin_sort_static: bad sizes (n >= 0, capacity >= 0, tiles > 0)");
        return GS_ERR_ARG;
    }
    const size_t need = gs_bin_sort_workspace_size(n, capacity, tiles_x, tiles_y);
    if (need > (size_t)GS_BIN_SORT_STATIC_SCRATCH_BYTES) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "gs_bin_sort_static: n=%d, capacity=%lld need %zu bytes of scratch; the static array holds "
                      "%u (use gs_bin_sort with a caller workspace)",
                      n, (long long)capacity, need, (unsigned)GS_BIN_SORT_STATIC_SCRATCH_BYTES);
        gs_host::set_error(msg);
        return GS_ERR_ARG;
    }
    // The array's device address in the calling thread's current context, looked up on every
    // call: an address kept from an earlier call could belong to another context (a plugin's own
    // context, or one destroyed by cudaDeviceReset). Once the module is loaded this is a
    // host-side table lookup that allocates nothing.
    void* scratch = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&scratch, g_bin_sort_scratch);
    if (e != cudaSuccess || scratch == nullptr) {
        char msg[256];
        std::snprintf(msg, sizeof(msg), "gs_bin_sort_static: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
        gs_host::set_error(msg);
        return GS_ERR_CUDA;
    }
    return gs_bin_sort(n, rects, tiles_touched, splats, depth_keys, tiles_x, tiles_y, scratch,
                       (size_t)GS_BIN_SORT_STATIC_SCRATCH_BYTES, capacity, sorted_ids, ranges, num_pairs,
                       num_pairs_max, stream);
}

}  // extern "C"
