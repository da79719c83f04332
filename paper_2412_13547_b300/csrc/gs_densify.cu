// gs_densify.cu -- densification and pruning under a Gaussian budget
// (Sec. 3.2, Sec. 3.3): the position-appearance candidate rule with a budget
// cut by an exact radix select of the score, the baseline clone/split, and
// order-preserving compaction for the prune. Runs once per densification
// interval; every pass is a plain streaming kernel over the Gaussians.
#include <cmath>

#include "gs_common.cuh"

namespace gs {
namespace {

constexpr int kBlk = 1024;          // elements per scan block (one per thread)
constexpr int kWarpsBlk = kBlk / 32;
constexpr int kHistBins = 1 << 16;  // radix-select digit: 16 bits

// Device scalars of the selection, in the workspace.
struct SelState {
    int candidates;   // Gaussians passing the thresholds
    int all;          // 1: every candidate fits the budget
    unsigned thr;     // the budget's score key T (select key > T, and the first need_eq with key == T)
    int need_eq;
    int hi_above;     // candidates with hi digit above the chosen bin
    unsigned hi_bin;
    int total;        // selected count
};

struct DsWs {
    unsigned* keys;
    int* rank;
    int* blk;
    int* blk_base;
    unsigned* hist;
    SelState* st;
    size_t bytes;
};

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

DsWs carve(void* base, int n)
{
    DsWs w{};
    const int nb = (n + kBlk - 1) / kBlk;
    char* p = static_cast<char*>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* q = p ? p + off : nullptr;
        off += align_up(bytes);
        return q;
    };
    w.keys = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * (size_t)n));
    w.rank = reinterpret_cast<int*>(take(sizeof(int) * (size_t)n));
    w.blk = reinterpret_cast<int*>(take(sizeof(int) * (size_t)nb));
    w.blk_base = reinterpret_cast<int*>(take(sizeof(int) * (size_t)nb));
    w.hist = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * kHistBins));
    w.st = reinterpret_cast<SelState*>(take(sizeof(SelState)));
    w.bytes = off + 256;
    return w;
}

// --------------------------------------------------------------------------
// Block-level counting and ranking of a predicate (one element per thread)
// --------------------------------------------------------------------------

// Exclusive rank of this thread's flag within its block; *block_total gets
// the block's count (all threads).
__device__ __forceinline__ int block_rank(bool flag, int* s_warp, int* block_total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ball = __ballot_sync(0xffffffffu, flag);
    const int in_warp = __popc(ball & ((1u << lane) - 1u));
    if (lane == 0) s_warp[warp] = __popc(ball);
    __syncthreads();
    if (warp == 0) {
        const int c = lane < kWarpsBlk ? s_warp[lane] : 0;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < kWarpsBlk) s_warp[lane] = x - c;  // exclusive warp bases
        if (lane == 31) s_warp[32] = x;
    }
    __syncthreads();
    const int r = s_warp[warp] + in_warp;
    *block_total = s_warp[32];
    __syncthreads();
    return r;
}

// Exclusive scan of the per-block counts (one block), total to *total.
__global__ void __launch_bounds__(kBlk) k_scan_blocks(int nb, const int* __restrict__ cnt, int* __restrict__ base,
                                                      int* __restrict__ total)
{
    kernel_prologue();
    __shared__ int s_warp[33];
    int run = 0;
    for (int b0 = 0; b0 < nb; b0 += kBlk) {
        const int b = b0 + (int)threadIdx.x;
        const int c = b < nb ? cnt[b] : 0;
        int tot;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int w = lane < kWarpsBlk ? s_warp[lane] : 0;
            int z = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            if (lane < kWarpsBlk) s_warp[lane] = z - w;
            if (lane == 31) s_warp[32] = z;
        }
        __syncthreads();
        if (b < nb) base[b] = run + s_warp[warp] + x - c;
        tot = s_warp[32];
        __syncthreads();
        run += tot;
    }
    if (threadIdx.x == 0 && total) *total = run;
}

// --------------------------------------------------------------------------
// Selection (Sec. 3.3)
// --------------------------------------------------------------------------

// Candidate flag and ranking key of Gaussian i (FP32, IEEE division).
__device__ __forceinline__ unsigned score_key(int i, const float* pos, const float* col, const int* cnt, float tau_pos,
                                              float tau_color, int branch)
{
    const int c = cnt[i];
    if (c <= 0) return 0u;
    const float fc = (float)c;
    const float sp = __fdiv_rn(pos[i], fc), sc = __fdiv_rn(col[i], fc);
    const bool cand = sp > tau_pos || (branch && sc > tau_color);
    if (!cand) return 0u;
    const float a = __fdiv_rn(sp, tau_pos);
    const float b = branch ? __fdiv_rn(sc, tau_color) : 0.0f;
    const float s = fmaxf(a, b);
    // candidates score above 0; keep the key of a candidate nonzero
    return max(__float_as_uint(s), 1u);
}

__global__ void __launch_bounds__(kBlk) k_ds_keys(int n, const float* __restrict__ pos, const float* __restrict__ col,
                                                  const int* __restrict__ cnt, float tau_pos, float tau_color,
                                                  int branch, unsigned* __restrict__ keys, unsigned* __restrict__ hist,
                                                  SelState* __restrict__ st)
{
    kernel_prologue();
    __shared__ int s_warp[33];
    const int i = blockIdx.x * kBlk + threadIdx.x;
    unsigned k = 0u;
    if (i < n) {
        k = score_key(i, pos, col, cnt, tau_pos, tau_color, branch);
        keys[i] = k;
        if (k) atomicAdd(&hist[k >> 16], 1u);
    }
    int tot;
    block_rank(k != 0u, s_warp, &tot);
    if (threadIdx.x == 0 && tot) atomicAdd(&st->candidates, tot);
}

// Finds the digit bin holding the budget's cut, scanning bins from the top.
// phase 0: hi digit over all candidates; phase 1: lo digit inside hi_bin.
__global__ void __launch_bounds__(kBlk) k_ds_find(int max_new, int phase, const unsigned* __restrict__ hist,
                                                  SelState* __restrict__ st)
{
    kernel_prologue();
    __shared__ unsigned s_part[kBlk];
    constexpr int PER = kHistBins / kBlk;  // 64 bins per thread, thread 0 holds the top bins
    if (phase == 0 && st->candidates <= max_new) {
        if (threadIdx.x == 0) {
            st->all = 1;
            st->thr = 0u;
            st->need_eq = 0;
        }
        return;
    }
    if (phase == 1 && st->all) return;
    const int want = phase == 0 ? max_new : max_new - st->hi_above;
    // thread t owns bins [hi - (t+1) PER, hi - t PER) counted from the top
    unsigned s = 0;
    for (int k = 0; k < PER; ++k) s += hist[kHistBins - 1 - (threadIdx.x * PER + k)];
    s_part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned above = 0;
        int t = 0;
        for (; t < kBlk; ++t) {
            if (above + s_part[t] >= (unsigned)want) break;
            above += s_part[t];
        }
        int bin = kHistBins - 1 - t * PER;
        for (int k = 0; k < PER; ++k, --bin) {
            const unsigned h = hist[bin];
            if (above + h >= (unsigned)want) break;
            above += h;
        }
        if (phase == 0) {
            st->all = 0;
            st->hi_bin = (unsigned)bin;
            st->hi_above = (int)above;
        } else {
            st->thr = (st->hi_bin << 16) | (unsigned)bin;
            st->need_eq = want - (int)above;
        }
    }
}

__global__ void __launch_bounds__(kBlk) k_ds_hist_lo(int n, const unsigned* __restrict__ keys,
                                                     unsigned* __restrict__ hist, const SelState* __restrict__ st)
{
    kernel_prologue();
    if (st->all) return;
    const int i = blockIdx.x * kBlk + threadIdx.x;
    if (i >= n) return;
    const unsigned k = keys[i];
    if (k && (k >> 16) == st->hi_bin) atomicAdd(&hist[k & 0xffffu], 1u);
}

// Per-block counts of the keys equal to the cut.
__global__ void __launch_bounds__(kBlk) k_ds_count_eq(int n, const unsigned* __restrict__ keys,
                                                      const SelState* __restrict__ st, int* __restrict__ blk)
{
    kernel_prologue();
    __shared__ int s_warp[33];
    const int i = blockIdx.x * kBlk + threadIdx.x;
    const bool eq = !st->all && i < n && keys[i] == st->thr;
    int tot;
    block_rank(eq, s_warp, &tot);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

__device__ __forceinline__ bool selected_flag(int i, int n, const unsigned* keys, const int* rank_eq,
                                              const SelState* st)
{
    if (i >= n) return false;
    const unsigned k = keys[i];
    if (st->all) return k != 0u;
    return k > st->thr || (k == st->thr && rank_eq[i] < st->need_eq);
}

// Global rank of each key equal to the cut (index order), then per-block
// counts of the selected Gaussians.
__global__ void __launch_bounds__(kBlk) k_ds_rank_eq(int n, const unsigned* __restrict__ keys,
                                                     const SelState* __restrict__ st, const int* __restrict__ base_eq,
                                                     int* __restrict__ rank_eq, int* __restrict__ blk)
{
    kernel_prologue();
    __shared__ int s_warp[33];
    const int i = blockIdx.x * kBlk + threadIdx.x;
    const bool eq = !st->all && i < n && keys[i] == st->thr;
    int tot;
    const int r = block_rank(eq, s_warp, &tot);
    if (i < n) rank_eq[i] = eq ? base_eq[blockIdx.x] + r : 0x7fffffff;
    __syncthreads();
    const bool sel = selected_flag(i, n, keys, rank_eq, st);
    block_rank(sel, s_warp, &tot);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kBlk) k_ds_write(int n, const unsigned* __restrict__ keys,
                                                   const int* __restrict__ rank_eq, const SelState* __restrict__ st,
                                                   const int* __restrict__ base, int* __restrict__ out)
{
    kernel_prologue();
    __shared__ int s_warp[33];
    const int i = blockIdx.x * kBlk + threadIdx.x;
    const bool sel = selected_flag(i, n, keys, rank_eq, st);
    int tot;
    const int r = block_rank(sel, s_warp, &tot);
    if (sel) out[base[blockIdx.x] + r] = i;
}

// --------------------------------------------------------------------------
// Prune
// --------------------------------------------------------------------------

__device__ __forceinline__ bool keep_flag(int i, int n, const float* logits, float logit_min, const float* ls,
                                          float ls_max)
{
    if (i >= n) return false;
    bool k = logits[i] >= logit_min;
    if (ls) k = k && fmaxf(fmaxf(ls[3 * i], ls[3 * i + 1]), ls[3 * i + 2]) <= ls_max;
    return k;
}

__global__ void __launch_bounds__(kBlk) k_keep_count(int n, const float* __restrict__ logits, float logit_min,
                                                     const float* __restrict__ ls, float ls_max,
                                                     int* __restrict__ blk)
{
    kernel_prologue();
    __shared__ int s_warp[33];
    const int i = blockIdx.x * kBlk + threadIdx.x;
    int tot;
    block_rank(keep_flag(i, n, logits, logit_min, ls, ls_max), s_warp, &tot);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kBlk) k_keep_write(int n, const float* __restrict__ logits, float logit_min,
                                                     const float* __restrict__ ls, float ls_max,
                                                     const int* __restrict__ base, int* __restrict__ out)
{
    kernel_prologue();
    __shared__ int s_warp[33];
    const int i = blockIdx.x * kBlk + threadIdx.x;
    const bool k = keep_flag(i, n, logits, logit_min, ls, ls_max);
    int tot;
    const int r = block_rank(k, s_warp, &tot);
    if (k) out[base[blockIdx.x] + r] = i;
}

// --------------------------------------------------------------------------
// Row movement: gather, grow, split
// --------------------------------------------------------------------------

// dst row i <- src row map(i) in 4-byte words; map(i) = index[i] (gather) or,
// for growth, i below n_old and selected[i - n_old] above. zero_new: rows at
// or above n_old are written as zero instead; zero_all: every row is zero.
__global__ void k_rows(int n_out, int n_old, const int* __restrict__ index, const int* __restrict__ selected,
                       const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int words, int zero_new,
                       int zero_all)
{
    kernel_prologue();
    const int64_t total = (int64_t)n_out * words;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(w / words), col = (int)(w % words);
        uint32_t v = 0u;
        if (!zero_all) {
            int from;
            if (index) {
                from = index[row];
            } else if (row < n_old) {
                from = row;
            } else {
                from = zero_new ? -1 : selected[row - n_old];
            }
            if (from >= 0) v = src[(int64_t)from * words + col];
        }
        dst[w] = v;
    }
}

struct SplitArgs {
    const float* mean_src;
    float* mean_dst;
    const float* ls_src;
    float* ls_dst;
    const float4* quat_src;
    float* state[GS_MAX_ROW_TENSORS];
    int state_words[GS_MAX_ROW_TENSORS];
    int nstate;
};

// Split of the selected Gaussians whose largest log-scale exceeds the
// threshold: children at mean + R(q) diag(exp(log_scale)) z_k, log-scales
// reduced by log(1.6); child 0 in the parent's row, child 1 in the appended
// row. The parent's optimizer state restarts from zero.
__global__ void k_split(int n_old, int m, const int* __restrict__ selected, const float* __restrict__ noise,
                        float log_split, SplitArgs a)
{
    kernel_prologue();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int g = selected[j];
    const float l0 = a.ls_src[3 * g], l1 = a.ls_src[3 * g + 1], l2 = a.ls_src[3 * g + 2];
    if (!(fmaxf(fmaxf(l0, l1), l2) > log_split)) return;
    const float4 q = a.quat_src[g];
    const float qi = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float Rm[9];
    quat_rot(q.x * qi, q.y * qi, q.z * qi, q.w * qi, Rm);
    const float s[3] = {expf(l0), expf(l1), expf(l2)};
    const float dl = logf(1.6f);
    for (int k = 0; k < 2; ++k) {
        const int row = k == 0 ? g : n_old + j;
        const float* z = noise + 6 * (int64_t)j + 3 * k;
        const float v0 = s[0] * z[0], v1 = s[1] * z[1], v2 = s[2] * z[2];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            a.mean_dst[3 * (int64_t)row + r] =
                a.mean_src[3 * (int64_t)g + r] + (Rm[3 * r] * v0 + Rm[3 * r + 1] * v1 + Rm[3 * r + 2] * v2);
        a.ls_dst[3 * (int64_t)row] = l0 - dl;
        a.ls_dst[3 * (int64_t)row + 1] = l1 - dl;
        a.ls_dst[3 * (int64_t)row + 2] = l2 - dl;
    }
    for (int t = 0; t < a.nstate; ++t)
        for (int w = 0; w < a.state_words[t]; ++w) a.state[t][(int64_t)g * a.state_words[t] + w] = 0.0f;
}

bool check_rows(const GsRowTensor* t, int count, bool need_src)
{
    if (count < 1 || count > GS_MAX_ROW_TENSORS || !t) {
        gs_host::set_error("row tensors: need 1..GS_MAX_ROW_TENSORS entries");
        return false;
    }
    for (int i = 0; i < count; ++i) {
        if (!t[i].dst || t[i].row_bytes <= 0 || t[i].row_bytes % 4 != 0 || t[i].role < GS_ROW_COPY ||
            t[i].role > GS_ROW_ZERO || (need_src && t[i].role != GS_ROW_ZERO && !t[i].src) ||
            (t[i].src && t[i].src == t[i].dst)) {
            gs_host::set_error("row tensors: need distinct src and dst, row_bytes a positive multiple of 4, a role");
            return false;
        }
    }
    return true;
}

int grid_for(int64_t work)
{
    int64_t b = (work + 255) / 256;
    const int64_t bmax = (int64_t)gs_host::sm_count() * 16;
    return (int)(b > bmax ? bmax : (b < 1 ? 1 : b));
}

}  // namespace
}  // namespace gs

extern "C" {

size_t gs_densify_workspace_size(int32_t n)
{
    if (n < 0) return 0;
    return gs::carve(nullptr, n).bytes;
}

int32_t gs_densify_select(int32_t n, const float* pos_acc, const float* col_acc, const int32_t* count, float tau_pos,
                          float tau_color, int32_t color_branch, int32_t max_new, void* workspace,
                          size_t workspace_bytes, int32_t* selected, int32_t* num_selected, gs_stream_t stream)
{
    using namespace gs;
    if (n < 0 || max_new < 0 || !num_selected || (n > 0 && (!pos_acc || !col_acc || !count || !workspace)) ||
        (max_new > 0 && n > 0 && !selected) || !(tau_pos > 0.0f) || !(tau_color > 0.0f)) {
        gs_host::set_error("gs_densify_select: bad arguments (need n, max_new >= 0, positive thresholds, buffers)");
        return GS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(num_selected, 0, sizeof(int32_t), st);
    if (n == 0 || max_new == 0) return gs_host::check_launch("gs_densify_select");
    uintptr_t b = reinterpret_cast<uintptr_t>(workspace);
    void* al = reinterpret_cast<void*>((b + 255) & ~uintptr_t(255));
    DsWs w = carve(al, n);
    if (workspace_bytes < w.bytes) {
        gs_host::set_error("gs_densify_select: workspace too small");
        return GS_ERR_ARG;
    }
    const int nb = (n + kBlk - 1) / kBlk;
    cudaMemsetAsync(w.hist, 0, sizeof(unsigned) * kHistBins, st);
    cudaMemsetAsync(w.st, 0, sizeof(SelState), st);
    gs::launch(k_ds_keys, nb, kBlk, 0, st, n, pos_acc, col_acc, count, tau_pos, tau_color, color_branch, w.keys,
               w.hist, w.st);
    gs::launch(k_ds_find, 1, kBlk, 0, st, max_new, 0, w.hist, w.st);
    cudaMemsetAsync(w.hist, 0, sizeof(unsigned) * kHistBins, st);
    gs::launch(k_ds_hist_lo, nb, kBlk, 0, st, n, w.keys, w.hist, w.st);
    gs::launch(k_ds_find, 1, kBlk, 0, st, max_new, 1, w.hist, w.st);
    gs::launch(k_ds_count_eq, nb, kBlk, 0, st, n, w.keys, w.st, w.blk);
    gs::launch(k_scan_blocks, 1, kBlk, 0, st, nb, w.blk, w.blk_base, nullptr);
    gs::launch(k_ds_rank_eq, nb, kBlk, 0, st, n, w.keys, w.st, w.blk_base, w.rank, w.blk);
    gs::launch(k_scan_blocks, 1, kBlk, 0, st, nb, w.blk, w.blk_base, num_selected);
    gs::launch(k_ds_write, nb, kBlk, 0, st, n, w.keys, w.rank, w.st, w.blk_base, selected);
    return gs_host::check_launch("gs_densify_select");
}

int32_t gs_prune_select(int32_t n, const float* opacity_logits, float logit_min, const float* log_scales,
                        float log_scale_max, void* workspace, size_t workspace_bytes, int32_t* keep,
                        int32_t* num_keep, gs_stream_t stream)
{
    using namespace gs;
    if (n < 0 || !num_keep || (n > 0 && (!opacity_logits || !keep || !workspace))) {
        gs_host::set_error("gs_prune_select: bad arguments");
        return GS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(num_keep, 0, sizeof(int32_t), st);
    if (n == 0) return gs_host::check_launch("gs_prune_select");
    uintptr_t b = reinterpret_cast<uintptr_t>(workspace);
    void* al = reinterpret_cast<void*>((b + 255) & ~uintptr_t(255));
    DsWs w = carve(al, n);
    if (workspace_bytes < w.bytes) {
        gs_host::set_error("gs_prune_select: workspace too small");
        return GS_ERR_ARG;
    }
    const int nb = (n + kBlk - 1) / kBlk;
    gs::launch(k_keep_count, nb, kBlk, 0, st, n, opacity_logits, logit_min, log_scales, log_scale_max, w.blk);
    gs::launch(k_scan_blocks, 1, kBlk, 0, st, nb, w.blk, w.blk_base, num_keep);
    gs::launch(k_keep_write, nb, kBlk, 0, st, n, opacity_logits, logit_min, log_scales, log_scale_max, w.blk_base,
               keep);
    return gs_host::check_launch("gs_prune_select");
}

int32_t gs_gather_rows(int32_t n_out, const int32_t* index, const GsRowTensor* tensors, int32_t count,
                       gs_stream_t stream)
{
    using namespace gs;
    if (n_out < 0 || (n_out > 0 && !index) || !check_rows(tensors, count, true)) {
        if (n_out < 0 || (n_out > 0 && !index)) gs_host::set_error("gs_gather_rows: bad arguments");
        return GS_ERR_ARG;
    }
    if (n_out == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int t = 0; t < count; ++t) {
        const int words = tensors[t].row_bytes / 4;
        gs::launch(k_rows, grid_for((int64_t)n_out * words), 256, 0, st, n_out, 0, index, nullptr,
                   static_cast<const uint32_t*>(tensors[t].src), static_cast<uint32_t*>(tensors[t].dst), words, 0,
                   tensors[t].role == GS_ROW_ZERO);
    }
    return gs_host::check_launch("gs_gather_rows");
}

int32_t gs_densify_grow(int32_t n_old, int32_t m, const int32_t* selected, const float* noise, float log_split_scale,
                        const GsRowTensor* tensors, int32_t count, gs_stream_t stream)
{
    using namespace gs;
    if (n_old < 0 || m < 0 || (m > 0 && (!selected || !noise))) {
        gs_host::set_error("gs_densify_grow: bad arguments");
        return GS_ERR_ARG;
    }
    if (!check_rows(tensors, count, true)) return GS_ERR_ARG;
    SplitArgs sa{};
    int roles[6] = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < count; ++t) {
        const GsRowTensor& r = tensors[t];
        roles[r.role]++;
        if (r.role == GS_ROW_MEANS || r.role == GS_ROW_LOG_SCALES) {
            if (r.row_bytes != 12) {
                gs_host::set_error("gs_densify_grow: means and log_scales rows are 3 floats");
                return GS_ERR_ARG;
            }
        }
        if (r.role == GS_ROW_MEANS) {
            sa.mean_src = static_cast<const float*>(r.src);
            sa.mean_dst = static_cast<float*>(r.dst);
        } else if (r.role == GS_ROW_LOG_SCALES) {
            sa.ls_src = static_cast<const float*>(r.src);
            sa.ls_dst = static_cast<float*>(r.dst);
        } else if (r.role == GS_ROW_QUATS) {
            if (r.row_bytes != 16 || (reinterpret_cast<uintptr_t>(r.src) & 15) != 0) {
                gs_host::set_error("gs_densify_grow: quaternion rows are 4 floats, 16-byte aligned");
                return GS_ERR_ARG;
            }
            sa.quat_src = static_cast<const float4*>(r.src);
        } else if (r.role == GS_ROW_STATE) {
            sa.state[sa.nstate] = static_cast<float*>(r.dst);
            sa.state_words[sa.nstate] = r.row_bytes / 4;
            sa.nstate++;
        }
    }
    if (roles[GS_ROW_MEANS] != 1 || roles[GS_ROW_LOG_SCALES] != 1 || roles[GS_ROW_QUATS] != 1) {
        gs_host::set_error("gs_densify_grow: exactly one means, one log_scales and one quats tensor");
        return GS_ERR_ARG;
    }
    const int n_new = n_old + m;
    if (n_new == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int t = 0; t < count; ++t) {
        const int words = tensors[t].row_bytes / 4;
        gs::launch(k_rows, grid_for((int64_t)n_new * words), 256, 0, st, n_new, n_old, nullptr, selected,
                   static_cast<const uint32_t*>(tensors[t].src), static_cast<uint32_t*>(tensors[t].dst), words,
                   tensors[t].role == GS_ROW_STATE, tensors[t].role == GS_ROW_ZERO);
    }
    if (m > 0) gs::launch(k_split, (m + 255) / 256, 256, 0, st, n_old, m, selected, noise, log_split_scale, sa);
    return gs_host::check_launch("gs_densify_grow");
}

}  // extern "C"
