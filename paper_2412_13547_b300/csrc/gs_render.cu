// gs_render.cu -- front-to-back alpha blending of the dilated lattice pixels
// (Sec. 3 Eq. 2; Sec. 3.1 Eq. 5), its backward replay, and the L1 loss.
//
// One CTA per downsampled tile, one thread per downsampled pixel. The tile's
// depth-ordered list is streamed through shared memory in batches of one
// record per thread; each record is re-based to the tile's hr origin while it
// is staged, so the per-pixel offset is a difference of two small numbers.
#include "gs_common.cuh"

namespace gs {
namespace {

__device__ __forceinline__ void load_stage(const float4* __restrict__ splats, uint32_t g, float X0, float Y0,
                                           float2& p, float4& co, float4& rgb)
{
    const float4 v0 = __ldg(splats + 4 * (int64_t)g);
    const float4 v1 = __ldg(splats + 4 * (int64_t)g + 1);
    const float4 v2 = __ldg(splats + 4 * (int64_t)g + 2);
    p.x = __fadd_rn(__fsub_rn(v0.x, X0), v2.z);
    p.y = __fadd_rn(__fsub_rn(v0.y, Y0), v2.w);
    co = make_float4(v0.z, v0.w, v1.x, v1.y);
    rgb = make_float4(v1.z, v1.w, v2.x, 0.0f);
}

// The region where a splat can pass the alpha gate: o exp(-q/2) >= 1/255 <=>
// q = d^T K d <= tau = 2 ln(255 o), an ellipse. Gate::box is its bounding box
// (x0, x1, y0, y1; tile-relative hr pixels), half-extents sqrt(tau Sigma_xx),
// sqrt(tau Sigma_yy) with Sigma = K^-1. tau and the extents are padded well
// beyond the FP32 error of the gate itself, so every pixel outside the region
// fails the gate in the kernel's own arithmetic: skipping it changes nothing.
// exact = false when only the box may be used (a degenerate conic).
struct Gate {
    float4 box;
    float tau;
    bool exact;
};

__device__ __forceinline__ Gate gate_region(float2 p, float4 co)
{
    const float inf = __int_as_float(0x7f800000);
    Gate G;
    G.tau = 0.0f;
    G.exact = false;
    if (!(co.w * 255.0f >= 1.0f)) {  // never passes
        G.box = make_float4(inf, -inf, inf, -inf);
        return G;
    }
    const float detK = det2(co.x, co.y, co.y, co.z);  // A C - B^2, FMA-exact
    const float tau = fmaxf(2.0f * __logf(255.0f * co.w), 0.0f) * 1.001f + 1e-3f;
    const float s = tau * __fdividef(1.0f, detK);
    const float ex = sqrtf(s * co.z) * 1.001f + 0.01f;
    const float ey = sqrtf(s * co.x) * 1.001f + 0.01f;
    if (!(detK > 0.0f) || !(co.x > 0.0f) || !(co.z > 0.0f) || !(ex < 1e30f) || !(ey < 1e30f)) {
        G.box = make_float4(-inf, inf, -inf, inf);
        return G;
    }
    G.box = make_float4(p.x - ex, p.x + ex, p.y - ey, p.y + ey);
    G.tau = tau;
    G.exact = true;
    return G;
}

// Lower bound of q = A u^2 + 2 B u v + C v^2 at (u, v), less a relative margin
// for the rounding of its terms.
__device__ __forceinline__ float quad_lo(float4 co, float u, float v)
{
    const float a = co.x * u * u, c = co.z * v * v, b = 2.0f * co.y * u * v;
    return (a + c + b) - 1e-5f * (a + c + fabsf(b));
}

// Whether the ellipse q(x - p) <= tau meets the rectangle [x0, x1] x [y0, y1]
// (coordinates relative to p): the centre is inside, or the minimum of the
// convex q over one of the four edges is within tau (each edge minimum is the
// unconstrained one along the edge, clamped to it).
__device__ __forceinline__ bool ellipse_meets_rect(float4 co, float kv, float ku, float tau, float x0, float x1,
                                                   float y0, float y1)
{
    if (x0 <= 0.0f && x1 >= 0.0f && y0 <= 0.0f && y1 >= 0.0f) return true;
    float q = quad_lo(co, x0, fminf(fmaxf(kv * x0, y0), y1));
    q = fminf(q, quad_lo(co, x1, fminf(fmaxf(kv * x1, y0), y1)));
    q = fminf(q, quad_lo(co, fminf(fmaxf(ku * y0, x0), x1), y0));
    q = fminf(q, quad_lo(co, fminf(fmaxf(ku * y1, x0), x1), y1));
    return q <= tau;
}

// Whether blend tile (tx, ty) lies in the blend-tile rectangle of record g
// (its own tile list holds g iff so).
__device__ __forceinline__ bool in_blend_rect(const float4* __restrict__ splats, uint32_t g, int tx, int ty)
{
    const float4 r = __ldg(splats + 4 * (int64_t)g + 3);
    return __float_as_int(r.x) <= tx && tx <= __float_as_int(r.z) && __float_as_int(r.y) <= ty &&
           ty <= __float_as_int(r.w);
}

// Exclusive rank of this thread's flag in its CTA of NT threads; *total gets
// the CTA's count. s_w: NT/32 + 1 ints of shared memory.
template <int NT>
__device__ __forceinline__ int cta_rank(bool flag, int* s_w, int* total)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ball = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) s_w[warp] = __popc(ball);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < NW; ++w) {
            const int c = s_w[w];
            s_w[w] = run;
            run += c;
        }
        s_w[NW] = run;
    }
    __syncthreads();
    const int r = s_w[warp] + __popc(ball & ((1u << lane) - 1u));
    *total = s_w[NW];
    __syncthreads();
    return r;
}

// Pixels of a CTA: each warp owns a compact 8-column block of 4*PPT rows and
// each lane one column and PPT rows of it (WarpBlock). Several pixels per
// thread share one shared-memory read of each staged record and, in the
// backward, one warp reduction per list entry.
template <int TILE, int PPT>
struct TileGeom {
    static constexpr int PIXELS = TILE * TILE;
    static constexpr int THREADS = PIXELS / PPT;
    // staged list entries per batch: 256, but 176 for the 64-thread CTAs of tile 16 at 4 pixels per
    // thread (the backward's default), whose staging arrays then leave shared memory for 13 CTAs
    // per SM
    static constexpr int BATCH = (TILE == 16 && PPT == 4) ? 176 : (PIXELS < 256 ? PIXELS : 256);
    static constexpr int WROWS = 4 * PPT;        // rows of a warp's block
    static constexpr int WCOLS = TILE / 8;       // warp blocks across the tile
};

// Bit w set when the gate region meets the pixel block of warp w (the blocks
// of WarpBlock below): computed once per staged entry, so a warp walks only
// the entries that can reach its pixels. A block must meet the region's box
// and, for a regular conic, the ellipse itself.
template <int TILE, int PPT>
__device__ __forceinline__ uint32_t warp_mask(float2 p, float4 co, int d)
{
    using Geo = TileGeom<TILE, PPT>;
    constexpr int NW = Geo::THREADS / 32;
    const Gate G = gate_region(p, co);
    const float4 box = G.box;
    // minimisers of q along an edge: v = -B u / C on x = const, u = -B v / A on y = const
    const float kv = -co.y * __fdividef(1.0f, co.z), ku = -co.y * __fdividef(1.0f, co.x);
    uint32_t m = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int bx = w % Geo::WCOLS, by = w / Geo::WCOLS;
        const float wx0 = (float)(d * bx * 8), wx1 = (float)(d * (bx * 8 + 7));
        const float wy0 = (float)(d * by * Geo::WROWS), wy1 = (float)(d * (by * Geo::WROWS + Geo::WROWS - 1));
        bool hit = !(box.x > wx1 || box.y < wx0 || box.z > wy1 || box.w < wy0);
        if (hit && G.exact)
            hit = ellipse_meets_rect(co, kv, ku, G.tau, wx0 - p.x, wx1 - p.x, wy0 - p.y, wy1 - p.y);
        m |= hit ? (1u << w) : 0u;
    }
    return m;
}

// A warp covers an 8-column block of 4 PPT rows; lane l takes column l % 8 and,
// with ILV (interleaved), rows l / 8 + 4k (k < PPT), else rows PPT (l / 8) + k.
// Interleaved, the rows a small splat covers fall on fewer of the lanes' pixel
// indices k, so a warp runs fewer of its per-pixel branches per entry.
template <int TILE, int PPT, bool ILV>
struct WarpBlock {
    static constexpr int RSTEP = ILV ? 4 : 1;  // rows between a thread's pixels
    int lx, ly0;                               // this thread's column and first row in the tile
    __device__ __forceinline__ WarpBlock(int tid)
    {
        using Geo = TileGeom<TILE, PPT>;
        const int warp = tid >> 5, lane = tid & 31;
        const int bx = warp % Geo::WCOLS, by = warp / Geo::WCOLS;
        lx = bx * 8 + (lane & 7);
        ly0 = by * Geo::WROWS + (lane >> 3) * (ILV ? 1 : PPT);
    }
    __device__ __forceinline__ int row(int k) const { return ly0 + RSTEP * k; }
};

constexpr bool kFwdInterleave = true;
constexpr bool kBwdInterleave = true;

// Blend of one tile (the body of the single-view and the batched kernels).
// FILTER: the list is the binning tile's; entries outside this blend tile are
// dropped while staging (what remains is this tile's own list, in order).
// COUNT: the blend counts are accumulated (instrumentation, compiled out
// when the caller passes no counts).
// flags (GS_FWD_*, uniform over the launch): GS_FWD_ZERO_GRAD2D, this tile's
// slice of the view's n 2D-gradient rows is zeroed (the CTAs of a view cover
// all its rows; the forward leaves DRAM idle, so the stores cost it nothing);
// GS_FWD_L1, each pixel's L1 loss term and dL/dimg are computed from the colour
// in registers (the gs_loss_l1 arithmetic) and the tile's sum added to *loss.
template <int TILE, int PPT, bool FILTER, bool COUNT>
__device__ __forceinline__ void render_fwd_tile(int tile, const float4* __restrict__ splats,
                                                const uint32_t* __restrict__ ids, const uint2* __restrict__ ranges,
                                                const Dil& dil, float3 bg, float* __restrict__ img,
                                                float* __restrict__ t_final, uint32_t* __restrict__ last,
                                                unsigned long long* __restrict__ counts, const ViewDev& V, int n,
                                                uint32_t flags)
{
    using Geo = TileGeom<TILE, PPT>;
    constexpr int NT = Geo::THREADS, BATCH = Geo::BATCH;
    constexpr int ROUND = NT < BATCH ? NT : BATCH;  // candidates per filtering round
    __shared__ float2 s_p[BATCH];
    __shared__ uint32_t s_mask[BATCH];
    __shared__ float4 s_co[BATCH];
    __shared__ float4 s_rgb[BATCH];
    __shared__ uint32_t s_pos[FILTER ? BATCH : 1];
    __shared__ int s_w[NT / 32 + 1];
    __shared__ unsigned long long s_cnt[3];

    const int tx = tile % dil.tiles_x, ty = tile / dil.tiles_x;
    const WarpBlock<TILE, PPT, kFwdInterleave> wb(threadIdx.x);
    const int u = tx * TILE + wb.lx;
    // hr origin of the tile and this thread's hr offsets from it (small exact floats)
    const float X0 = (float)(dil.d * tx * TILE + dil.ox), Y0 = (float)(dil.d * ty * TILE + dil.oy);
    const float xr = (float)(dil.d * wb.lx);

    if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0ull;
    if (flags & GS_FWD_ZERO_GRAD2D) {
        // rows [r0, r1) of this tile's share; a row is 3 float4 (16-byte aligned, checked on the host)
        const int ntiles = dil.tiles_x * dil.tiles_y;
        const int64_t per = ((int64_t)n + ntiles - 1) / ntiles;
        const int64_t r0 = min((int64_t)n, (int64_t)tile * per), r1 = min((int64_t)n, r0 + per);
        float4* g4 = reinterpret_cast<float4*>(V.grad2d);
        for (int64_t i = 3 * r0 + threadIdx.x; i < 3 * r1; i += NT) g4[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    const uint2 rg = ranges[FILTER ? bin_tile_of(dil, tile) : tile];
    float T[PPT], C0[PPT], C1[PPT], C2[PPT], yr[PPT];
    uint32_t last_pos[PPT], last_own[PPT];  // last blended entry: binning-list and own-list position + 1
    bool done[PPT];
    int n_live = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        T[k] = 1.0f; C0[k] = C1[k] = C2[k] = 0.0f; last_pos[k] = 0; last_own[k] = 0;
        yr[k] = (float)(dil.d * wb.row(k));
        done[k] = !(u < dil.w_ds && ty * TILE + wb.row(k) < dil.h_ds);
        n_live += done[k] ? 0 : 1;
    }
    uint32_t n_eval = 0, n_blend = 0;

    uint32_t next = rg.x;
    uint32_t own_base = 0;  // entries of this tile's own list staged before the batch
    while (next < rg.y) {
        if (__syncthreads_count(n_live == 0) == NT) break;
        const uint32_t start = next;
        int cnt;
        if constexpr (!FILTER) {
            cnt = (int)((rg.y - next) < (uint32_t)BATCH ? (rg.y - next) : (uint32_t)BATCH);
            for (int i = threadIdx.x; i < cnt; i += NT) {
                float2 p; float4 co, rgb;
                load_stage(splats, __ldg(ids + start + i), X0, Y0, p, co, rgb);
                s_p[i] = p;
                s_mask[i] = warp_mask<TILE, PPT>(p, co, dil.d);
                s_co[i] = conic_exp2(co);
                s_rgb[i] = rgb;
            }
            next += (uint32_t)cnt;
        } else {
            // rounds of ROUND candidates until the batch is full or the list ends
            cnt = 0;
            while (cnt + ROUND <= BATCH && next < rg.y) {
                const uint32_t e = next + threadIdx.x;
                uint32_t g = 0;
                bool keep = false;
                if ((int)threadIdx.x < ROUND && e < rg.y) {
                    g = __ldg(ids + e);
                    keep = in_blend_rect(splats, g, tx, ty);
                }
                int total;
                const int r = cta_rank<NT>(keep, s_w, &total);
                if (keep) {
                    float2 p; float4 co, rgb;
                    load_stage(splats, g, X0, Y0, p, co, rgb);
                    s_p[cnt + r] = p;
                    s_mask[cnt + r] = warp_mask<TILE, PPT>(p, co, dil.d);
                    s_co[cnt + r] = conic_exp2(co);
                    s_rgb[cnt + r] = rgb;
                    s_pos[cnt + r] = e - rg.x + 1;
                }
                cnt += total;
                next = (rg.y - next) < (uint32_t)ROUND ? rg.y : next + ROUND;
                }
        }
        __syncthreads();
        int lj[PPT];  // batch slot of the pixel's last blended entry in this batch, or -1
#pragma unroll
        for (int k = 0; k < PPT; ++k) lj[k] = -1;
        {
            // every live pixel visits every entry (the blend count of the method); a warp
            // takes only the entries whose gate box meets its pixel block, 32 at a time.
            // The loops below are uniform over the warp (they hold warp votes): a thread whose
            // pixels are done keeps stepping with its warp and does nothing.
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                if (!__any_sync(0xffffffffu, n_live > 0)) break;
                const int c1 = min(cnt, c0 + 32);
                const bool hit = c0 + lane < c1 && ((s_mask[c0 + lane] >> warp) & 1u);
                uint32_t m = __ballot_sync(0xffffffffu, hit);
                int next_j = c0;  // entries before next_j are counted in n_eval
                while (m != 0u) {
                    const int j = c0 + __ffs(m) - 1;
                    m &= m - 1u;
                    if constexpr (COUNT) {
                        n_eval += (uint32_t)n_live * (uint32_t)(j - next_j + 1);
                        next_j = j + 1;
                    }
                    const float2 p = s_p[j];
                    const float4 co = s_co[j];
                    const float dx = __fsub_rn(xr, p.x);
                    const SplatRow row = splat_row(dx, co);
                    // the gates of all this thread's pixels first, free of branches so that
                    // their dependency chains interleave; then the blends, in pixel order
                    float e2[PPT];
                    bool use[PPT];
                    if constexpr (PPT % 2 == 0) {
                        // pixel pairs on the paired FP32 instructions, each element rounded as the
                        // scalar form rounds it (forward 0.408 -> 0.397 ms on the 4K step)
                        const f32x2 pyP = pk(p.y, p.y), czzP = pk(co.z, co.z);
                        const f32x2 adxP = pk(row.adx2, row.adx2), bdxP = pk(row.bdx, row.bdx);
#pragma unroll
                        for (int q = 0; q < PPT / 2; ++q) {
                            const f32x2 dyP = sub2(pk(yr[2 * q], yr[2 * q + 1]), pyP);
                            unpk(fma2(bdxP, dyP, fma2(czzP, mul2(dyP, dyP), adxP)), e2[2 * q], e2[2 * q + 1]);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < PPT; ++k) e2[k] = splat_power(row, __fsub_rn(yr[k], p.y), co.z);
                    }
#pragma unroll
                    for (int k = 0; k < PPT; ++k) use[k] = !done[k] && splat_gate(e2[k], co.w);
                    const float4 c = s_rgb[j];  // once per entry, not per blending pixel
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (!use[k]) continue;
                        const float alpha = fminf(kAlphaMax, exp2_sfu(e2[k]));
                        // T (1 - alpha) in two operations with w reused, rounding pinned so that no
                        // launch shape contracts it differently
                        const float w = __fmul_rn(alpha, T[k]);
                        const float Tn = __fsub_rn(T[k], w);
                        if (Tn < kTStop) { done[k] = true; --n_live; continue; }
                        C0[k] = fmaf(c.x, w, C0[k]);
                        C1[k] = fmaf(c.y, w, C1[k]);
                        C2[k] = fmaf(c.z, w, C2[k]);
                        T[k] = Tn;
                        lj[k] = j;
                        if constexpr (COUNT) ++n_blend;
                    }
                    // no vote per entry on whether the warp still has live pixels: done pixels skip
                    // their gates above, and the chunk loop votes before the next 32 entries
                    // (a vote per entry cost 5% of the forward on the 4K step)
                }
                if constexpr (COUNT) n_eval += (uint32_t)n_live * (uint32_t)(c1 - next_j);
            }
        }
        // positions of the last blended entries, read before the next batch is staged
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (lj[k] < 0) continue;
            last_pos[k] = FILTER ? s_pos[lj[k]] : start + (uint32_t)lj[k] - rg.x + 1;
            if constexpr (COUNT) last_own[k] = own_base + (uint32_t)lj[k] + 1;
        }
        own_base += (uint32_t)cnt;
    }
    const bool l1 = (flags & GS_FWD_L1) != 0;
    const bool t8 = V.target_dtype == GS_TARGET_U8;
    const float inv = (float)(1.0 / (3.0 * (double)dil.w_ds * (double)dil.h_ds));
    float l1_acc = 0.0f;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int v = ty * TILE + wb.row(k);
        if (u < dil.w_ds && v < dil.h_ds) {
            const int64_t pix = (int64_t)v * dil.w_ds + u;
            const float col[3] = {fmaf(T[k], bg.x, C0[k]), fmaf(T[k], bg.y, C1[k]), fmaf(T[k], bg.z, C2[k])};
            img[3 * pix] = col[0];
            img[3 * pix + 1] = col[1];
            img[3 * pix + 2] = col[2];
            t_final[pix] = T[k];
            last[pix] = last_pos[k];
            if (l1) {
                // the L1 term against the hr target at the lattice pixel (gs_loss_l1's arithmetic)
                const int64_t h = ((int64_t)(dil.d * v + dil.oy) * V.cam.width + (dil.d * u + dil.ox)) * 3;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float tg = t8 ? target_value<GS_TARGET_U8>(V.target, h + ch)
                                        : target_value<GS_TARGET_F32>(V.target, h + ch);
                    const float r = col[ch] - tg;
                    l1_acc += fabsf(r);
                    V.dl[3 * pix + ch] = r > 0.0f ? inv : (r < 0.0f ? -inv : 0.0f);
                }
            }
        }
    }
    if (l1) {
        __shared__ float s_l1[NT / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l1_acc += __shfl_down_sync(0xffffffffu, l1_acc, o);
        if ((threadIdx.x & 31) == 0) s_l1[threadIdx.x >> 5] = l1_acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int w = 0; w < NT / 32; ++w) t += s_l1[w];
            atomicAdd(V.loss, t * inv);
        }
    }
    if constexpr (COUNT) {
        unsigned long long e = n_eval, b = n_blend, r = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) r += last_own[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_down_sync(0xffffffffu, e, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
            r += __shfl_down_sync(0xffffffffu, r, o);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&s_cnt[0], e);
            atomicAdd(&s_cnt[1], b);
            atomicAdd(&s_cnt[2], r);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&counts[0], s_cnt[0]);
            atomicAdd(&counts[1], s_cnt[1]);
            atomicAdd(&counts[2], s_cnt[2]);
        }
    }
}

// Sum of 9 per-lane values over a warp by recursive halving: at each step a
// lane keeps one half of its live slots and sends the other half to its xor
// partner (5 + 3 + 2 + 1 + 1 = 12 shuffles instead of 9 x 5). On return lane L
// holds the warp total of component comp (or comp = -1); lanes L and L^1 hold
// the same component, and components 0..8 each sit on one such pair.
__device__ __forceinline__ float warp_sum9(const float (&v)[9], int lane, int& comp)
{
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
    float w[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float hi = i < 4 ? v[5 + i] : 0.0f;
        const float keep = h16 ? hi : v[i];
        const float send = h16 ? v[i] : hi;
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float x[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float hi = i < 2 ? w[3 + i] : 0.0f;
        const float keep = h8 ? hi : w[i];
        const float send = h8 ? w[i] : hi;
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float y[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float hi = i < 1 ? x[2] : 0.0f;
        const float keep = h4 ? hi : x[i];
        const float send = h4 ? x[i] : hi;
        y[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float z = (h2 ? y[1] : y[0]) + __shfl_xor_sync(0xffffffffu, h2 ? y[0] : y[1], 2);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    // slot bookkeeping: y slot -> x slot -> w slot -> component
    int ys = h2 ? 1 : 0;
    int xs = h4 ? (ys == 0 ? 2 : -1) : ys;
    int ws = xs < 0 ? -1 : (h8 ? (xs < 2 ? 3 + xs : -1) : xs);
    comp = ws < 0 ? -1 : (h16 ? (ws < 4 ? 5 + ws : -1) : ws);
    return z;
}

// dL/d centre (x, y), dL/dA and dL/dB of one entry's conic (A, B, C) from
// the tile's sums a[0..5] = sum q, q dy, q dy^2, dx q, dx^2 q, dx dy q over its
// pixels, q = dL/d(ln G) with ln G = -(A dx^2 + C dy^2)/2 - B dx dy, and the
// staged base-2 coefficients s = (a, b, c, .) = log2(e) (-A/2, -B, -C/2, .):
// dL/dA = -a[4]/2, dL/dB = -a[5] (dL/dC = -a[2]/2 and dL/do = a[0]/o are formed
// by the caller), and d(ln G)/dp = (A dx + B dy, C dy + B dx)
// = -ln 2 (2a dx + b dy, 2c dy + b dx).
__device__ __forceinline__ float4 grad_from_sums(const float* a, float4 s)
{
    const float gx = -kLn2 * fmaf(s.y, a[1], 2.0f * s.x * a[3]);
    const float gy = -kLn2 * fmaf(s.y, a[3], 2.0f * s.z * a[1]);
    return make_float4(gx, gy, -0.5f * a[4], -a[5]);
}

// Backward: replay each pixel's list back to front from (t_final, last),
// recovering T_i = T_{i+1} / (1 - alpha_i). A warp skips entries past the last
// contributor of all its pixels and entries whose gate box misses its block.
// Per remaining entry a thread sums 9 values over its pixels (the colour
// gradients and the six sums the other gradients are linear in), the warp sums
// them (warp_sum9), one lane per value adds the total into a per-batch
// shared-memory accumulator, and at the end of the batch each (tile, Gaussian)
// expands its sums into its 2D gradient (grad_from_sums) and adds that with one
// set of vector atomics.
template <int TILE, int PPT, bool FILTER>
__device__ __forceinline__ void render_bwd_tile(int tile, const float4* __restrict__ splats,
                                                const uint32_t* __restrict__ ids, const uint2* __restrict__ ranges,
                                                const Dil& dil, float3 bg, const float* __restrict__ t_final,
                                                const uint32_t* __restrict__ last, const float* __restrict__ dl_dimg,
                                                float* __restrict__ grad2d)
{
    using Geo = TileGeom<TILE, PPT>;
    constexpr int NT = Geo::THREADS, BATCH = Geo::BATCH;
    constexpr int ROUND = NT < BATCH ? NT : BATCH;  // candidates per filtering round
    __shared__ float2 s_p[BATCH];
    __shared__ uint32_t s_mask[BATCH];
    __shared__ float4 s_co[BATCH];
    __shared__ float4 s_rgb[BATCH];
    __shared__ uint32_t s_id[BATCH];
    __shared__ float s_acc[BATCH][9];
    __shared__ uint32_t s_rel[FILTER ? BATCH : 1];
    __shared__ int s_w[NT / 32 + 1];
    __shared__ uint32_t s_max_last;

    const int tx = tile % dil.tiles_x, ty = tile / dil.tiles_x;
    const WarpBlock<TILE, PPT, kBwdInterleave> wb(threadIdx.x);
    const int lane = threadIdx.x & 31;
    const int u = tx * TILE + wb.lx;
    const float X0 = (float)(dil.d * tx * TILE + dil.ox), Y0 = (float)(dil.d * ty * TILE + dil.oy);
    const float xr = (float)(dil.d * wb.lx);
    const uint2 rg = ranges[FILTER ? bin_tile_of(dil, tile) : tile];

    // gS: the pixel's colour gradient dotted with the colour accumulated behind the entry
    // being replayed (starting with T_final * bg). dL/dalpha only needs that dot product,
    // so one scalar per pixel replaces the three accumulated channels.
    float T[PPT], gS[PPT], g0[PPT], g1[PPT], g2[PPT], yr[PPT];
    uint32_t n_last[PPT];
    uint32_t my_max = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int v = ty * TILE + wb.row(k);
        yr[k] = (float)(dil.d * wb.row(k));
        T[k] = 1.0f; g0[k] = g1[k] = g2[k] = 0.0f; n_last[k] = 0;
        if (u < dil.w_ds && v < dil.h_ds) {
            const int64_t pix = (int64_t)v * dil.w_ds + u;
            T[k] = t_final[pix];
            n_last[k] = last[pix];
            g0[k] = dl_dimg[3 * pix];
            g1[k] = dl_dimg[3 * pix + 1];
            g2[k] = dl_dimg[3 * pix + 2];
        }
        gS[k] = T[k] * (g0[k] * bg.x + g1[k] * bg.y + g2[k] * bg.z);
        my_max = max(my_max, n_last[k]);
    }
    // with an even number of pixels a thread replays them in pairs, two pixels per paired FP32
    // instruction (pair q holds pixels 2q and 2q + 1)
    constexpr bool PAIRS = (PPT % 2) == 0;
    constexpr int NP = PAIRS ? PPT / 2 : 1;
    f32x2 TP[NP], gSP[NP], g0P[NP], g1P[NP], g2P[NP], yrP[NP];
    if constexpr (PAIRS) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            TP[q] = pk(T[2 * q], T[2 * q + 1]);
            gSP[q] = pk(-gS[2 * q], -gS[2 * q + 1]);  // the paired form carries -g.S
            g0P[q] = pk(g0[2 * q], g0[2 * q + 1]);
            g1P[q] = pk(g1[2 * q], g1[2 * q + 1]);
            g2P[q] = pk(g2[2 * q], g2[2 * q + 1]);
            yrP[q] = pk(yr[2 * q], yr[2 * q + 1]);
        }
    }
    const uint32_t warp_max = __reduce_max_sync(0xffffffffu, my_max);
    if (threadIdx.x == 0) s_max_last = 0;
    __syncthreads();
    if (lane == 0 && warp_max > 0) atomicMax(&s_max_last, warp_max);
    __syncthreads();
    const uint32_t n_proc = s_max_last;
    if (n_proc == 0) return;

    // batches walk the list positions [0, n_proc) back to front. With FILTER a
    // batch gathers rounds of ROUND candidate positions, highest first, into the
    // top of the staging arrays until the next round might not fit; the kept
    // entries then sit in slots [base, BATCH) in ascending list order.
    uint32_t hi = n_proc;
    while (hi > 0) {
        int cnt, base;
        uint32_t lo = 0;
        __syncthreads();
        if constexpr (!FILTER) {
            lo = hi > (uint32_t)BATCH ? hi - BATCH : 0u;
            cnt = (int)(hi - lo);
            base = 0;
            for (int i = threadIdx.x; i < cnt; i += NT) {
                const uint32_t g = __ldg(ids + rg.x + lo + i);
                float2 p; float4 co, rgb;
                load_stage(splats, g, X0, Y0, p, co, rgb);
                s_p[i] = p;
                s_mask[i] = warp_mask<TILE, PPT>(p, co, dil.d);
                s_co[i] = conic_exp2(co);
                s_rgb[i] = make_float4(rgb.x, rgb.y, rgb.z, co.w > 0.0f ? __frcp_rn(co.w) : 0.0f);  // w: 1/o
                s_id[i] = g;
#pragma unroll
                for (int k = 0; k < 9; ++k) s_acc[i][k] = 0.0f;
            }
            hi = lo;
        } else {
            int filled = 0;
            while (filled + ROUND <= BATCH && hi > 0) {
                lo = hi > (uint32_t)ROUND ? hi - ROUND : 0u;
                const uint32_t rel = lo + threadIdx.x;
                uint32_t g = 0;
                bool keep = false;
                if ((int)threadIdx.x < ROUND && rel < hi) {
                    g = __ldg(ids + rg.x + rel);
                    keep = in_blend_rect(splats, g, tx, ty);
                }
                int total;
                const int r = cta_rank<NT>(keep, s_w, &total);
                if (keep) {
                    const int slot = BATCH - filled - total + r;
                    float2 p; float4 co, rgb;
                    load_stage(splats, g, X0, Y0, p, co, rgb);
                    s_p[slot] = p;
                    s_mask[slot] = warp_mask<TILE, PPT>(p, co, dil.d);
                    s_co[slot] = conic_exp2(co);
                    s_rgb[slot] = make_float4(rgb.x, rgb.y, rgb.z, co.w > 0.0f ? __frcp_rn(co.w) : 0.0f);  // w: 1/o
                    s_id[slot] = g;
                    s_rel[slot] = rel;
#pragma unroll
                    for (int k = 0; k < 9; ++k) s_acc[slot][k] = 0.0f;
                }
                filled += total;
                hi = lo;
            }
            cnt = filled;
            base = BATCH - filled;
        }
        __syncthreads();
        const int warp = threadIdx.x >> 5;
        // 32 entries at a time, from the top: those whose gate box meets this warp's pixel
        // block and that lie before the last contributor of one of its pixels
        for (int c1 = base + cnt; c1 > base; c1 -= 32) {
            const int c0 = max(base, c1 - 32);
            const int jj = c0 + lane;
            bool hit = false;
            if (jj < c1) {
                const uint32_t pj = FILTER ? s_rel[jj] : lo + (uint32_t)jj;
                hit = pj < warp_max && ((s_mask[jj] >> warp) & 1u);
            }
            uint32_t m = __ballot_sync(0xffffffffu, hit);
            while (m != 0u) {
                const int bit = 31 - __clz(m);
                m &= ~(1u << bit);
                const int j = c0 + bit;
                const uint32_t pos = FILTER ? s_rel[j] : lo + (uint32_t)j;
                float r[9];
                // dL/dpower summed over the thread's pixels, and times dy and dy^2: the conic,
                // centre and opacity gradients are those three sums times per-entry factors
                float q0 = 0.0f, q1 = 0.0f, q2 = 0.0f;
                bool contrib = false;
                const float2 p = s_p[j];
                const float4 co = s_co[j];
                const float4 c = s_rgb[j];
                const float dx = __fsub_rn(xr, p.x);
                const SplatRow row = splat_row(dx, co);
                if constexpr (PAIRS) {
                    // Pairs of pixels, branch-free: a pixel the entry does not reach (gate, or past
                    // its last contributor) takes alpha = 0, so that its transmittance is divided
                    // by 1 exactly and its weight and opacity terms are 0; the exponent is the
                    // scalar form's, element by element.
                    const f32x2 pyP = pk(p.y, p.y), czzP = pk(co.z, co.z);
                    const f32x2 adxP = pk(row.adx2, row.adx2), bdxP = pk(row.bdx, row.bdx);
                    const f32x2 cxP = pk(c.x, c.x), cyP = pk(c.y, c.y), czP = pk(c.z, c.z), oneP = pk(1.0f, 1.0f);
                    f32x2 q0P = pk(0.0f, 0.0f), q1P = q0P, q2P = q0P, r6P = q0P, r7P = q0P, r8P = q0P;
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const f32x2 dyP = sub2(yrP[q], pyP);
                        const f32x2 e2P = fma2(bdxP, dyP, fma2(czzP, mul2(dyP, dyP), adxP));
                        float e0, e1;
                        unpk(e2P, e0, e1);
                        const bool u0 = pos < n_last[2 * q] && splat_gate(e0, co.w);
                        const bool u1 = pos < n_last[2 * q + 1] && splat_gate(e1, co.w);
                        const float a0 = exp2_sfu(e0), a1 = exp2_sfu(e1);  // alpha before the clamp
                        // with the signs folded in: nal = -alpha (clamped), nw = -w, and gSP = -g.S,
                        // so that dL/dalpha = T_i g.c - (1 / (1 - alpha)) g.S is one multiply and one
                        // FMA; the colour and dL/dpower sums come out negated (pk_sum_neg below)
                        const float nal0 = u0 ? fmaxf(-kAlphaMax, -a0) : 0.0f;
                        const float nal1 = u1 ? fmaxf(-kAlphaMax, -a1) : 0.0f;
                        // the opacity and conic terms only below the clamp (nal > -kAlphaMax: -nal
                        // is the unclamped alpha of a replayed pixel, or 0)
                        const f32x2 naP = pk(nal0 > -kAlphaMax ? nal0 : 0.0f, nal1 > -kAlphaMax ? nal1 : 0.0f);
                        const f32x2 nalP = pk(nal0, nal1);
                        float o0, o1;
                        unpk(add2(oneP, nalP), o0, o1);
                        const f32x2 invP = pk(__fdividef(1.0f, o0), __fdividef(1.0f, o1));
                        const f32x2 TiP = mul2(TP[q], invP);
                        const f32x2 nwP = mul2(nalP, TiP);
                        r6P = fma2(nwP, g0P[q], r6P);
                        r7P = fma2(nwP, g1P[q], r7P);
                        r8P = fma2(nwP, g2P[q], r8P);
                        const f32x2 gcP = fma2(g2P[q], czP, fma2(g1P[q], cyP, mul2(g0P[q], cxP)));
                        const f32x2 dalP = fma2(TiP, gcP, mul2(invP, gSP[q]));
                        gSP[q] = fma2(nwP, gcP, gSP[q]);
                        TP[q] = TiP;
                        const f32x2 dpP = mul2(naP, dalP);
                        const f32x2 tP = mul2(dpP, dyP);
                        q0P = add2(q0P, dpP);
                        q1P = add2(q1P, tP);
                        q2P = fma2(tP, dyP, q2P);
                    }
                    q0 = pk_sum_neg(q0P);
                    q1 = pk_sum_neg(q1P);
                    q2 = pk_sum_neg(q2P);
                    r[6] = pk_sum_neg(r6P);
                    r[7] = pk_sum_neg(r7P);
                    r[8] = pk_sum_neg(r8P);
                } else {
                // gates of all this thread's pixels first (branch-free), then the replay
                r[6] = r[7] = r[8] = 0.0f;
                float dyk[PPT], e2[PPT];
                bool use[PPT];
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    dyk[k] = __fsub_rn(yr[k], p.y);
                    e2[k] = splat_power(row, dyk[k], co.z);
                    use[k] = pos < n_last[k] && splat_gate(e2[k], co.w);
                }
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (!use[k]) continue;
                    const float dy = dyk[k];
                    const float a_raw = exp2_sfu(e2[k]);  // alpha before the 0.99 clamp, as in the forward
                    const float alpha = fminf(kAlphaMax, a_raw);
                    contrib = true;
                    // one SFU reciprocal serves both divisions by (1 - alpha) >= 0.01 (a few
                    // ulp per replayed entry, far inside the gradient tolerance)
                    const float inv = __fdividef(1.0f, 1.0f - alpha);
                    const float Ti = T[k] * inv;
                    const float w = alpha * Ti;
                    r[6] = fmaf(w, g0[k], r[6]);
                    r[7] = fmaf(w, g1[k], r[7]);
                    r[8] = fmaf(w, g2[k], r[8]);
                    // dL/dalpha = sum_ch g_ch (T_i c_ch - S_ch / (1 - alpha)) = (T g.c - g.S) / (1 - alpha)
                    const float gc = fmaf(g2[k], c.z, fmaf(g1[k], c.y, g0[k] * c.x));
                    const float dalpha = inv * fmaf(T[k], gc, -gS[k]);
                    gS[k] = fmaf(w, gc, gS[k]);
                    T[k] = Ti;
                    if (a_raw < kAlphaMax) {
                        const float dpower = a_raw * dalpha;
                        const float t = dpower * dy;
                        q0 += dpower;
                        q1 += t;
                        q2 = fmaf(t, dy, q2);
                    }
                }
                }
                // the six sums the conic, centre and opacity gradients are linear in (a lane's
                // pixels share dx): q0, q1 = sum dpower dy, q2 = sum dpower dy^2, and dx q0,
                // dx^2 q0, dx q1. The tile's totals are expanded once per entry when the batch
                // is flushed (grad_from_sums), not on every warp visit.
                r[0] = q0;
                r[1] = q1;
                r[2] = q2;
                r[3] = dx * q0;
                r[4] = r[3] * dx;
                r[5] = dx * q1;
                // the paired form reduces on every visit: nearly all visits (97% on the 4K step)
                // have a contributing pixel, and a visit without one adds zeros
                if (PAIRS || __any_sync(0xffffffffu, contrib)) {
                    int comp;
                    const float z = warp_sum9(r, lane, comp);
                    if (comp >= 0 && (lane & 1) == 0) atomicAdd(&s_acc[j][comp], z);
                }
        }
        }
        __syncthreads();
        for (int i = base + (int)threadIdx.x; i < base + cnt; i += NT) {
            const float* a = s_acc[i];
            bool any = false;
#pragma unroll
            for (int k = 0; k < 9; ++k) any |= (a[k] != 0.0f);
            if (any) {
                const float4 g = grad_from_sums(a, s_co[i]);
                const float4 h = make_float4(-0.5f * a[2], a[0] * s_rgb[i].w, a[6], a[7]);
                float* dst = grad2d + (int64_t)GS_GRAD2D_FLOATS * s_id[i];
                atomicAdd(reinterpret_cast<float4*>(dst), g);
                atomicAdd(reinterpret_cast<float4*>(dst + 4), h);
                atomicAdd(dst + 8, a[8]);
            }
        }
    }
}

// One CTA per tile of the batch; with an order, CTA i takes tile order[i]
// (longest lists first, so the block scheduler dispatches greedily
// longest-first across all views).
// MULTI false: one view, whose fields the kernel reads at fixed offsets.
// FILTER: the views bin with coarser tiles than they blend (bin_shift > 0).
// With up to 2 pixels per thread the forward is held to 64 registers (1024
// threads' worth of CTAs per SM), which it fits without spilling; the
// backward keeps what it needs (about 72), measured faster than spilling for
// the extra CTA.
template <int TILE, int PPT>
constexpr int fwd_min_blocks()
{
    // tile 16 at 2 pixels per thread: 9 CTAs of 128 threads (56 registers, no spills), 2% faster
    // than 8; 10 spilled
    return (TILE == 16 && PPT == 2) ? 9 : (PPT <= 2 ? 1024 / TileGeom<TILE, PPT>::THREADS : 1);
}

// The backward at tile 16 and 4 pixels per thread (64-thread CTAs) is held to
// 13 CTAs per SM (69 registers, no spills; 176-entry batches, so that shared
// memory holds 13): 5% faster than 12 CTAs with 192-entry batches, and 14 CTAs
// with 160-entry batches gave no more.
template <int TILE, int PPT>
constexpr int bwd_min_blocks()
{
    return (TILE == 16 && PPT == 4) ? 13 : 1;
}

template <int TILE, int PPT, bool MULTI, bool FILTER, bool COUNT>
__global__ void __launch_bounds__(TileGeom<TILE, PPT>::THREADS, (fwd_min_blocks<TILE, PPT>()))
k_render_fwd(const __grid_constant__ Batch b, const uint32_t* __restrict__ order, float3 bg,
             unsigned long long* __restrict__ counts, int n, uint32_t flags)
{
    kernel_prologue();
    const int gt = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    const ViewDev& V = b.v[MULTI ? view_of_tile(b, gt) : 0];
    render_fwd_tile<TILE, PPT, FILTER, COUNT>(gt - V.tile_begin, V.splats, V.ids, V.ranges, V.dil, bg, V.img,
                                              V.t_final, V.last, counts, V, n, flags);
}

template <int TILE, int PPT, bool MULTI, bool FILTER>
__global__ void __launch_bounds__(TileGeom<TILE, PPT>::THREADS, (bwd_min_blocks<TILE, PPT>()))
k_render_bwd(const __grid_constant__ Batch b, const uint32_t* __restrict__ order, float3 bg)
{
    kernel_prologue();
    const int gt = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    const ViewDev& V = b.v[MULTI ? view_of_tile(b, gt) : 0];
    render_bwd_tile<TILE, PPT, FILTER>(gt - V.tile_begin, V.splats, V.ids, V.ranges, V.dil, bg, V.t_final, V.last,
                                       V.dl, reinterpret_cast<float*>(V.grad2d));
}

__global__ void k_loss_zero(const __grid_constant__ Batch b)
{
    kernel_prologue();
    if ((int)threadIdx.x < b.nviews) *b.v[threadIdx.x].loss = 0.0f;
}

// L1 loss of each view (blockIdx.y) and its gradient sign/(3P) w.r.t. the
// rendered pixels, against the hr target sampled at the view's lattice.
// The L1 terms of the lattice pixels a thread takes (grid-stride), for a
// target of type TD; returns the thread's sum of |img - target|.
template <int TD>
__device__ __forceinline__ float loss_l1_pixels(const ViewDev& V, float inv)
{
    const Dil& dil = V.dil;
    const int width = V.cam.width;
    const int64_t P = (int64_t)dil.w_ds * dil.h_ds;
    const float* __restrict__ img = V.img;
    float* __restrict__ dl = V.dl;
    float acc = 0.0f;
    for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < P;
         pix += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(pix % dil.w_ds), v = (int)(pix / dil.w_ds);
        const int64_t h = ((int64_t)(dil.d * v + dil.oy) * width + (dil.d * u + dil.ox)) * 3;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float r = img[3 * pix + ch] - target_value<TD>(V.target, h + ch);
            acc += fabsf(r);
            dl[3 * pix + ch] = r > 0.0f ? inv : (r < 0.0f ? -inv : 0.0f);
        }
    }
    return acc;
}

__global__ void k_loss_l1(const __grid_constant__ Batch b)
{
    kernel_prologue();
    const ViewDev& V = b.v[blockIdx.y];
    const Dil& dil = V.dil;
    const int64_t P = (int64_t)dil.w_ds * dil.h_ds;
    const float inv = (float)(1.0 / (3.0 * (double)P));
    float acc = V.target_dtype == GS_TARGET_U8 ? loss_l1_pixels<GS_TARGET_U8>(V, inv)
                                               : loss_l1_pixels<GS_TARGET_F32>(V, inv);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ float s_sum[32];
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_sum[w];
        atomicAdd(V.loss, t * inv);
    }
}

// Pixels per thread: 0 picks the default; otherwise 1, 2 or 4 such that the
// CTA is whole warps and at most 512 threads (tile 8: 1 or 2; tile 32: 2 or 4).
// The kernels use full-warp shuffles and votes, so a partial warp is refused.
// Defaults: the forward 1 at tile 8, else 2; the backward the same, but 4 at
// tile 16 when the launch has at least kWideBwdTiles tiles: its per-entry warp
// reduction then serves 128 pixels (8% faster on the 4K step, 8160 tiles),
// while on fewer tiles the halved warps per CTA leave the SMs short of warps
// (30% slower at 1920x1080 d=2, 2040 tiles). The forward is fastest at 2.
constexpr int kWideBwdTiles = 4096;

int resolve_ppt(int tile, int ppt, bool bwd, int tiles)
{
    if (ppt == 0) return tile == 8 ? 1 : ((bwd && tile == 16 && tiles >= kWideBwdTiles) ? 4 : 2);
    const int threads = (ppt == 1 || ppt == 2 || ppt == 4) ? tile * tile / ppt : 0;
    if (threads < 32 || threads > 512 || threads % 32 != 0) {
        gs_host::set_error("pixels_per_thread must be 0 (default), 1, 2 or 4, giving 32..512 threads per tile "
                           "(tile 8: 1 or 2; tile 16: 1, 2 or 4; tile 32: 2 or 4)");
        return -1;
    }
    return ppt;
}

// Tile order, longest list first: 256 buckets of the list length (8 per
// octave, descending), one block. Order inside a bucket is arbitrary; it only
// affects scheduling, never results.
// Longest-first bucket of a work key: 8 buckets per power of two, descending.
__device__ __forceinline__ int order_bucket(uint32_t len)
{
    const uint32_t x = len + 1u;
    const int e = 31 - __clz(x);
    const int m = (int)((x >> (e > 3 ? e - 3 : 0)) << (e > 3 ? 0 : 3 - e)) & 7;
    return 255 - min(255, e * 8 + m);
}

__device__ __forceinline__ uint2 batch_range(const Batch& b, int gt)
{
    const ViewDev& V = b.v[view_of_tile(b, gt)];
    return V.ranges[bin_tile_of(V.dil, gt - V.tile_begin)];
}

// Exclusive prefix sums of the 256 bucket counts in s_hist, into s_off (the
// first 256 threads of a 1024-thread CTA; s_w: 9 words of scratch).
__device__ __forceinline__ void scan_buckets(const uint32_t* s_hist, uint32_t* s_off, uint32_t* s_w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = 0, inc = 0;
    if (threadIdx.x < 256) {
        x = s_hist[threadIdx.x];
        inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = s_w[w];
            s_w[w] = run;
            run += c;
        }
    }
    __syncthreads();
    if (threadIdx.x < 256) s_off[threadIdx.x] = s_w[warp] + inc - x;
    __syncthreads();
}

// Longest-first order of T tiles from their buckets (s_b, one byte per tile,
// in shared memory): counts, prefix sums, then each tile takes the next slot
// of its bucket. Slots within a bucket go in no particular order.
__device__ __forceinline__ void order_from_buckets(int T, const uint8_t* s_b, uint32_t* __restrict__ order)
{
    __shared__ uint32_t s_hist[256];
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_w[9];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) atomicAdd(&s_hist[s_b[t]], 1u);
    __syncthreads();
    scan_buckets(s_hist, s_off, s_w);
    for (int t = threadIdx.x; t < T; t += blockDim.x) order[atomicAdd(&s_off[s_b[t]], 1u)] = (uint32_t)t;
}

// Longest-first order by list length (of the binning tile's list), one CTA:
// the buckets are computed once into dynamic shared memory (T bytes).
__global__ void __launch_bounds__(1024) k_tile_order(const __grid_constant__ Batch b, uint32_t* __restrict__ order)
{
    kernel_prologue();
    extern __shared__ uint8_t s_bkt[];
    const int T = b.total_tiles;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const uint2 r = batch_range(b, t);
        s_bkt[t] = (uint8_t)order_bucket(r.y - r.x);
    }
    __syncthreads();
    order_from_buckets(T, s_bkt, order);
}

// Backward work key of every blend tile of the batch: the largest `last` over
// its pixels (the list positions its backward replays), one warp per tile,
// written to key[global tile].
__global__ void __launch_bounds__(256) k_tile_last_max(const __grid_constant__ Batch b, uint32_t* __restrict__ key)
{
    kernel_prologue();
    const int gt = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (gt >= b.total_tiles) return;  // uniform over the warp
    const ViewDev& V = b.v[view_of_tile(b, gt)];
    const int t = gt - V.tile_begin, T = V.dil.tile;
    const int tx = t % V.dil.tiles_x, ty = t / V.dil.tiles_x;
    const int u0 = tx * T, v0 = ty * T;
    const int w = min(T, V.dil.w_ds - u0), h = min(T, V.dil.h_ds - v0);
    uint32_t m = 0u;
    for (int i = lane; i < w * h; i += 32) {
        const int du = i % w, dv = i / w;
        m = max(m, V.last[(int64_t)(v0 + dv) * V.dil.w_ds + u0 + du]);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0) key[gt] = m;
}

// Longest-first order of the tiles by the keys in `order` (read into shared
// memory first, then overwritten by the order). One CTA; T keys fit in
// its dynamic shared memory.
// The same order for more tiles than shared memory holds buckets for: the
// buckets are recomputed from global memory in both passes.
__global__ void __launch_bounds__(1024) k_tile_order_global(const __grid_constant__ Batch b,
                                                            uint32_t* __restrict__ order)
{
    kernel_prologue();
    const int T = b.total_tiles;
    __shared__ uint32_t s_hist[256];
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_w[9];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const uint2 r = batch_range(b, t);
        atomicAdd(&s_hist[order_bucket(r.y - r.x)], 1u);
    }
    __syncthreads();
    scan_buckets(s_hist, s_off, s_w);
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const uint2 r = batch_range(b, t);
        order[atomicAdd(&s_off[order_bucket(r.y - r.x)], 1u)] = (uint32_t)t;
    }
}

__global__ void __launch_bounds__(1024) k_tile_order_keys(int T, uint32_t* __restrict__ order)
{
    kernel_prologue();
    extern __shared__ uint8_t s_bkt[];
    for (int t = threadIdx.x; t < T; t += blockDim.x) s_bkt[t] = (uint8_t)order_bucket(order[t]);
    __syncthreads();
    order_from_buckets(T, s_bkt, order);
}

constexpr int kMaxKeyedOrderTiles = 192 * 1024;  // one bucket byte per tile in shared memory

// Longest-first order by list length, in shared memory when the buckets fit.
int32_t launch_tile_order(const Batch& b, uint32_t* order, cudaStream_t st, const char* what)
{
    const int T = b.total_tiles;
    if (T <= kMaxKeyedOrderTiles) {
        if (T > 48 * 1024) cudaFuncSetAttribute(k_tile_order, cudaFuncAttributeMaxDynamicSharedMemorySize, T);
        gs::launch(k_tile_order, 1, 1024, (size_t)T, st, b, order);
    } else {
        gs::launch(k_tile_order_global, 1, 1024, 0, st, b, order);
    }
    return gs_host::check_launch(what);
}

bool check_render_view(int32_t n, const ViewDev& v)
{
    if (!v.ranges || (n > 0 && (!v.splats || !v.ids))) {
        gs_host::set_error("render: null splats, sorted_ids or ranges");
        return false;
    }
    if ((reinterpret_cast<uintptr_t>(v.splats) & 15) != 0 || (reinterpret_cast<uintptr_t>(v.ranges) & 7) != 0) {
        gs_host::set_error("splats must be 16-byte and ranges 8-byte aligned");
        return false;
    }
    return true;
}

bool any_shift(const Batch& b)
{
    for (int i = 0; i < b.nviews; ++i)
        if (b.v[i].dil.shift > 0) return true;
    return false;
}

template <int TILE, int PPT>
void launch_fwd(const Batch& b, const uint32_t* order, float3 bg, unsigned long long* counts, int n, uint32_t flags,
                cudaStream_t st)
{
    const bool multi = b.nviews > 1, filter = any_shift(b);
    auto kern = counts != nullptr
        ? (multi ? (filter ? k_render_fwd<TILE, PPT, true, true, true> : k_render_fwd<TILE, PPT, true, false, true>)
                 : (filter ? k_render_fwd<TILE, PPT, false, true, true> : k_render_fwd<TILE, PPT, false, false, true>))
        : (multi ? (filter ? k_render_fwd<TILE, PPT, true, true, false> : k_render_fwd<TILE, PPT, true, false, false>)
                 : (filter ? k_render_fwd<TILE, PPT, false, true, false>
                           : k_render_fwd<TILE, PPT, false, false, false>));
    gs::launch(kern, b.total_tiles, TileGeom<TILE, PPT>::THREADS, 0, st, b, order, bg, counts, n, flags);
}

template <int TILE, int PPT>
void launch_bwd(const Batch& b, const uint32_t* order, float3 bg, cudaStream_t st)
{
    const bool multi = b.nviews > 1, filter = any_shift(b);
    auto kern = multi ? (filter ? k_render_bwd<TILE, PPT, true, true> : k_render_bwd<TILE, PPT, true, false>)
                      : (filter ? k_render_bwd<TILE, PPT, false, true> : k_render_bwd<TILE, PPT, false, false>);
    gs::launch(kern, b.total_tiles, TileGeom<TILE, PPT>::THREADS, 0, st, b, order, bg);
}

// The instantiated (tile, pixels per thread) pairs.
#define GS_TILE_SWITCH(tile, ppt, FN, ...)                \
    switch ((tile) * 8 + (ppt)) {                         \
        case 8 * 8 + 1: FN<8, 1>(__VA_ARGS__); break;     \
        case 8 * 8 + 2: FN<8, 2>(__VA_ARGS__); break;     \
        case 16 * 8 + 1: FN<16, 1>(__VA_ARGS__); break;   \
        case 16 * 8 + 2: FN<16, 2>(__VA_ARGS__); break;   \
        case 16 * 8 + 4: FN<16, 4>(__VA_ARGS__); break;   \
        case 32 * 8 + 2: FN<32, 2>(__VA_ARGS__); break;   \
        default: FN<32, 4>(__VA_ARGS__); break;           \
    }

GsView single_view(const GsCamera* cam, const GsDilation* dil)
{
    GsView v{};
    v.cam = *cam;
    v.dil = *dil;
    return v;
}

}  // namespace
}  // namespace gs

extern "C" {

int32_t gs_render_fwd(int32_t n, const float* splats, const uint32_t* sorted_ids, const uint32_t* ranges,
                      const GsCamera* cam, const GsDilation* dil, const float* bg, float* img, float* t_final,
                      uint32_t* last, unsigned long long* counts, int32_t pixels_per_thread,
                      const uint32_t* tile_order, gs_stream_t stream)
{
    if (!cam || !dil) { gs_host::set_error("gs_render_fwd: camera or dilation is null"); return GS_ERR_ARG; }
    GsView v = gs::single_view(cam, dil);
    v.splats = const_cast<float*>(splats);
    v.sorted_ids = const_cast<uint32_t*>(sorted_ids);
    v.ranges = const_cast<uint32_t*>(ranges);
    v.img = img;
    v.t_final = t_final;
    v.last = last;
    return gs_render_fwd_batch(n, &v, 1, bg, tile_order, counts, pixels_per_thread, 0, stream);
}

int32_t gs_render_fwd_l1(int32_t n, const float* splats, const uint32_t* sorted_ids, const uint32_t* ranges,
                         const GsCamera* cam, const GsDilation* dil, const float* bg, float* img, float* t_final,
                         uint32_t* last, const void* target, int32_t target_dtype, float* dl_dimg, float* loss,
                         float* grad2d_zero, unsigned long long* counts, int32_t pixels_per_thread,
                         const uint32_t* tile_order, gs_stream_t stream)
{
    if (!cam || !dil) { gs_host::set_error("gs_render_fwd_l1: camera or dilation is null"); return GS_ERR_ARG; }
    GsView v = gs::single_view(cam, dil);
    v.splats = const_cast<float*>(splats);
    v.sorted_ids = const_cast<uint32_t*>(sorted_ids);
    v.ranges = const_cast<uint32_t*>(ranges);
    v.img = img;
    v.t_final = t_final;
    v.last = last;
    v.target = target;
    v.target_dtype = target_dtype;
    v.dl_dimg = dl_dimg;
    v.loss = loss;
    v.grad2d = grad2d_zero;
    const int32_t flags = GS_FWD_L1 | (grad2d_zero ? GS_FWD_ZERO_GRAD2D : 0);
    return gs_render_fwd_batch(n, &v, 1, bg, tile_order, counts, pixels_per_thread, flags, stream);
}

int32_t gs_render_fwd_batch(int32_t n, const GsView* views, int32_t nviews, const float* bg,
                            const uint32_t* tile_order, unsigned long long* counts, int32_t pixels_per_thread,
                            int32_t flags, gs_stream_t stream)
{
    using namespace gs;
    if (n < 0) { gs_host::set_error("n must be >= 0"); return GS_ERR_ARG; }
    Batch b;
    if (!gs_host::make_batch(views, nviews, &b)) return GS_ERR_ARG;
    for (int i = 0; i < nviews; ++i) {
        if (!check_render_view(n, b.v[i])) return GS_ERR_ARG;
        if (!b.v[i].img || !b.v[i].t_final || !b.v[i].last) {
            gs_host::set_error("gs_render_fwd: null img, t_final or last");
            return GS_ERR_ARG;
        }
    }
    if (!bg) { gs_host::set_error("gs_render_fwd: bg is null"); return GS_ERR_ARG; }
    if ((flags & ~(GS_FWD_L1 | GS_FWD_ZERO_GRAD2D)) != 0) {
        gs_host::set_error("gs_render_fwd: unknown flags");
        return GS_ERR_ARG;
    }
    for (int i = 0; i < nviews; ++i) {
        const ViewDev& v = b.v[i];
        if ((flags & GS_FWD_L1) && (!v.target || !v.dl || !v.loss)) {
            gs_host::set_error("gs_render_fwd: the fused loss needs target, dl_dimg and loss");
            return GS_ERR_ARG;
        }
        if ((flags & GS_FWD_ZERO_GRAD2D) && n > 0 &&
            (!v.grad2d || (reinterpret_cast<uintptr_t>(v.grad2d) & 15) != 0)) {
            gs_host::set_error("gs_render_fwd: zeroing needs a 16-byte aligned grad2d");
            return GS_ERR_ARG;
        }
    }
    const int ppt = resolve_ppt(b.v[0].dil.tile, pixels_per_thread, false, b.total_tiles);
    if (ppt < 0) return GS_ERR_ARG;
    const float3 c = make_float3(bg[0], bg[1], bg[2]);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (flags & GS_FWD_L1) gs::launch(k_loss_zero, 1, 32, 0, st, b);
    GS_TILE_SWITCH(b.v[0].dil.tile, ppt, launch_fwd, b, tile_order, c, counts, n, (uint32_t)flags, st);
    return gs_host::check_launch("gs_render_fwd");
}

int32_t gs_render_bwd(int32_t n, const float* splats, const uint32_t* sorted_ids, const uint32_t* ranges,
                      const GsCamera* cam, const GsDilation* dil, const float* bg, const float* t_final,
                      const uint32_t* last, const float* dl_dimg, float* grad2d, int32_t zero_grad2d,
                      int32_t pixels_per_thread, const uint32_t* tile_order, gs_stream_t stream)
{
    if (!cam || !dil) { gs_host::set_error("gs_render_bwd: camera or dilation is null"); return GS_ERR_ARG; }
    GsView v = gs::single_view(cam, dil);
    v.splats = const_cast<float*>(splats);
    v.sorted_ids = const_cast<uint32_t*>(sorted_ids);
    v.ranges = const_cast<uint32_t*>(ranges);
    v.t_final = const_cast<float*>(t_final);
    v.last = const_cast<uint32_t*>(last);
    v.dl_dimg = const_cast<float*>(dl_dimg);
    v.grad2d = grad2d;
    return gs_render_bwd_batch(n, &v, 1, bg, tile_order, zero_grad2d, pixels_per_thread, stream);
}

int32_t gs_render_bwd_batch(int32_t n, const GsView* views, int32_t nviews, const float* bg,
                            const uint32_t* tile_order, int32_t zero_grad2d, int32_t pixels_per_thread,
                            gs_stream_t stream)
{
    using namespace gs;
    if (n < 0) { gs_host::set_error("n must be >= 0"); return GS_ERR_ARG; }
    Batch b;
    if (!gs_host::make_batch(views, nviews, &b)) return GS_ERR_ARG;
    for (int i = 0; i < nviews; ++i) {
        const ViewDev& v = b.v[i];
        if (!check_render_view(n, v)) return GS_ERR_ARG;
        if (!v.t_final || !v.last || !v.dl || (n > 0 && !v.grad2d)) {
            gs_host::set_error("gs_render_bwd: null t_final, last, dl_dimg or grad2d");
            return GS_ERR_ARG;
        }
        if ((reinterpret_cast<uintptr_t>(v.grad2d) & 15) != 0) {
            gs_host::set_error("gs_render_bwd: grad2d must be 16-byte aligned");
            return GS_ERR_ARG;
        }
    }
    if (!bg) { gs_host::set_error("gs_render_bwd: bg is null"); return GS_ERR_ARG; }
    const int ppt = resolve_ppt(b.v[0].dil.tile, pixels_per_thread, true, b.total_tiles);
    if (ppt < 0) return GS_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (zero_grad2d && n > 0)
        for (int i = 0; i < nviews; ++i)
            cudaMemsetAsync(b.v[i].grad2d, 0, (size_t)n * GS_GRAD2D_FLOATS * sizeof(float), st);
    const float3 c = make_float3(bg[0], bg[1], bg[2]);
    GS_TILE_SWITCH(b.v[0].dil.tile, ppt, launch_bwd, b, tile_order, c, st);
    return gs_host::check_launch("gs_render_bwd");
}

int32_t gs_tile_order(const uint32_t* ranges, int32_t num_tiles, uint32_t* order, gs_stream_t stream)
{
    using namespace gs;
    if (num_tiles < 0 || (num_tiles > 0 && (!ranges || !order))) {
        gs_host::set_error("gs_tile_order: bad arguments");
        return GS_ERR_ARG;
    }
    if (num_tiles == 0) return GS_OK;
    Batch b{};
    b.nviews = 1;
    b.v[0].ranges = reinterpret_cast<const uint2*>(ranges);
    // one row of num_tiles blend tiles, each its own binning tile
    b.v[0].dil.tiles_x = b.v[0].dil.bin_tiles_x = num_tiles;
    b.v[0].dil.tiles_y = b.v[0].dil.bin_tiles_y = 1;
    b.total_tiles = num_tiles;
    return launch_tile_order(b, order, reinterpret_cast<cudaStream_t>(stream), "gs_tile_order");
}

int32_t gs_tile_order_batch(const GsView* views, int32_t nviews, uint32_t* order, gs_stream_t stream)
{
    using namespace gs;
    Batch b;
    if (!gs_host::make_batch(views, nviews, &b)) return GS_ERR_ARG;
    for (int i = 0; i < nviews; ++i)
        if (!b.v[i].ranges) { gs_host::set_error("gs_tile_order_batch: null ranges"); return GS_ERR_ARG; }
    if (!order) { gs_host::set_error("gs_tile_order_batch: order is null"); return GS_ERR_ARG; }
    return launch_tile_order(b, order, reinterpret_cast<cudaStream_t>(stream), "gs_tile_order_batch");
}

int32_t gs_tile_order_by_last_batch(const GsView* views, int32_t nviews, uint32_t* order, gs_stream_t stream)
{
    using namespace gs;
    Batch b;
    if (!gs_host::make_batch(views, nviews, &b)) return GS_ERR_ARG;
    for (int i = 0; i < nviews; ++i)
        if (!b.v[i].last) {
            gs_host::set_error("gs_tile_order_by_last_batch: null last");
            return GS_ERR_ARG;
        }
    if (!order) { gs_host::set_error("gs_tile_order_by_last_batch: order is null"); return GS_ERR_ARG; }
    const int T = b.total_tiles;
    if (T == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (T > kMaxKeyedOrderTiles)  // more tiles than shared memory holds buckets for: the list-length order
        return launch_tile_order(b, order, st, "gs_tile_order_by_last_batch");
    gs::launch(k_tile_last_max, (int)(((int64_t)T * 32 + 255) / 256), 256, 0, st, b, order);
    if (T > 48 * 1024) cudaFuncSetAttribute(k_tile_order_keys, cudaFuncAttributeMaxDynamicSharedMemorySize, T);
    gs::launch(k_tile_order_keys, 1, 1024, (size_t)T, st, T, order);
    return gs_host::check_launch("gs_tile_order_by_last_batch");
}

int32_t gs_loss_l1(const GsCamera* cam, const GsDilation* dil, const float* img, const void* target,
                   int32_t target_dtype, float* dl_dimg, float* loss, gs_stream_t stream)
{
    if (!cam || !dil) { gs_host::set_error("gs_loss_l1: camera or dilation is null"); return GS_ERR_ARG; }
    GsView v = gs::single_view(cam, dil);
    v.img = const_cast<float*>(img);
    v.target = target;
    v.target_dtype = target_dtype;
    v.dl_dimg = dl_dimg;
    v.loss = loss;
    return gs_loss_l1_batch(&v, 1, stream);
}

int32_t gs_loss_l1_batch(const GsView* views, int32_t nviews, gs_stream_t stream)
{
    using namespace gs;
    Batch b;
    if (!gs_host::make_batch(views, nviews, &b)) return GS_ERR_ARG;
    int64_t pmax = 0;
    for (int i = 0; i < nviews; ++i) {
        const ViewDev& v = b.v[i];
        if (!v.img || !v.target || !v.dl || !v.loss) {
            gs_host::set_error("gs_loss_l1: null img, target, dl_dimg or loss");
            return GS_ERR_ARG;
        }
        const int64_t P = (int64_t)v.dil.w_ds * v.dil.h_ds;
        if (P > pmax) pmax = P;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    gs::launch(k_loss_zero, 1, 32, 0, st, b);
    int64_t bx = (pmax + 255) / 256;
    const int64_t cap = ((int64_t)gs_host::sm_count() * 16 + nviews - 1) / nviews;
    if (bx > cap) bx = cap;
    gs::launch(k_loss_l1, dim3((unsigned)bx, (unsigned)nviews), 256, 0, st, b);
    return gs_host::check_launch("gs_loss_l1");
}

}  // extern "C"
