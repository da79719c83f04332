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

struct SplatStage {
    float2 p;   // centre relative to the tile's hr origin
    float4 co;  // conic A, B, C, opacity
    float4 rgb;
};

__device__ __forceinline__ void load_stage(const float4* __restrict__ splats, uint32_t g, float X0, float Y0,
                                           float2& p, float4& co, float4& rgb)
{
    const float4 v0 = __ldg(splats + 3 * (int64_t)g);
    const float4 v1 = __ldg(splats + 3 * (int64_t)g + 1);
    const float4 v2 = __ldg(splats + 3 * (int64_t)g + 2);
    p.x = __fadd_rn(__fsub_rn(v0.x, X0), v2.z);
    p.y = __fadd_rn(__fsub_rn(v0.y, Y0), v2.w);
    co = make_float4(v0.z, v0.w, v1.x, v1.y);
    rgb = make_float4(v1.z, v1.w, v2.x, 0.0f);
}

template <int TILE>
__global__ void __launch_bounds__(TILE * TILE)
k_render_fwd(const float4* __restrict__ splats, const uint32_t* __restrict__ ids, const uint2* __restrict__ ranges,
             Dil dil, float3 bg, float* __restrict__ img, float* __restrict__ t_final, uint32_t* __restrict__ last,
             unsigned long long* __restrict__ counts)
{
    constexpr int BLOCK = TILE * TILE;
    constexpr int BATCH = BLOCK < 256 ? BLOCK : 256;
    __shared__ float2 s_p[BATCH];
    __shared__ float4 s_co[BATCH];
    __shared__ float4 s_rgb[BATCH];
    __shared__ unsigned long long s_cnt[2];

    const int tile = blockIdx.x;
    const int tx = tile % dil.tiles_x, ty = tile / dil.tiles_x;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int u = tx * TILE + lx, v = ty * TILE + ly;
    const bool inside = u < dil.w_ds && v < dil.h_ds;
    // hr origin of the tile and this pixel's hr offset from it (small exact floats)
    const float X0 = (float)(dil.d * tx * TILE + dil.ox), Y0 = (float)(dil.d * ty * TILE + dil.oy);
    const float xr = (float)(dil.d * lx), yr = (float)(dil.d * ly);

    if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0ull;
    const uint2 rg = ranges[tile];
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last_pos = 0, n_eval = 0, n_blend = 0;
    bool done = !inside;

    for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
        if (__syncthreads_count(done) == BLOCK) break;
        const uint32_t idx = start + threadIdx.x;
        if ((int)threadIdx.x < BATCH && idx < rg.y) {
            float2 p; float4 co, rgb;
            load_stage(splats, __ldg(ids + idx), X0, Y0, p, co, rgb);
            s_p[threadIdx.x] = p;
            s_co[threadIdx.x] = co;
            s_rgb[threadIdx.x] = rgb;
        }
        __syncthreads();
        if (!done) {
            const int cnt = (int)((rg.y - start) < (uint32_t)BATCH ? (rg.y - start) : (uint32_t)BATCH);
            for (int j = 0; j < cnt; ++j) {
                ++n_eval;
                const float2 p = s_p[j];
                const float4 co = s_co[j];
                const float dx = __fsub_rn(xr, p.x), dy = __fsub_rn(yr, p.y);
                const float power = splat_power(dx, dy, co.x, co.y, co.z);
                if (power > 0.0f) continue;
                const float alpha = fminf(kAlphaMax, splat_alpha_raw(power, co.w));
                if (alpha < kAlphaMin) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < kTStop) { done = true; break; }
                const float4 c = s_rgb[j];
                const float w = alpha * T;
                C0 = fmaf(c.x, w, C0);
                C1 = fmaf(c.y, w, C1);
                C2 = fmaf(c.z, w, C2);
                T = Tn;
                last_pos = start + j - rg.x + 1;
                ++n_blend;
            }
        }
    }
    if (inside) {
        const int64_t pix = (int64_t)v * dil.w_ds + u;
        img[3 * pix] = fmaf(T, bg.x, C0);
        img[3 * pix + 1] = fmaf(T, bg.y, C1);
        img[3 * pix + 2] = fmaf(T, bg.z, C2);
        t_final[pix] = T;
        last[pix] = last_pos;
    }
    if (counts != nullptr) {
        unsigned long long e = n_eval, b = n_blend;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_down_sync(0xffffffffu, e, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&s_cnt[0], e);
            atomicAdd(&s_cnt[1], b);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&counts[0], s_cnt[0]);
            atomicAdd(&counts[1], s_cnt[1]);
        }
    }
}

// Backward: replay each pixel's list back to front from (t_final, last),
// recovering T_i = T_{i+1} / (1 - alpha_i). Per list entry the 32 lanes of a
// warp evaluate the same Gaussian; their 9 partial gradients are summed with
// xor shuffles, folded into a per-batch shared-memory accumulator (9 lanes,
// one component each), and flushed with one set of vector atomics per
// (tile, Gaussian) at the end of the batch.
template <int TILE>
__global__ void __launch_bounds__(TILE * TILE)
k_render_bwd(const float4* __restrict__ splats, const uint32_t* __restrict__ ids, const uint2* __restrict__ ranges,
             Dil dil, float3 bg, const float* __restrict__ t_final, const uint32_t* __restrict__ last,
             const float* __restrict__ dl_dimg, float* __restrict__ grad2d)
{
    constexpr int BLOCK = TILE * TILE;
    constexpr int BATCH = BLOCK < 256 ? BLOCK : 256;
    __shared__ float2 s_p[BATCH];
    __shared__ float4 s_co[BATCH];
    __shared__ float4 s_rgb[BATCH];
    __shared__ uint32_t s_id[BATCH];
    __shared__ float s_acc[BATCH][9];
    __shared__ uint32_t s_max_last;

    const int tile = blockIdx.x;
    const int tx = tile % dil.tiles_x, ty = tile / dil.tiles_x;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    const int lane = threadIdx.x & 31;
    const int u = tx * TILE + lx, v = ty * TILE + ly;
    const bool inside = u < dil.w_ds && v < dil.h_ds;
    const float X0 = (float)(dil.d * tx * TILE + dil.ox), Y0 = (float)(dil.d * ty * TILE + dil.oy);
    const float xr = (float)(dil.d * lx), yr = (float)(dil.d * ly);
    const uint2 rg = ranges[tile];

    float T = 1.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    uint32_t n_last = 0;
    if (inside) {
        const int64_t pix = (int64_t)v * dil.w_ds + u;
        T = t_final[pix];
        n_last = last[pix];
        g0 = dl_dimg[3 * pix];
        g1 = dl_dimg[3 * pix + 1];
        g2 = dl_dimg[3 * pix + 2];
    }
    float S0 = T * bg.x, S1 = T * bg.y, S2 = T * bg.z;
    if (threadIdx.x == 0) s_max_last = 0;
    __syncthreads();
    if (n_last > 0) atomicMax(&s_max_last, n_last);
    __syncthreads();
    const uint32_t n_proc = s_max_last;
    if (n_proc == 0) return;

    for (int b = (int)((n_proc - 1) / BATCH); b >= 0; --b) {
        const uint32_t bstart = (uint32_t)b * BATCH;
        const int cnt = (int)((n_proc - bstart) < (uint32_t)BATCH ? (n_proc - bstart) : (uint32_t)BATCH);
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const uint32_t g = __ldg(ids + rg.x + bstart + threadIdx.x);
            float2 p; float4 co, rgb;
            load_stage(splats, g, X0, Y0, p, co, rgb);
            s_p[threadIdx.x] = p;
            s_co[threadIdx.x] = co;
            s_rgb[threadIdx.x] = rgb;
            s_id[threadIdx.x] = g;
#pragma unroll
            for (int k = 0; k < 9; ++k) s_acc[threadIdx.x][k] = 0.0f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const uint32_t pos = bstart + (uint32_t)j;
            float r[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) r[k] = 0.0f;
            bool contrib = false;
            if (pos < n_last) {
                const float2 p = s_p[j];
                const float4 co = s_co[j];
                const float dx = __fsub_rn(xr, p.x), dy = __fsub_rn(yr, p.y);
                const float power = splat_power(dx, dy, co.x, co.y, co.z);
                if (power <= 0.0f) {
                    const float G = __expf(power);
                    const float a_raw = __fmul_rn(co.w, G);  // as splat_alpha_raw
                    const float alpha = fminf(kAlphaMax, a_raw);
                    if (alpha >= kAlphaMin) {
                        contrib = true;
                        const float4 c = s_rgb[j];
                        const float one_m = 1.0f - alpha;
                        const float Ti = T / one_m;
                        const float w = alpha * Ti;
                        r[6] = w * g0;
                        r[7] = w * g1;
                        r[8] = w * g2;
                        const float inv = 1.0f / one_m;
                        const float dalpha = g0 * (Ti * c.x - S0 * inv) + g1 * (Ti * c.y - S1 * inv) +
                                             g2 * (Ti * c.z - S2 * inv);
                        S0 = fmaf(c.x, w, S0);
                        S1 = fmaf(c.y, w, S1);
                        S2 = fmaf(c.z, w, S2);
                        T = Ti;
                        if (a_raw < kAlphaMax) {
                            const float dpower = a_raw * dalpha;
                            r[5] = G * dalpha;
                            r[2] = -0.5f * dx * dx * dpower;
                            r[3] = -dx * dy * dpower;
                            r[4] = -0.5f * dy * dy * dpower;
                            r[0] = dpower * (co.x * dx + co.y * dy);
                            r[1] = dpower * (co.z * dy + co.y * dx);
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int k = 0; k < 9; ++k) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) r[k] += __shfl_xor_sync(0xffffffffu, r[k], o);
                }
                float mine = r[0];
#pragma unroll
                for (int k = 1; k < 9; ++k)
                    if (lane == k) mine = r[k];
                if (lane < 9) atomicAdd(&s_acc[j][lane], mine);
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const float* a = s_acc[threadIdx.x];
            bool any = false;
#pragma unroll
            for (int k = 0; k < 9; ++k) any |= (a[k] != 0.0f);
            if (any) {
                float* dst = grad2d + (int64_t)GS_GRAD2D_FLOATS * s_id[threadIdx.x];
                atomicAdd(reinterpret_cast<float4*>(dst), make_float4(a[0], a[1], a[2], a[3]));
                atomicAdd(reinterpret_cast<float4*>(dst + 4), make_float4(a[4], a[5], a[6], a[7]));
                atomicAdd(dst + 8, a[8]);
            }
        }
    }
}

__global__ void k_loss_l1(Dil dil, int width, const float* __restrict__ img, const float* __restrict__ target,
                          float* __restrict__ dl, float* __restrict__ loss, float inv)
{
    const int64_t P = (int64_t)dil.w_ds * dil.h_ds;
    float acc = 0.0f;
    for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < P;
         pix += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(pix % dil.w_ds), v = (int)(pix / dil.w_ds);
        const int64_t h = ((int64_t)(dil.d * v + dil.oy) * width + (dil.d * u + dil.ox)) * 3;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float r = img[3 * pix + ch] - target[h + ch];
            acc += fabsf(r);
            dl[3 * pix + ch] = r > 0.0f ? inv : (r < 0.0f ? -inv : 0.0f);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ float s_sum[32];
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_sum[w];
        atomicAdd(loss, t * inv);
    }
}

bool check_render_args(int32_t n, const float* splats, const uint32_t* ids, const uint32_t* ranges)
{
    if (n < 0) { gs_host::set_error("n must be >= 0"); return false; }
    if (!ranges || (n > 0 && (!splats || !ids))) { gs_host::set_error("null pointer"); return false; }
    if ((reinterpret_cast<uintptr_t>(splats) & 15) != 0 || (reinterpret_cast<uintptr_t>(ranges) & 7) != 0) {
        gs_host::set_error("splats must be 16-byte and ranges 8-byte aligned");
        return false;
    }
    return true;
}

}  // namespace
}  // namespace gs

extern "C" {

int32_t gs_render_fwd(int32_t n, const float* splats, const uint32_t* sorted_ids, const uint32_t* ranges,
                      const GsCamera* cam, const GsDilation* dil, const float* bg, float* img, float* t_final,
                      uint32_t* last, unsigned long long* counts, gs_stream_t stream)
{
    using namespace gs;
    Dil d;
    if (!gs_host::make_dil(cam, dil, &d)) return GS_ERR_ARG;
    if (!check_render_args(n, splats, sorted_ids, ranges)) return GS_ERR_ARG;
    if (!bg || !img || !t_final || !last) { gs_host::set_error("gs_render_fwd: null pointer"); return GS_ERR_ARG; }
    const float3 b = make_float3(bg[0], bg[1], bg[2]);
    const int tiles = d.tiles_x * d.tiles_y;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float4* sp = reinterpret_cast<const float4*>(splats);
    const uint2* rg = reinterpret_cast<const uint2*>(ranges);
    switch (d.tile) {
        case 8: k_render_fwd<8><<<tiles, 64, 0, st>>>(sp, sorted_ids, rg, d, b, img, t_final, last, counts); break;
        case 16: k_render_fwd<16><<<tiles, 256, 0, st>>>(sp, sorted_ids, rg, d, b, img, t_final, last, counts); break;
        default: k_render_fwd<32><<<tiles, 1024, 0, st>>>(sp, sorted_ids, rg, d, b, img, t_final, last, counts); break;
    }
    return gs_host::check_launch("gs_render_fwd");
}

int32_t gs_render_bwd(int32_t n, const float* splats, const uint32_t* sorted_ids, const uint32_t* ranges,
                      const GsCamera* cam, const GsDilation* dil, const float* bg, const float* t_final,
                      const uint32_t* last, const float* dl_dimg, float* grad2d, int32_t zero_grad2d,
                      gs_stream_t stream)
{
    using namespace gs;
    Dil d;
    if (!gs_host::make_dil(cam, dil, &d)) return GS_ERR_ARG;
    if (!check_render_args(n, splats, sorted_ids, ranges)) return GS_ERR_ARG;
    if (!bg || !t_final || !last || !dl_dimg || (n > 0 && !grad2d)) {
        gs_host::set_error("gs_render_bwd: null pointer");
        return GS_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(grad2d) & 15) != 0) {
        gs_host::set_error("gs_render_bwd: grad2d must be 16-byte aligned");
        return GS_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (zero_grad2d && n > 0) cudaMemsetAsync(grad2d, 0, (size_t)n * GS_GRAD2D_FLOATS * sizeof(float), st);
    const float3 b = make_float3(bg[0], bg[1], bg[2]);
    const int tiles = d.tiles_x * d.tiles_y;
    const float4* sp = reinterpret_cast<const float4*>(splats);
    const uint2* rg = reinterpret_cast<const uint2*>(ranges);
    switch (d.tile) {
        case 8: k_render_bwd<8><<<tiles, 64, 0, st>>>(sp, sorted_ids, rg, d, b, t_final, last, dl_dimg, grad2d); break;
        case 16: k_render_bwd<16><<<tiles, 256, 0, st>>>(sp, sorted_ids, rg, d, b, t_final, last, dl_dimg, grad2d); break;
        default: k_render_bwd<32><<<tiles, 1024, 0, st>>>(sp, sorted_ids, rg, d, b, t_final, last, dl_dimg, grad2d); break;
    }
    return gs_host::check_launch("gs_render_bwd");
}

int32_t gs_loss_l1(const GsCamera* cam, const GsDilation* dil, const float* img, const float* target, float* dl_dimg,
                   float* loss, gs_stream_t stream)
{
    using namespace gs;
    Dil d;
    if (!gs_host::make_dil(cam, dil, &d)) return GS_ERR_ARG;
    if (!img || !target || !dl_dimg || !loss) { gs_host::set_error("gs_loss_l1: null pointer"); return GS_ERR_ARG; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(loss, 0, sizeof(float), st);
    const int64_t P = (int64_t)d.w_ds * d.h_ds;
    const float inv = (float)(1.0 / (3.0 * (double)P));
    int blocks = (int)((P + 255) / 256);
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_loss_l1<<<blocks, 256, 0, st>>>(d, cam->width, img, target, dl_dimg, loss, inv);
    return gs_host::check_launch("gs_loss_l1");
}

}  // extern "C"
