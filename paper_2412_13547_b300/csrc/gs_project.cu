// gs_project.cu -- projection forward (Sec. 3, Sec. 3.1 EWA + dilated binning
// geometry), its backward, and the densification statistics (Sec. 3.3).
//
// One thread per Gaussian, 4 warps per block. Each warp first copies the rows
// of its 32 Gaussians (means, log-scales and the SH block, which is 192 of the
// 236 bytes per Gaussian at degree 3) from global memory with coalesced 16-byte
// loads into shared memory, padded to an odd row stride so the per-lane reads
// that follow are free of bank conflicts.
#include <cmath>

#include "gs_common.cuh"

namespace gs {
namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;

template <int W>
struct RowStride {
    static constexpr int value = (W % 2 == 0) ? W + 1 : W;
};

// Copy rows [g0, g0+32) of a row-major array of W 32-bit words per row into
// shared memory with row stride S. Full warps use 16-byte loads, all of a lane's
// in flight at once (12 for SH degree 3 in FP32: the fused optimizer pass 3%
// faster than 4 at a time), or 4 at a time with FEW (the batched projection,
// whose registers are taken by the views' loop).
template <int W, int S, bool FEW = false>
__device__ __forceinline__ void warp_stage(const uint32_t* __restrict__ src, int n, int g0,
                                           uint32_t* __restrict__ dst, int lane)
{
    const int rows = min(32, n - g0);
    const uint32_t* base = src + (int64_t)g0 * W;
    if (rows == 32 && (W % 4 == 0 || ((reinterpret_cast<uintptr_t>(base) & 15) == 0))) {
        const uint4* b4 = reinterpret_cast<const uint4*>(base);
        constexpr int KN = (8 * W + 31) / 32;  // vectors per lane, the last one partial when W % 4 != 0
        auto put = [&](int q) {
            const uint4 v = __ldg(b4 + q);
            const int w0 = 4 * q;
            if constexpr (W % 4 == 0 && S % 4 == 0) {
                // 16-byte aligned rows (dst 16-byte aligned): one vector store, conflict-free
                *reinterpret_cast<uint4*>(dst + (w0 / W) * S + w0 % W) = v;
            } else {
                dst[((w0 + 0) / W) * S + (w0 + 0) % W] = v.x;
                dst[((w0 + 1) / W) * S + (w0 + 1) % W] = v.y;
                dst[((w0 + 2) / W) * S + (w0 + 2) % W] = v.z;
                dst[((w0 + 3) / W) * S + (w0 + 3) % W] = v.w;
            }
        };
        if constexpr (FEW) {
#pragma unroll 4
            for (int k = 0; k < KN; ++k)
                if (lane + 32 * k < 8 * W) put(lane + 32 * k);
        } else {
#pragma unroll
            for (int k = 0; k < KN; ++k)
                if (lane + 32 * k < 8 * W) put(lane + 32 * k);
        }
    } else {
        for (int w = lane; w < rows * W; w += 32) dst[(w / W) * S + w % W] = __ldg(base + w);
    }
    __syncwarp();
}

// A lane's row of 3K floats in shared memory (16-byte aligned, 3K a multiple
// of 4) to c, and back, as 16-byte vectors: with a row stride that is a
// multiple of 4 words but not of 32 lanes' worth, 8 lanes' vectors fall on
// distinct banks, so these are conflict-free where per-float accesses to such
// rows would conflict.
template <int K>
__device__ __forceinline__ void row_load_vec(const float* row, float (&c)[16][3])
{
    static_assert((3 * K) % 4 == 0, "whole vectors");
#pragma unroll
    for (int i = 0; i < 3 * K / 4; ++i) {
        const float4 v = reinterpret_cast<const float4*>(row)[i];
        c[(4 * i + 0) / 3][(4 * i + 0) % 3] = v.x;
        c[(4 * i + 1) / 3][(4 * i + 1) % 3] = v.y;
        c[(4 * i + 2) / 3][(4 * i + 2) % 3] = v.z;
        c[(4 * i + 3) / 3][(4 * i + 3) % 3] = v.w;
    }
}

template <int N, bool VEC>
__device__ __forceinline__ void zero_row(float* row)
{
    if constexpr (VEC) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) reinterpret_cast<float4*>(row)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
#pragma unroll
        for (int e = 0; e < N; ++e) row[e] = 0.0f;
    }
}

template <int N>
__device__ __forceinline__ void row_store_vec(float* row, const float* vals)
{
    static_assert(N % 4 == 0, "whole vectors");
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
        reinterpret_cast<float4*>(row)[i] = make_float4(vals[4 * i], vals[4 * i + 1], vals[4 * i + 2], vals[4 * i + 3]);
}

template <int DEG, int DT>
struct ShLayout {
    static constexpr int K = (DEG + 1) * (DEG + 1);
    static constexpr int BYTES = K * 3 * (DT == GS_DTYPE_F32 ? 4 : 2);
    static constexpr bool STAGE = (BYTES % 4) == 0;
    static constexpr int W = STAGE ? BYTES / 4 : 1;
    static constexpr int S = RowStride<W>::value;
    static constexpr int WARP_WORDS = 32 * (3 + 3) + (STAGE ? 32 * S : 0);
};

template <int DEG, int DT, int STRIDE = ShLayout<DEG, DT>::S>
__device__ __forceinline__ void read_sh(const uint32_t* s_sh, const void* sh, int g, int lane,
                                        float (&c)[16][3])
{
    using L = ShLayout<DEG, DT>;
    if constexpr (L::STAGE) {
        const uint32_t* row = s_sh + lane * STRIDE;
        if constexpr (DT == GS_DTYPE_F32 && STRIDE % 4 == 0 && (L::K * 3) % 4 == 0) {
            row_load_vec<L::K>(reinterpret_cast<const float*>(row), c);
        } else if constexpr (DT != GS_DTYPE_F32 && STRIDE % 4 == 0 && L::W % 4 == 0) {
            // 16-bit values, 8 to a 16-byte vector
#pragma unroll
            for (int i = 0; i < L::W / 4; ++i) {
                const uint4 wv = reinterpret_cast<const uint4*>(row)[i];
                const uint32_t w4[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const uint16_t hv = (h & 1) ? (uint16_t)(w4[h >> 1] >> 16) : (uint16_t)(w4[h >> 1] & 0xffffu);
                    float f;
                    if constexpr (DT == GS_DTYPE_BF16) f = __bfloat162float(__ushort_as_bfloat16(hv));
                    else f = __half2float(__ushort_as_half(hv));
                    c[(8 * i + h) / 3][(8 * i + h) % 3] = f;
                }
            }
        } else if constexpr (DT == GS_DTYPE_F32) {
#pragma unroll
            for (int k = 0; k < L::K; ++k)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) c[k][ch] = __uint_as_float(row[3 * k + ch]);
        } else {
#pragma unroll
            for (int e = 0; e < L::K * 3; ++e) {
                uint32_t wv = row[e >> 1];
                uint16_t hv = (e & 1) ? (uint16_t)(wv >> 16) : (uint16_t)(wv & 0xffffu);
                float f;
                if constexpr (DT == GS_DTYPE_BF16) f = __bfloat162float(__ushort_as_bfloat16(hv));
                else f = __half2float(__ushort_as_half(hv));
                c[e / 3][e % 3] = f;
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < L::K * 3; ++e) c[e / 3][e % 3] = load_sh_elem(sh, (int64_t)g * L::K * 3 + e, DT);
    }
}

// Everything the forward projection of one Gaussian computes; the backward
// recomputes it instead of storing it.
struct Proj {
    bool culled;
    float s[3], qn[4], inv_qnorm, R[9], M[9];
    float tz, u, v, uc, vc;
    bool clamp_x, clamp_y;
    float Tm[6], N[6];
    float a, b, c, det, A, B, C;
    int radius;
    ff px, py;
    float dir[3], inv_vlen;
    float rgb_raw[3];
    float opacity;
    int4 rect;   // binning tiles
    int4 frect;  // blend tiles
    int tiles;
};

// View-dependent colour (Sec. 3: SH coefficients): the unit direction from the
// camera centre, its inverse distance and rgb_raw = sum_k Y_k(dir) sh_k + 0.5
// (the colour is max(0, rgb_raw)).
template <int DEG>
__device__ __forceinline__ void sh_colour(const Cam& cam, const float* mean, const float (&sh)[16][3], float* dir,
                                          float& inv_vlen, float* rgb_raw)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    // rounding pinned with intrinsics (as in sh_basis): the colour, and so the clamp of each
    // channel, is the same in the forward and in every backward that recomputes it
    const float vx = __fsub_rn(mean[0], cam.ccx), vy = __fsub_rn(mean[1], cam.ccy), vz = __fsub_rn(mean[2], cam.ccz);
    // a Gaussian at the camera centre (culled: depth 0) gets the zero direction, so that
    // its colour and colour gradients stay finite instead of 0 * inf
    const float len2 = __fmaf_rn(vx, vx, __fmaf_rn(vy, vy, __fmul_rn(vz, vz)));
    inv_vlen = len2 > 0.0f ? rsqrtf(len2) : 0.0f;
    dir[0] = __fmul_rn(vx, inv_vlen); dir[1] = __fmul_rn(vy, inv_vlen); dir[2] = __fmul_rn(vz, inv_vlen);
    float Y[16];
    sh_basis(DEG, dir[0], dir[1], dir[2], Y);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) acc = __fmaf_rn(Y[k], sh[k][ch], acc);
        rgb_raw[ch] = __fadd_rn(acc, 0.5f);
    }
}

// Backward of sh_colour for dL/drgb = grgb (zero where the colour was clamped):
// dL/dsh_k = Y_k grgb into gsh[3k + ch] (written, or added when ACC), and the
// mean's gradient through the direction into gm.
template <int DEG, bool ACC, bool VEC = false>
__device__ __forceinline__ void sh_colour_bwd(const float* dir, float inv_vlen, const float* rgb_raw,
                                              const float (&c)[16][3], float g0, float g1, float g2, float* gsh,
                                              float* gm)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float grgb[3] = {rgb_raw[0] > 0.0f ? g0 : 0.0f, rgb_raw[1] > 0.0f ? g1 : 0.0f,
                           rgb_raw[2] > 0.0f ? g2 : 0.0f};
    float Y[16];
    sh_basis(DEG, dir[0], dir[1], dir[2], Y);
    float wsh[16];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        wsh[k] = grgb[0] * c[k][0] + grgb[1] * c[k][1] + grgb[2] * c[k][2];
        if constexpr (!VEC) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
                gsh[3 * k + ch] = ACC ? gsh[3 * k + ch] + Y[k] * grgb[ch] : Y[k] * grgb[ch];
        }
    }
    if constexpr (VEC) {
        // a 16-byte aligned row of 3K floats (3K a multiple of 4), written as vectors
        static_assert(!ACC, "the vector form writes");
        float gv[48];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gv[3 * k + ch] = Y[k] * grgb[ch];
        row_store_vec<3 * K>(gsh, gv);
    }
    float gdx, gdy, gdz;
    sh_basis_vjp(DEG, dir[0], dir[1], dir[2], wsh, gdx, gdy, gdz);
    const float dd = gdx * dir[0] + gdy * dir[1] + gdz * dir[2];
    gm[0] = (gdx - dir[0] * dd) * inv_vlen;
    gm[1] = (gdy - dir[1] * dd) * inv_vlen;
    gm[2] = (gdz - dir[2] * dd) * inv_vlen;
}

// Geometry of the projection: everything of project_one but the colour.
template <int DEG>
__device__ __forceinline__ void project_geometry(const Cam& cam, const Dil& dil, const float* mean,
                                                 const float* log_scale, float4 q, float logit, Proj& P)
{
    P.culled = true;
    P.rect = make_int4(0, 0, -1, -1);
    P.tiles = 0;
    P.radius = 0;
    // the SFU's exp, reciprocal and reciprocal square root (a few ulp) throughout:
    // no IEEE division or square-root sequences with their slow-path branches
    P.opacity = __fdividef(1.0f, 1.0f + __expf(-logit));
#pragma unroll
    for (int j = 0; j < 3; ++j) P.s[j] = __expf(log_scale[j]);
    float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    if (!(qn2 > 0.0f)) return;
    P.inv_qnorm = rsqrtf(qn2);
    P.qn[0] = q.x * P.inv_qnorm; P.qn[1] = q.y * P.inv_qnorm;
    P.qn[2] = q.z * P.inv_qnorm; P.qn[3] = q.w * P.inv_qnorm;
    quat_rot(P.qn[0], P.qn[1], P.qn[2], P.qn[3], P.R);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P.M[3 * i + j] = P.R[3 * i + j] * P.s[j];

    // camera space, float-float
    ff tx = ff_dot3_add(cam.R[0], mean[0], cam.R[1], mean[1], cam.R[2], mean[2], cam.T[0]);
    ff ty = ff_dot3_add(cam.R[3], mean[0], cam.R[4], mean[1], cam.R[5], mean[2], cam.T[1]);
    ff tz = ff_dot3_add(cam.R[6], mean[0], cam.R[7], mean[1], cam.R[8], mean[2], cam.T[2]);
    P.tz = tz.hi;
    if (!(P.tz > cam.z_near)) return;
    const float itz = __fdividef(1.0f, tz.hi);
    ff u = ff_div_rcp(tx, tz, itz), v = ff_div_rcp(ty, tz, itz);
    P.u = u.hi;
    P.v = v.hi;
    P.clamp_x = fabsf(P.u) > cam.lim_x;
    P.clamp_y = fabsf(P.v) > cam.lim_y;
    P.uc = P.clamp_x ? copysignf(cam.lim_x, P.u) : P.u;
    P.vc = P.clamp_y ? copysignf(cam.lim_y, P.v) : P.v;

    // Tm = J W with J = [[fx/tz, 0, -fx uc/tz], [0, fy/tz, -fy vc/tz]]
    float j00 = cam.fx * itz, j02 = -cam.fx * P.uc * itz;
    float j11 = cam.fy * itz, j12 = -cam.fy * P.vc * itz;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        P.Tm[j] = j00 * cam.R[j] + j02 * cam.R[6 + j];
        P.Tm[3 + j] = j11 * cam.R[3 + j] + j12 * cam.R[6 + j];
    }
    // N = Tm M, Sigma' = N N^T + low-pass
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            P.N[3 * i + k] = P.Tm[3 * i] * P.M[k] + P.Tm[3 * i + 1] * P.M[3 + k] + P.Tm[3 * i + 2] * P.M[6 + k];
    float a0 = P.N[0] * P.N[0] + P.N[1] * P.N[1] + P.N[2] * P.N[2];
    float b0 = P.N[0] * P.N[3] + P.N[1] * P.N[4] + P.N[2] * P.N[5];
    float c0 = P.N[3] * P.N[3] + P.N[4] * P.N[4] + P.N[5] * P.N[5];
    // det(N N^T) as the sum of squared 2x2 minors (Cauchy-Binet): no cancellation
    float m01 = det2(P.N[0], P.N[1], P.N[3], P.N[4]);
    float m02 = det2(P.N[0], P.N[2], P.N[3], P.N[5]);
    float m12 = det2(P.N[1], P.N[2], P.N[4], P.N[5]);
    float det0 = m01 * m01 + m02 * m02 + m12 * m12;
    P.a = a0 + kLowPass;
    P.b = b0;
    P.c = c0 + kLowPass;
    P.det = det0 + kLowPass * (a0 + c0) + kLowPass * kLowPass;
    if (!(P.det > 0.0f)) return;
    float inv_det = __fdividef(1.0f, P.det);
    P.A = P.c * inv_det;
    P.B = -P.b * inv_det;
    P.C = P.a * inv_det;
    float hd = 0.5f * (P.a - P.c);
    float disc = hd * hd + P.b * P.b;  // = mid^2 - det, without cancellation
    const float dfl = fmaxf(disc, kDiscFloor);
    float lam = 0.5f * (P.a + P.c) + dfl * rsqrtf(dfl);
    P.radius = (int)ceilf(3.0f * (lam * rsqrtf(lam)));

    P.px = ff_affine(cam.fx, u, cam.cx);
    P.py = ff_affine(cam.fy, v, cam.cy);

    // downsampled centre (Eq. 3 with the lattice of the offset, or Eq. 3+5 literal)
    float shx = dil.mode == 0 ? (float)dil.ox : 0.5f * (float)(dil.d - 1);
    float shy = dil.mode == 0 ? (float)dil.oy : 0.5f * (float)(dil.d - 1);
    float pdx = __fdiv_rn(__fadd_rn(__fsub_rn(P.px.hi, shx), P.px.lo), (float)dil.d);
    float pdy = __fdiv_rn(__fadd_rn(__fsub_rn(P.py.hi, shy), P.py.lo), (float)dil.d);
    float rds = __fdiv_rn((float)P.radius, (float)dil.d);  // Eq. 4
    float inv_tile = 1.0f / (float)dil.tile;               // exact (power of two)
    int x0 = (int)floorf(__fmul_rn(__fsub_rn(pdx, rds), inv_tile));
    int x1 = (int)floorf(__fmul_rn(__fadd_rn(pdx, rds), inv_tile));
    int y0 = (int)floorf(__fmul_rn(__fsub_rn(pdy, rds), inv_tile));
    int y1 = (int)floorf(__fmul_rn(__fadd_rn(pdy, rds), inv_tile));
    x0 = max(x0, 0);
    y0 = max(y0, 0);
    x1 = min(x1, dil.tiles_x - 1);
    y1 = min(y1, dil.tiles_y - 1);
    if (P.radius <= 0 || x0 > x1 || y0 > y1) return;
    P.frect = make_int4(x0, y0, x1, y1);
    // binning tiles: floor(v / (tile 2^s)) = floor(v / tile) >> s for the clipped bounds
    P.rect = make_int4(x0 >> dil.shift, y0 >> dil.shift, x1 >> dil.shift, y1 >> dil.shift);
    P.tiles = (P.rect.z - P.rect.x + 1) * (P.rect.w - P.rect.y + 1);
    P.culled = false;
}

template <int DEG>
__device__ __forceinline__ void project_one(const Cam& cam, const Dil& dil, const float* mean,
                                            const float* log_scale, float4 q, float logit,
                                            const float (&sh)[16][3], Proj& P)
{
    project_geometry<DEG>(cam, dil, mean, log_scale, q, logit, P);
    if (!P.culled) sh_colour<DEG>(cam, mean, sh, P.dir, P.inv_vlen, P.rgb_raw);
}

// Projection of every Gaussian into every view of the batch. The warp stages
// its 32 parameter rows once and loops over the views, so the parameters are
// read once per batch whatever the number of views.
// The outputs of one Gaussian's projection into view V: the splat record, radius,
// binning rect, tile count and depth key (an empty record for a culled one).
__device__ __forceinline__ void write_projection(const ViewDev& V, int g, const Proj& P)
{
    float4* out = V.splats + 4 * (int64_t)g;
    if (P.culled) {
        out[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        out[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        out[2] = make_float4(0.f, P.tz, 0.f, 0.f);
        out[3] = make_float4(0.f, 0.f, __int_as_float(-1), __int_as_float(-1));
        V.radii[g] = 0;
        V.rects[g] = make_int4(0, 0, -1, -1);
        V.tiles[g] = 0;
        if (V.keys) V.keys[g] = 0xffffffffu;
        return;
    }
    out[0] = make_float4(P.px.hi, P.py.hi, P.A, P.B);
    out[1] = make_float4(P.C, P.opacity, fmaxf(P.rgb_raw[0], 0.0f), fmaxf(P.rgb_raw[1], 0.0f));
    out[2] = make_float4(fmaxf(P.rgb_raw[2], 0.0f), P.tz, P.px.lo, P.py.lo);
    out[3] = make_float4(__int_as_float(P.frect.x), __int_as_float(P.frect.y), __int_as_float(P.frect.z),
                         __int_as_float(P.frect.w));
    V.radii[g] = P.radius;
    V.rects[g] = P.rect;
    V.tiles[g] = P.tiles;
    // the depth sort key: the float bits order like the positive depth; all ones is kept
    // for the culled
    if (V.keys) V.keys[g] = min(__float_as_uint(P.tz), 0xfffffffeu);
}

template <int DEG, int DT, bool MULTI>
__global__ void __launch_bounds__(kThreads, MULTI ? 1 : 8)
k_project(int n, const float* __restrict__ means, const float* __restrict__ log_scales,
          const float4* __restrict__ quats, const float* __restrict__ logits, const void* __restrict__ sh,
          const __grid_constant__ Batch b)
{
    kernel_prologue();
    using L = ShLayout<DEG, DT>;
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g0 = (blockIdx.x * kWarps + warp) * 32;
    if (g0 >= n) return;
    uint32_t* s_mean = smem + warp * L::WARP_WORDS;
    uint32_t* s_scale = s_mean + 32 * 3;
    uint32_t* s_sh = s_scale + 32 * 3;
    warp_stage<3, 3>(reinterpret_cast<const uint32_t*>(means), n, g0, s_mean, lane);
    warp_stage<3, 3>(reinterpret_cast<const uint32_t*>(log_scales), n, g0, s_scale, lane);
    if constexpr (L::STAGE)
        warp_stage<L::W, L::S, MULTI>(reinterpret_cast<const uint32_t*>(sh), n, g0, s_sh, lane);
    const int g = g0 + lane;
    if (g >= n) return;

    float mean[3], ls[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        mean[j] = __uint_as_float(s_mean[lane * 3 + j]);
        ls[j] = __uint_as_float(s_scale[lane * 3 + j]);
    }
    const float4 q = quats[g];
    const float logit = logits[g];
    const int nv = MULTI ? b.nviews : 1;
    for (int vi = 0; vi < nv; ++vi) {
        const ViewDev& V = b.v[MULTI ? vi : 0];
        // project_one, with the SH coefficients read from the staged row only for a view
        // that keeps the Gaussian (they are live for its colour alone)
        Proj P;
        project_geometry<DEG>(V.cam, V.dil, mean, ls, q, logit, P);
        if (!P.culled) {
            float c[16][3];
            read_sh<DEG, DT>(s_sh, sh, g, lane, c);
            sh_colour<DEG>(V.cam, mean, c, P.dir, P.inv_vlen, P.rgb_raw);
        }
        write_projection(V, g, P);
    }
}

// ---------------------------------------------------------------------------
// Backward of the projection (chain rule through conic, Sigma' = N N^T + lp,
// N = J W M, M = R(q) S, the image-plane centre and the SH direction).
// ---------------------------------------------------------------------------
struct ParamGrad {
    float gm[3], gls[3];
    float4 gq;
    float glogit;
};

// Gradients of one visible Gaussian from its 2D gradient record (G0, G1):
// everything but the colour (sh_colour_bwd), with R.gm starting from gm0 (the
// mean's gradient through the view direction).
__device__ __forceinline__ void project_bwd_one(const Cam& cam, const Proj& P, float4 G0, float4 G1,
                                                const float* gm0, ParamGrad& R)
{
    const float gpx = G0.x, gpy = G0.y, gA = G0.z, gB = G0.w, gC = G1.x, gop = G1.y;
#pragma unroll
    for (int j = 0; j < 3; ++j) R.gm[j] = gm0[j];
    // opacity = sigmoid(logit)
    R.glogit = gop * P.opacity * (1.0f - P.opacity);

    // conic = inverse of Sigma': dL/dSigma' = -K Gk K, Gk = [[gA, gB/2], [gB/2, gC]]
    float k00 = P.A * gA + P.B * 0.5f * gB, k01 = P.A * 0.5f * gB + P.B * gC;
    float k10 = P.B * gA + P.C * 0.5f * gB, k11 = P.B * 0.5f * gB + P.C * gC;
    float s00 = -(k00 * P.A + k01 * P.B);
    float s01 = -(k00 * P.B + k01 * P.C);
    float s11 = -(k10 * P.B + k11 * P.C);
    // Sigma' = N N^T + lp: dL/dN = 2 S N
    float dN[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dN[k] = 2.0f * (s00 * P.N[k] + s01 * P.N[3 + k]);
        dN[3 + k] = 2.0f * (s01 * P.N[k] + s11 * P.N[3 + k]);
    }
    // N = Tm M: dTm = dN M^T, dM = Tm^T dN
    float dTm[6], dM[9];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dTm[3 * i + j] = dN[3 * i] * P.M[3 * j] + dN[3 * i + 1] * P.M[3 * j + 1] + dN[3 * i + 2] * P.M[3 * j + 2];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) dM[3 * j + k] = P.Tm[j] * dN[k] + P.Tm[3 + j] * dN[3 + k];
    // Tm = J W: dJ_il = sum_j dTm_ij W_lj (only J00, J02, J11, J12 vary)
    float dJ00 = dTm[0] * cam.R[0] + dTm[1] * cam.R[1] + dTm[2] * cam.R[2];
    float dJ02 = dTm[0] * cam.R[6] + dTm[1] * cam.R[7] + dTm[2] * cam.R[8];
    float dJ11 = dTm[3] * cam.R[3] + dTm[4] * cam.R[4] + dTm[5] * cam.R[5];
    float dJ12 = dTm[3] * cam.R[6] + dTm[4] * cam.R[7] + dTm[5] * cam.R[8];
    const float tz = P.tz, itz = __fdividef(1.0f, tz), itz2 = itz * itz;
    float dt0 = 0.f, dt1 = 0.f, dt2 = 0.f;
    dt2 += -(dJ00 * cam.fx + dJ11 * cam.fy) * itz2;
    if (P.clamp_x) {
        dt2 += dJ02 * cam.fx * P.uc * itz2;
    } else {
        dt0 += -dJ02 * cam.fx * itz2;
        dt2 += 2.0f * dJ02 * cam.fx * P.u * itz2;
    }
    if (P.clamp_y) {
        dt2 += dJ12 * cam.fy * P.vc * itz2;
    } else {
        dt1 += -dJ12 * cam.fy * itz2;
        dt2 += 2.0f * dJ12 * cam.fy * P.v * itz2;
    }
    // image-plane centre p = (fx tx/tz + cx, fy ty/tz + cy)
    dt0 += gpx * cam.fx * itz;
    dt1 += gpy * cam.fy * itz;
    dt2 += -(gpx * cam.fx * P.u + gpy * cam.fy * P.v) * itz;
    // t = W mean + T
#pragma unroll
    for (int j = 0; j < 3; ++j) R.gm[j] += cam.R[j] * dt0 + cam.R[3 + j] * dt1 + cam.R[6 + j] * dt2;

    // M = R diag(s)
    float dR[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            acc += dM[3 * j + k] * P.R[3 * j + k];
            dR[3 * j + k] = dM[3 * j + k] * P.s[k];
        }
        R.gls[k] = acc * P.s[k];
    }
    // R(w, x, y, z)
    const float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
    float gw = 2.0f * (z * (dR[3] - dR[1]) + y * (dR[2] - dR[6]) + x * (dR[7] - dR[5]));
    float gx = 2.0f * (y * (dR[1] + dR[3]) + z * (dR[2] + dR[6]) + w * (dR[7] - dR[5]) - 2.0f * x * (dR[4] + dR[8]));
    float gy = 2.0f * (x * (dR[1] + dR[3]) + z * (dR[5] + dR[7]) + w * (dR[2] - dR[6]) - 2.0f * y * (dR[0] + dR[8]));
    float gz = 2.0f * (x * (dR[2] + dR[6]) + y * (dR[5] + dR[7]) + w * (dR[3] - dR[1]) - 2.0f * z * (dR[0] + dR[4]));
    float qd = gw * w + gx * x + gy * y + gz * z;
    R.gq = make_float4((gw - w * qd) * P.inv_qnorm, (gx - x * qd) * P.inv_qnorm,
                     (gy - y * qd) * P.inv_qnorm, (gz - z * qd) * P.inv_qnorm);

}

__device__ __forceinline__ void densify_one(int g, const int* tiles_touched, float4 G0, float4 G1, float4 G2,
                                            float* pos_acc, float* col_acc, int* count)
{
    if (pos_acc != nullptr && tiles_touched[g] > 0) {
        pos_acc[g] += sqrtf(G0.x * G0.x + G0.y * G0.y);
        col_acc[g] += sqrtf(G1.z * G1.z + G1.w * G1.w + G2.x * G2.x);
        count[g] += 1;
    }
}

template <int DEG, int DT>
__global__ void __launch_bounds__(kThreads)
k_project_bwd(int n, const float* __restrict__ means, const float* __restrict__ log_scales,
              const float4* __restrict__ quats, const float* __restrict__ logits,
              const void* __restrict__ sh, Cam cam, Dil dil, const int* __restrict__ tiles_touched,
              const float4* __restrict__ grad2d, float* __restrict__ d_means,
              float* __restrict__ d_log_scales, float4* __restrict__ d_quats,
              float* __restrict__ d_logits, float* __restrict__ d_sh, float* __restrict__ pos_acc,
              float* __restrict__ col_acc, int* __restrict__ count)
{
    kernel_prologue();
    using L = ShLayout<DEG, DT>;
    constexpr int K = L::K;
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g0 = (blockIdx.x * kWarps + warp) * 32;
    if (g0 >= n) return;
    uint32_t* s_mean = smem + warp * L::WARP_WORDS;
    uint32_t* s_scale = s_mean + 32 * 3;
    uint32_t* s_sh = s_scale + 32 * 3;
    warp_stage<3, 3>(reinterpret_cast<const uint32_t*>(means), n, g0, s_mean, lane);
    warp_stage<3, 3>(reinterpret_cast<const uint32_t*>(log_scales), n, g0, s_scale, lane);
    if constexpr (L::STAGE) warp_stage<L::W, L::S>(reinterpret_cast<const uint32_t*>(sh), n, g0, s_sh, lane);
    const int g = g0 + lane;
    if (g >= n) return;

    float mean[3], ls[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        mean[j] = __uint_as_float(s_mean[lane * 3 + j]);
        ls[j] = __uint_as_float(s_scale[lane * 3 + j]);
    }
    float c[16][3];
    read_sh<DEG, DT>(s_sh, sh, g, lane, c);
    Proj P;
    project_one<DEG>(cam, dil, mean, ls, quats[g], logits[g], c, P);
    float* gsh = d_sh + (int64_t)g * K * 3;
    if (P.culled) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            d_means[3 * (int64_t)g + j] = 0.f;
            d_log_scales[3 * (int64_t)g + j] = 0.f;
        }
        d_quats[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        d_logits[g] = 0.f;
#pragma unroll
        for (int e = 0; e < K * 3; ++e) gsh[e] = 0.f;
        return;
    }
    const float4 G0 = grad2d[3 * (int64_t)g], G1 = grad2d[3 * (int64_t)g + 1], G2 = grad2d[3 * (int64_t)g + 2];
    densify_one(g, tiles_touched, G0, G1, G2, pos_acc, col_acc, count);
    float gm_dir[3];
    sh_colour_bwd<DEG, false>(P.dir, P.inv_vlen, P.rgb_raw, c, G1.z, G1.w, G2.x, gsh, gm_dir);
    ParamGrad R;
    project_bwd_one(cam, P, G0, G1, gm_dir, R);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        d_means[3 * (int64_t)g + j] = R.gm[j];
        d_log_scales[3 * (int64_t)g + j] = R.gls[j];
    }
    d_quats[g] = R.gq;
    d_logits[g] = R.glogit;
}

// ---------------------------------------------------------------------------
// Projection backward + densification statistics + Adam in one pass: each
// warp takes 32 Gaussians, computes their gradients into shared memory and
// then updates the parameter rows and their moments with coalesced accesses
// over the warp's contiguous segment of every tensor.
// ---------------------------------------------------------------------------
struct AdamDev {
    float* p[5];
    float* m[5];
    float* v[5];
    float lr[5];
    float b1, b2, eps, inv_bc1, inv_bc2;
    const float* bias;  // device (1/(1-b1^t), 1/(1-b2^t)) replacing inv_bc1/2 when set
    int sparse;
    void* shadow;
    int shadow_dtype;
    float* gout[5];
    int lowp;            // SH kept only in sh_store (BF16/FP16), rounded stochastically
    uint32_t sr_seed;
    int step;            // t of the rounding stream when step_dev is null
    const int* step_dev;
};

template <int DEG, int DT, bool MULTI>
struct FusedLayout {
    using L = ShLayout<DEG, DT>;
    static constexpr int KW = L::K * 3;                   // SH floats per Gaussian
    static constexpr int GS0 = KW % 2 == 0 ? KW + 1 : KW;  // odd stride of the SH gradient rows
    // VEC (one view, rows of whole 16-byte vectors both as stored and as FP32 gradients): the rows are 16-byte
    // aligned with an odd number of vectors per row, and every access to them is a
    // 16-byte vector (the staging, the reads of the staged row, the gradient row's
    // writes, Adam's reads of the gradients and write-back of the new values, the
    // next view's projection): conflict-free, where the per-float accesses to the
    // odd-stride rows of the other forms conflict 4 ways in the vector passes
    static constexpr bool VEC = !MULTI && KW % 4 == 0 && (DT == GS_DTYPE_F32 || (KW / 2) % 4 == 0);
    // one region per lane row: first the staged SH coefficients, then (same lane,
    // after it has read them) its SH gradients
    static constexpr int GS = VEC ? ((KW / 4) % 2 == 1 ? KW : KW + 4) : ((L::STAGE && L::S > GS0) ? L::S : GS0);
    static constexpr int WARP_WORDS = 32 * (3 + 3) + 32 * 7 + 32 * GS;
    static_assert(!VEC || WARP_WORDS % 4 == 0, "16-byte aligned warp regions");
};

// Visible in at least one view of the batch (the rows sparse Adam updates).
__device__ __forceinline__ bool visible_any(const Batch& b, int g)
{
    for (int i = 0; i < b.nviews; ++i)
        if (b.v[i].tiles[g] > 0) return true;
    return false;
}

// Adam over the warp's contiguous segment [g0*W, (g0+rows)*W) of one tensor,
// gradients read from shared memory rows of stride GSTRIDE at column offset
// goff. A full, dense warp moves 16-byte vectors with several in flight per
// lane; otherwise one element at a time. Bit r of vis marks row r visible
// (sparse Adam updates only those rows). WB: each element's gradient slot in
// shared memory takes the element's new value as the projection will read it
// (the shadow's rounding when there is a shadow copy), for a projection of the
// updated parameters in the same kernel (dense Adam only).
template <int W, int GSTRIDE, bool WB = false>
__device__ __forceinline__ void adam_segment(const AdamDev& a, int t, int g0, int rows, float* s_grad,
                                             int goff, unsigned vis, float bc1, float bc2, int lane, void* shadow,
                                             int shadow_dtype)
{
    const int64_t base = (int64_t)g0 * W;
    float* P = a.p[t] + base;
    float* M = a.m[t] + base;
    float* V = a.v[t] + base;
    const uintptr_t al = reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(M) |
                         reinterpret_cast<uintptr_t>(V);
    // the shadow copy is written 4 values at a time (8 bytes for BF16/FP16, 16 for FP32) when
    // those vectors are aligned
    const int64_t seb = shadow_dtype == GS_DTYPE_F32 ? 4 : 2;
    const bool shadow4 = shadow != nullptr && base % 4 == 0 &&
                         ((reinterpret_cast<uintptr_t>(shadow) + seb * base) & (uintptr_t)(4 * seb - 1)) == 0;
    if (rows == 32 && !a.sparse && (al & 15) == 0 && (shadow == nullptr || shadow4)) {
        constexpr int Q = 8 * W;            // 16-byte vectors in the segment (32 W floats)
        constexpr int KN = (Q + 31) / 32;   // vectors per lane, the last one partial when Q % 32 != 0
        constexpr int B = KN < 4 ? KN : 4;  // vectors of each array loaded before any is stored
        float4* P4 = reinterpret_cast<float4*>(P);
        float4* M4 = reinterpret_cast<float4*>(M);
        float4* V4 = reinterpret_cast<float4*>(V);
#pragma unroll
        for (int k0 = 0; k0 < KN; k0 += B) {
            // all loads of the group first: the stores of one vector could alias the next
            // one's loads as far as the compiler knows, which would leave one vector per array
            // in flight per lane
            float4 p[B], m[B], v[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int q = lane + 32 * (k0 + u);
                if (k0 + u < KN && q < Q) {
                    p[u] = P4[q];
                    m[u] = M4[q];
                    v[u] = V4[q];
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int q = lane + 32 * (k0 + u);
                if (k0 + u >= KN || q >= Q) continue;
                float* pp = &p[u].x;
                float* mm = &m[u].x;
                float* vv = &v[u].x;
                if constexpr (GSTRIDE % 4 == 0 && W % 4 == 0) {
                    // 16-byte aligned gradient rows (goff 0): the vector's 4 slots as one vector
                    float4* gslot = reinterpret_cast<float4*>(s_grad + ((4 * q) / W) * GSTRIDE + goff + (4 * q) % W);
                    const float4 g4 = *gslot;
                    const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        adam_step(pp[c], gv[c], mm[c], vv[c], a.b1, a.b2, a.eps, bc1, bc2, a.lr[t]);
                        if (a.gout[t]) a.gout[t][base + 4 * q + c] = gv[c];
                    }
                    if constexpr (WB) *gslot = p[u];
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int e = 4 * q + c;
                        const int slot = (e / W) * GSTRIDE + goff + e % W;
                        const float g = s_grad[slot];
                        adam_step(pp[c], g, mm[c], vv[c], a.b1, a.b2, a.eps, bc1, bc2, a.lr[t]);
                        if (a.gout[t]) a.gout[t][base + e] = g;
                        if constexpr (WB) s_grad[slot] = pp[c];
                    }
                }
                P4[q] = p[u];
                M4[q] = m[u];
                V4[q] = v[u];
                if (shadow) store4_as(shadow, shadow_dtype, base + 4 * q, p[u]);
            }
        }
        if constexpr (WB) {
            // the shadow's rounding of the new values, in a pass of its own (a select in the
            // loop above costs registers the streaming loads need)
            if (shadow && shadow_dtype != GS_DTYPE_F32) {
                __syncwarp();
                for (int e = lane; e < 32 * W; e += 32) {
                    const int slot = (e / W) * GSTRIDE + goff + e % W;
                    s_grad[slot] = stored_value(shadow_dtype, s_grad[slot]);
                }
            }
        }
        return;
    }
    for (int e = lane; e < rows * W; e += 32) {
        const int row = e / W, col = e % W;
        const int slot = row * GSTRIDE + goff + col;
        const float g = s_grad[slot];
        if (a.gout[t]) a.gout[t][base + e] = g;
        if (a.sparse && !((vis >> row) & 1u)) continue;
        float p = P[e], m = M[e], v = V[e];
        adam_step(p, g, m, v, a.b1, a.b2, a.eps, bc1, bc2, a.lr[t]);
        P[e] = p;
        M[e] = m;
        V[e] = v;
        if (shadow) store_as(shadow, shadow_dtype, base + e, p);
        if constexpr (WB) s_grad[slot] = shadow ? stored_value(shadow_dtype, p) : p;
    }
}

// Adam over the warp's segment of the SH kept only in 16 bits (BF16/FP16 sh_store,
// no FP32 copy): the update is computed in FP32 from the stored value and rounded
// stochastically (element e of the tensor draws sr_bits16(sr, e)). A full, dense
// warp moves units of 4 values like adam_segment (an 8-byte vector of the
// parameter, a 16-byte one of each moment: every warp access is contiguous), 4
// units in flight per lane; otherwise one element at a time.
template <int W, int GSTRIDE, int DT, bool WB = false>
__device__ __forceinline__ void adam_segment_lowp(const AdamDev& a, int g0, int rows, float* s_grad,
                                                  unsigned vis, float bc1, float bc2, int lane, void* store,
                                                  uint32_t sr)
{
    if constexpr (DT != GS_DTYPE_F32) {
        const int64_t base = (int64_t)g0 * W;
        uint16_t* P = reinterpret_cast<uint16_t*>(store) + base;
        float* M = a.m[4] + base;
        float* V = a.v[4] + base;
        float* gout = a.gout[4];
        // the stored value as FP32: a shift for BF16, the conversion instruction for FP16 (one
        // instruction; an integer form with a branch for subnormals measured slower, 0.881 ->
        // 0.829 ms)
        auto tofloat = [](uint32_t h) {
            if constexpr (DT == GS_DTYPE_BF16) return __uint_as_float(h << 16);
            else return __half2float(__ushort_as_half((uint16_t)h));
        };
        const uintptr_t al = reinterpret_cast<uintptr_t>(M) | reinterpret_cast<uintptr_t>(V);
        if (rows == 32 && !a.sparse && (al & 15) == 0 && (reinterpret_cast<uintptr_t>(P) & 7) == 0) {
            constexpr int Q = 8 * W;            // units of 4 values in the segment (32 W values)
            constexpr int KN = (Q + 31) / 32;   // units per lane, the last one partial when Q % 32 != 0
            constexpr int B = KN < 4 ? KN : 4;  // units loaded before any is stored
            uint2* P2 = reinterpret_cast<uint2*>(P);
            float4* M4 = reinterpret_cast<float4*>(M);
            float4* V4 = reinterpret_cast<float4*>(V);
            // the groups of units one after another (not unrolled): the rounding's integer work
            // would otherwise crowd the instruction cache (BF16 0.744 -> 0.729 ms, FP16
            // 0.998 -> 0.881 ms on 3M Gaussians)
#pragma unroll 1
            for (int k0 = 0; k0 < KN; k0 += B) {
                uint2 p[B];
                float4 m[B], v[B];
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    const int q = lane + 32 * (k0 + u);
                    if (k0 + u < KN && q < Q) {
                        p[u] = P2[q];
                        m[u] = M4[q];
                        v[u] = V4[q];
                    }
                }
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    const int q = lane + 32 * (k0 + u);
                    if (k0 + u >= KN || q >= Q) continue;
                    float x[4] = {tofloat(p[u].x & 0xffffu), tofloat(p[u].x >> 16), tofloat(p[u].y & 0xffffu),
                                  tofloat(p[u].y >> 16)};
                    float* mm = &m[u].x;
                    float* vv = &v[u].x;
                    // the random bits of the unit's 4 elements: two hashes (base + 4q is even)
                    const uint32_t k2 = (uint32_t)((base + 4 * q) >> 1);
                    const uint32_t r01 = pcg_hash(sr + k2), r23 = pcg_hash(sr + k2 + 1u);
                    const uint32_t rb[4] = {r01 & 0xffffu, r01 >> 16, r23 & 0xffffu, r23 >> 16};
                    uint32_t h[4];
                    if constexpr (GSTRIDE % 4 == 0 && W % 4 == 0) {
                        // 16-byte aligned gradient rows: the unit's 4 slots as one vector
                        float4* gslot = reinterpret_cast<float4*>(s_grad + ((4 * q) / W) * GSTRIDE + (4 * q) % W);
                        const float4 g4 = *gslot;
                        const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            adam_step(x[c], gv[c], mm[c], vv[c], a.b1, a.b2, a.eps, bc1, bc2, a.lr[4]);
                            h[c] = sr_round(x[c], rb[c], DT);
                            if (gout) gout[base + 4 * q + c] = gv[c];
                        }
                        if constexpr (WB) *gslot = make_float4(tofloat(h[0]), tofloat(h[1]), tofloat(h[2]), tofloat(h[3]));
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int e = 4 * q + c;
                            const int slot = (e / W) * GSTRIDE + e % W;
                            const float g = s_grad[slot];
                            adam_step(x[c], g, mm[c], vv[c], a.b1, a.b2, a.eps, bc1, bc2, a.lr[4]);
                            h[c] = sr_round(x[c], rb[c], DT);
                            if (gout) gout[base + e] = g;
                            if constexpr (WB) s_grad[slot] = tofloat(h[c]);
                        }
                    }
                    P2[q] = make_uint2(__byte_perm(h[0], h[1], 0x5410), __byte_perm(h[2], h[3], 0x5410));
                    M4[q] = m[u];
                    V4[q] = v[u];
                }
            }
            return;
        }
        for (int e = lane; e < rows * W; e += 32) {
            const int row = e / W, col = e % W;
            const int slot = row * GSTRIDE + col;
            const float g = s_grad[slot];
            if (gout) gout[base + e] = g;
            if (a.sparse && !((vis >> row) & 1u)) continue;
            float x = tofloat(P[e]), m = M[e], v = V[e];
            adam_step(x, g, m, v, a.b1, a.b2, a.eps, bc1, bc2, a.lr[4]);
            const uint16_t hv = sr_round(x, sr_bits16(sr, (uint32_t)(base + e)), DT);
            P[e] = hv;
            M[e] = m;
            V[e] = v;
            if constexpr (WB) s_grad[slot] = tofloat(hv);
        }
    }
}

// The SH coefficients of Gaussian g straight from the storage array (one
// lane's own row): 16-byte vector loads when rows are whole 16-byte units and
// the array is 16-byte aligned, else element by element. Used by the batched
// optimizer pass, which re-reads them per view (from L1 after the first).
template <int DEG, int DT>
__device__ __forceinline__ void load_sh_row(const void* sh, int g, float (&c)[16][3])
{
    constexpr int K = (DEG + 1) * (DEG + 1), E = K * 3;
    constexpr int EB = DT == GS_DTYPE_F32 ? 4 : 2;
    if constexpr ((E * EB) % 16 == 0) {
        if ((reinterpret_cast<uintptr_t>(sh) & 15) == 0) {
            constexpr int NV = E * EB / 16;
            const uint4* row = reinterpret_cast<const uint4*>(static_cast<const char*>(sh) + (int64_t)g * E * EB);
            uint32_t w[NV * 4];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const uint4 x = __ldg(row + v);
                w[4 * v] = x.x; w[4 * v + 1] = x.y; w[4 * v + 2] = x.z; w[4 * v + 3] = x.w;
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if constexpr (DT == GS_DTYPE_F32) {
                    c[e / 3][e % 3] = __uint_as_float(w[e]);
                } else {
                    const uint16_t hv = (e & 1) ? (uint16_t)(w[e >> 1] >> 16) : (uint16_t)(w[e >> 1] & 0xffffu);
                    if constexpr (DT == GS_DTYPE_BF16) c[e / 3][e % 3] = __bfloat162float(__ushort_as_bfloat16(hv));
                    else c[e / 3][e % 3] = __half2float(__ushort_as_half(hv));
                }
            }
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) c[e / 3][e % 3] = load_sh_elem(sh, (int64_t)g * E + e, DT);
}

// Projection backward of one Gaussian in one view, added into the gradient
// rows (the batched form). A view that did not render the Gaussian (no tile
// touched) gave it a zero 2D gradient and is skipped, and so is a view whose
// recomputed projection culls it (as the one-view backward does). The SH
// coefficients are re-read for the view inside the colour part, so that they
// are live only there. False when the view is skipped.
template <int DEG, int DT>
__device__ __forceinline__ bool fused_view_grad(const ViewDev& V, int g, const float* mean, const float* ls,
                                                float4 q, float logit, const void* sh_store, float* grow,
                                                float* gshrow, float4& gq, float& glogit, float* pos_acc,
                                                float* col_acc, int* count)
{
    if (V.tiles[g] <= 0) return false;
    Proj P;
    project_geometry<DEG>(V.cam, V.dil, mean, ls, q, logit, P);
    if (P.culled) return false;
    const float4 G1 = V.grad2d[3 * (int64_t)g + 1], G2 = V.grad2d[3 * (int64_t)g + 2];
    float gm_dir[3];
    {
        float c[16][3];
        load_sh_row<DEG, DT>(sh_store, g, c);
        float dir[3], inv_vlen, rgb_raw[3];
        sh_colour<DEG>(V.cam, mean, c, dir, inv_vlen, rgb_raw);
        sh_colour_bwd<DEG, true>(dir, inv_vlen, rgb_raw, c, G1.z, G1.w, G2.x, gshrow, gm_dir);
    }
    const float4 G0 = V.grad2d[3 * (int64_t)g];
    densify_one(g, V.tiles, G0, G1, G2, pos_acc, col_acc, count);
    ParamGrad R;
    project_bwd_one(V.cam, P, G0, G1, gm_dir, R);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        grow[j] += R.gm[j];
        grow[3 + j] += R.gls[j];
    }
    gq.x += R.gq.x; gq.y += R.gq.y; gq.z += R.gq.z; gq.w += R.gq.w;
    glogit += R.glogit;
    return true;
}

// Adam over a full, dense warp's rows of means, log-scales, quaternions and
// logits with all their loads issued together (one round trip to memory for
// the four tensors): lanes below 24 take one 16-byte vector of each 3-float
// tensor's 96 floats, every lane its own quaternion and logit.
// The means and log-scales of the warp's 32 rows (16-byte vectors, lanes 0..23)
// and each lane's quaternion and opacity logit. The new means and log-scales also
// go to their gradient slots in s_gms, and the lane's new quaternion and logit to
// q_new and logit_new, for a projection of the updated parameters.
__device__ __forceinline__ void adam_small_rows(const AdamDev& a, int g0, int g, float* s_gms, float4 gq,
                                                float glogit, float bc1, float bc2, int lane, float4& q_new,
                                                float& logit_new)
{
    const bool act = lane < 24;
    const int64_t b3 = (int64_t)g0 * 3;
    float4 p[2], m[2], v[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (!act) continue;
        p[t] = reinterpret_cast<const float4*>(a.p[t] + b3)[lane];
        m[t] = reinterpret_cast<const float4*>(a.m[t] + b3)[lane];
        v[t] = reinterpret_cast<const float4*>(a.v[t] + b3)[lane];
    }
    float4 pq = reinterpret_cast<const float4*>(a.p[2])[g];
    float4 mq = reinterpret_cast<const float4*>(a.m[2])[g];
    float4 vq = reinterpret_cast<const float4*>(a.v[2])[g];
    float po = a.p[3][g], mo = a.m[3][g], vo = a.v[3][g];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (!act) continue;
        float* pp = &p[t].x;
        float* mm = &m[t].x;
        float* vv = &v[t].x;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int e = 4 * lane + c;
            const int slot = (e / 3) * 7 + 3 * t + e % 3;
            const float gr = s_gms[slot];
            adam_step(pp[c], gr, mm[c], vv[c], a.b1, a.b2, a.eps, bc1, bc2, a.lr[t]);
            if (a.gout[t]) a.gout[t][b3 + e] = gr;
            s_gms[slot] = pp[c];
        }
        reinterpret_cast<float4*>(a.p[t] + b3)[lane] = p[t];
        reinterpret_cast<float4*>(a.m[t] + b3)[lane] = m[t];
        reinterpret_cast<float4*>(a.v[t] + b3)[lane] = v[t];
    }
    adam_step(pq.x, gq.x, mq.x, vq.x, a.b1, a.b2, a.eps, bc1, bc2, a.lr[2]);
    adam_step(pq.y, gq.y, mq.y, vq.y, a.b1, a.b2, a.eps, bc1, bc2, a.lr[2]);
    adam_step(pq.z, gq.z, mq.z, vq.z, a.b1, a.b2, a.eps, bc1, bc2, a.lr[2]);
    adam_step(pq.w, gq.w, mq.w, vq.w, a.b1, a.b2, a.eps, bc1, bc2, a.lr[2]);
    reinterpret_cast<float4*>(a.p[2])[g] = pq;
    reinterpret_cast<float4*>(a.m[2])[g] = mq;
    reinterpret_cast<float4*>(a.v[2])[g] = vq;
    adam_step(po, glogit, mo, vo, a.b1, a.b2, a.eps, bc1, bc2, a.lr[3]);
    a.p[3][g] = po;
    a.m[3][g] = mo;
    a.v[3][g] = vo;
    if (a.gout[2]) reinterpret_cast<float4*>(a.gout[2])[g] = gq;
    if (a.gout[3]) a.gout[3][g] = glogit;
    q_new = pq;
    logit_new = po;
}

// The quaternion (16-byte row) and opacity logit of each lane's Gaussian, one
// row per lane; their new values to q_new and logit_new.
__device__ __forceinline__ void adam_quat_logit(const AdamDev& a, int g, bool valid, unsigned vis, float4 gq,
                                                float glogit, float bc1, float bc2, int lane, float4& q_new,
                                                float& logit_new)
{
    if (valid) {
        if (a.gout[2]) reinterpret_cast<float4*>(a.gout[2])[g] = gq;
        if (a.gout[3]) a.gout[3][g] = glogit;
    }
    if (valid && !(a.sparse && !((vis >> lane) & 1u))) {
        float4 p = reinterpret_cast<float4*>(a.p[2])[g];
        float4 m = reinterpret_cast<float4*>(a.m[2])[g];
        float4 v = reinterpret_cast<float4*>(a.v[2])[g];
        adam_step(p.x, gq.x, m.x, v.x, a.b1, a.b2, a.eps, bc1, bc2, a.lr[2]);
        adam_step(p.y, gq.y, m.y, v.y, a.b1, a.b2, a.eps, bc1, bc2, a.lr[2]);
        adam_step(p.z, gq.z, m.z, v.z, a.b1, a.b2, a.eps, bc1, bc2, a.lr[2]);
        adam_step(p.w, gq.w, m.w, v.w, a.b1, a.b2, a.eps, bc1, bc2, a.lr[2]);
        reinterpret_cast<float4*>(a.p[2])[g] = p;
        reinterpret_cast<float4*>(a.m[2])[g] = m;
        reinterpret_cast<float4*>(a.v[2])[g] = v;
        float po = a.p[3][g], mo = a.m[3][g], vo = a.v[3][g];
        adam_step(po, glogit, mo, vo, a.b1, a.b2, a.eps, bc1, bc2, a.lr[3]);
        a.p[3][g] = po;
        a.m[3][g] = mo;
        a.v[3][g] = vo;
        q_new = p;
        logit_new = po;
    }
}

// One warp per 32 Gaussians: stage the parameters, project and differentiate
// them in every view of the batch (gradients summed over views), then one
// Adam step for the warp's rows. MULTI false is the one-view form, which
// writes the gradients instead of accumulating them.
// NEXT (one view, dense Adam): the updated parameters, which the Adam step also
// leaves in the warp's shared-memory gradient slots, are then projected into
// the next step's view nv (gs_project's formulas on the same stored values;
// only the conic may round differently, as the two kernels contract its
// products differently), so the next step reads the parameters from HBM once
// instead of twice.
// 5 CTAs per SM (96 registers, no spills): with 4 vectors per array in flight per
// lane in the Adam step, 5 beat 4 and 6 (spills) on this streaming pass
template <int DEG, int DT, bool MULTI, bool NEXT = false>
__global__ void __launch_bounds__(kThreads, MULTI ? 4 : 5)
k_project_bwd_adam(int n, const void* sh_store, const __grid_constant__ Batch b, AdamDev a,
                   float* __restrict__ pos_acc, float* __restrict__ col_acc, int* __restrict__ count,
                   const __grid_constant__ ViewDev nv)
{
    kernel_prologue();
    using L = ShLayout<DEG, DT>;
    using F = FusedLayout<DEG, DT, MULTI>;
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g0 = (blockIdx.x * kWarps + warp) * 32;
    if (g0 >= n) return;
    const int rows = min(32, n - g0);
    uint32_t* s_mean = smem + warp * F::WARP_WORDS;
    uint32_t* s_scale = s_mean + 32 * 3;
    float* s_gms = reinterpret_cast<float*>(s_scale + 32 * 3);  // 32 x 7
    uint32_t* s_sh = reinterpret_cast<uint32_t*>(s_gms + 32 * 7);  // 32 rows of stride GS
    float* s_gsh = reinterpret_cast<float*>(s_sh);
    warp_stage<3, 3>(reinterpret_cast<const uint32_t*>(a.p[0]), n, g0, s_mean, lane);
    warp_stage<3, 3>(reinterpret_cast<const uint32_t*>(a.p[1]), n, g0, s_scale, lane);
    // the one-view form stages the SH rows; the batched form re-reads each row per view
    if constexpr (L::STAGE && !MULTI)
        warp_stage<L::W, F::GS>(reinterpret_cast<const uint32_t*>(sh_store), n, g0, s_sh, lane);
    const int g = g0 + lane;
    const bool valid = g < n;

    float4 gq = make_float4(0.f, 0.f, 0.f, 0.f);
    float glogit = 0.0f;
    float* grow = s_gms + lane * 7;
    float* gshrow = s_gsh + lane * F::GS;
#pragma unroll
    for (int j = 0; j < 6; ++j) grow[j] = 0.0f;
    bool have_grad = false;
    if (valid) {
        float mean[3], ls[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            mean[j] = __uint_as_float(s_mean[lane * 3 + j]);
            ls[j] = __uint_as_float(s_scale[lane * 3 + j]);
        }
        const float4 q = reinterpret_cast<const float4*>(a.p[2])[g];
        const float logit = a.p[3][g];
        if constexpr (MULTI) {
#pragma unroll
            for (int e = 0; e < F::KW; ++e) gshrow[e] = 0.0f;
            have_grad = true;
            for (int vi = 0; vi < b.nviews; ++vi)
                fused_view_grad<DEG, DT>(b.v[vi], g, mean, ls, q, logit, sh_store, grow, gshrow, gq, glogit,
                                         pos_acc, col_acc, count);
        } else if (b.v[0].tiles[g] > 0) {
            // the colour part first, so the SH coefficients are dead before the geometry (the
            // staged SH of this row is read into c, then the row takes the SH gradients). A
            // Gaussian the view did not render has a zero 2D gradient: the zero rows below.
            float c[16][3];
            read_sh<DEG, DT, F::GS>(s_sh, sh_store, g, lane, c);
            const ViewDev& V = b.v[0];
            const float4 G1 = V.grad2d[3 * (int64_t)g + 1], G2 = V.grad2d[3 * (int64_t)g + 2];
            float dir[3], inv_vlen, rgb_raw[3], gm_dir[3];
            sh_colour<DEG>(V.cam, mean, c, dir, inv_vlen, rgb_raw);
            sh_colour_bwd<DEG, false, F::VEC>(dir, inv_vlen, rgb_raw, c, G1.z, G1.w, G2.x, gshrow, gm_dir);
            have_grad = true;
            Proj P;
            project_geometry<DEG>(V.cam, V.dil, mean, ls, q, logit, P);
            if (P.culled) {
                // only with tiles counted at other parameters than these: no gradient, as in
                // the unfused backward
                zero_row<F::KW, F::VEC>(gshrow);
            } else {
                const float4 G0 = V.grad2d[3 * (int64_t)g];
                densify_one(g, V.tiles, G0, G1, G2, pos_acc, col_acc, count);
                ParamGrad R;
                project_bwd_one(V.cam, P, G0, G1, gm_dir, R);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    grow[j] = R.gm[j];
                    grow[3 + j] = R.gls[j];
                }
                gq = R.gq;
                glogit = R.glogit;
            }
        }
    }
    if (!have_grad) zero_row<F::KW, F::VEC>(gshrow);
    __syncwarp();
    // a Gaussian is visible for sparse Adam when it touches a tile in any view
    const unsigned vis = __ballot_sync(0xffffffffu, a.sparse && valid && visible_any(b, g));
    // coalesced Adam over the warp's rows of means, log-scales and SH
    const float bc1 = a.bias ? a.bias[0] : a.inv_bc1, bc2 = a.bias ? a.bias[1] : a.inv_bc2;
    uintptr_t al = 0;
#pragma unroll
    for (int t = 0; t < 2; ++t)
        al |= reinterpret_cast<uintptr_t>(a.p[t]) | reinterpret_cast<uintptr_t>(a.m[t]) |
              reinterpret_cast<uintptr_t>(a.v[t]);
    const bool grouped = rows == 32 && !a.sparse && (al & 15) == 0;
    float4 q_new = make_float4(0.f, 0.f, 0.f, 0.f);
    float logit_new = 0.0f;
    if (grouped) {
        adam_small_rows(a, g0, g, s_gms, gq, glogit, bc1, bc2, lane, q_new, logit_new);
    } else {
        adam_segment<3, 7, NEXT>(a, 0, g0, rows, s_gms, 0, vis, bc1, bc2, lane, nullptr, 0);
        adam_segment<3, 7, NEXT>(a, 1, g0, rows, s_gms, 3, vis, bc1, bc2, lane, nullptr, 0);
    }
    if (a.lowp) {
        // the SH parameters are sh_store itself: each warp writes only the rows it staged
        const uint32_t sr = sr_base(a.sr_seed, a.step_dev ? (uint32_t)*a.step_dev : (uint32_t)a.step);
        adam_segment_lowp<F::KW, F::GS, DT, NEXT>(a, g0, rows, s_gsh, vis, bc1, bc2, lane,
                                                  const_cast<void*>(sh_store), sr);
    } else {
        adam_segment<F::KW, F::GS, NEXT>(a, 4, g0, rows, s_gsh, 0, vis, bc1, bc2, lane, a.shadow, a.shadow_dtype);
    }
    if (!grouped) adam_quat_logit(a, g, valid, vis, gq, glogit, bc1, bc2, lane, q_new, logit_new);
    if constexpr (NEXT) {
        // the next step's projection from the updated values in the gradient slots
        __syncwarp();
        if (valid) {
            float mean[3], ls[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                mean[j] = grow[j];
                ls[j] = grow[3 + j];
            }
            // project_one, with the SH coefficients read only for a Gaussian the view keeps
            // (as in k_project: they are live for its colour alone)
            Proj P;
            project_geometry<DEG>(nv.cam, nv.dil, mean, ls, q_new, logit_new, P);
            if (!P.culled) {
                float c[16][3];
                if constexpr (F::VEC) {
                    row_load_vec<(DEG + 1) * (DEG + 1)>(gshrow, c);
                } else {
#pragma unroll
                    for (int k = 0; k < (DEG + 1) * (DEG + 1); ++k)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) c[k][ch] = gshrow[3 * k + ch];
                }
                sh_colour<DEG>(nv.cam, mean, c, P.dir, P.inv_vlen, P.rgb_raw);
            }
            write_projection(nv, g, P);
        }
    }
}


// Advances the device-side Adam step and writes the bias corrections of the
// new step, evaluated in double like the host path.
__global__ void k_adam_advance(int* step, float b1, float b2, float* bias)
{
    kernel_prologue();
    const int t = *step + 1;
    *step = t;
    bias[0] = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
    bias[1] = (float)(1.0 / (1.0 - pow((double)b2, (double)t)));
}

__global__ void k_densify(int n, const int* __restrict__ tiles_touched, const float4* __restrict__ grad2d,
                          float* __restrict__ pos_acc, float* __restrict__ col_acc, int* __restrict__ count)
{
    kernel_prologue();
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n || tiles_touched[g] <= 0) return;
    float4 G0 = grad2d[3 * (int64_t)g], G1 = grad2d[3 * (int64_t)g + 1], G2 = grad2d[3 * (int64_t)g + 2];
    pos_acc[g] += sqrtf(G0.x * G0.x + G0.y * G0.y);
    col_acc[g] += sqrtf(G1.z * G1.z + G1.w * G1.w + G2.x * G2.x);
    count[g] += 1;
}

// ---------------------------------------------------------------------------
// Dispatch over (degree, dtype)
// ---------------------------------------------------------------------------
template <int DEG, int DT>
int32_t launch_project(int n, const float* means, const float* log_scales, const float* quats, const float* logits,
                       const void* sh, const Batch& b, cudaStream_t st)
{
    using L = ShLayout<DEG, DT>;
    size_t smem = sizeof(uint32_t) * L::WARP_WORDS * kWarps;
    auto kern = b.nviews > 1 ? k_project<DEG, DT, true> : k_project<DEG, DT, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int blocks = (n + kThreads - 1) / kThreads;
    gs::launch(kern, blocks, kThreads, smem, st, n, means, log_scales, reinterpret_cast<const float4*>(quats), logits,
               sh, b);
    return gs_host::check_launch("gs_project");
}

template <int DEG, int DT>
int32_t launch_project_bwd(int n, const float* means, const float* log_scales, const float* quats,
                           const float* logits, const void* sh, const Cam& cam, const Dil& dil,
                           const int* tiles, const float* grad2d, float* d_means, float* d_ls, float* d_q,
                           float* d_logits, float* d_sh, float* pos, float* col, int* cnt, cudaStream_t st)
{
    using L = ShLayout<DEG, DT>;
    size_t smem = sizeof(uint32_t) * L::WARP_WORDS * kWarps;
    auto kern = k_project_bwd<DEG, DT>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int blocks = (n + kThreads - 1) / kThreads;
    gs::launch_serial(kern, blocks, kThreads, smem, st, n, means, log_scales, reinterpret_cast<const float4*>(quats),
                      logits, sh, cam, dil, tiles, reinterpret_cast<const float4*>(grad2d), d_means, d_ls,
                      reinterpret_cast<float4*>(d_q), d_logits, d_sh, pos, col, cnt);
    return gs_host::check_launch("gs_project_bwd");
}

template <int DEG, int DT>
int32_t launch_project_bwd_adam(int n, const void* sh_store, const Batch& b, const AdamDev& a, float* pos, float* col,
                                int* cnt, const ViewDev* next, cudaStream_t st)
{
    const bool multi = !next && b.nviews > 1;
    size_t smem = sizeof(uint32_t) * kWarps *
                  (multi ? FusedLayout<DEG, DT, true>::WARP_WORDS : FusedLayout<DEG, DT, false>::WARP_WORDS);
    auto kern = next ? k_project_bwd_adam<DEG, DT, false, true>
                     : (multi ? k_project_bwd_adam<DEG, DT, true> : k_project_bwd_adam<DEG, DT, false>);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int blocks = (n + kThreads - 1) / kThreads;
    const ViewDev nv = next ? *next : ViewDev{};
    gs::launch_serial(kern, blocks, kThreads, smem, st, n, sh_store, b, a, pos, col, cnt, nv);
    return gs_host::check_launch("gs_project_bwd_adam");
}

#define GS_DISPATCH_DEG_DT(deg, dt, FN, ...)                                                          \
    switch ((deg) * 3 + (dt)) {                                                                       \
        case 0: return FN<0, GS_DTYPE_F32>(__VA_ARGS__);                                              \
        case 1: return FN<0, GS_DTYPE_BF16>(__VA_ARGS__);                                             \
        case 2: return FN<0, GS_DTYPE_F16>(__VA_ARGS__);                                              \
        case 3: return FN<1, GS_DTYPE_F32>(__VA_ARGS__);                                              \
        case 4: return FN<1, GS_DTYPE_BF16>(__VA_ARGS__);                                             \
        case 5: return FN<1, GS_DTYPE_F16>(__VA_ARGS__);                                              \
        case 6: return FN<2, GS_DTYPE_F32>(__VA_ARGS__);                                              \
        case 7: return FN<2, GS_DTYPE_BF16>(__VA_ARGS__);                                             \
        case 8: return FN<2, GS_DTYPE_F16>(__VA_ARGS__);                                              \
        case 9: return FN<3, GS_DTYPE_F32>(__VA_ARGS__);                                              \
        case 10: return FN<3, GS_DTYPE_BF16>(__VA_ARGS__);                                            \
        default: return FN<3, GS_DTYPE_F16>(__VA_ARGS__);                                             \
    }

bool check_params(int32_t n, int32_t sh_degree, int32_t sh_dtype, const void* a, const void* b, const void* c,
                  const void* d, const void* e)
{
    if (n < 0) { gs_host::set_error("n must be >= 0"); return false; }
    if (sh_degree < 0 || sh_degree > 3) { gs_host::set_error("sh_degree must be in 0..3"); return false; }
    if (sh_dtype < GS_DTYPE_F32 || sh_dtype > GS_DTYPE_F16) { gs_host::set_error("bad sh_dtype"); return false; }
    if (n > 0 && (!a || !b || !c || !d || !e)) { gs_host::set_error("null parameter pointer"); return false; }
    if (n > 0 && ((reinterpret_cast<uintptr_t>(c) & 15) != 0)) {
        gs_host::set_error("quats must be 16-byte aligned");
        return false;
    }
    return true;
}

}  // namespace
}  // namespace gs

extern "C" {

int32_t gs_project(int32_t n, int32_t sh_degree, int32_t sh_dtype, const float* means, const float* log_scales,
                   const float* quats, const float* opacity_logits, const void* sh, const GsCamera* cam,
                   const GsDilation* dil, float* splats, int32_t* radii, int32_t* rects, int32_t* tiles_touched,
                   uint32_t* depth_keys, gs_stream_t stream)
{
    if (!cam || !dil) { gs_host::set_error("gs_project: camera or dilation is null"); return GS_ERR_ARG; }
    GsView v{};
    v.cam = *cam;
    v.dil = *dil;
    v.splats = splats;
    v.radii = radii;
    v.rects = rects;
    v.tiles_touched = tiles_touched;
    v.depth_keys = depth_keys;
    return gs_project_batch(n, sh_degree, sh_dtype, means, log_scales, quats, opacity_logits, sh, &v, 1, stream);
}

int32_t gs_project_batch(int32_t n, int32_t sh_degree, int32_t sh_dtype, const float* means, const float* log_scales,
                         const float* quats, const float* opacity_logits, const void* sh, const GsView* views,
                         int32_t nviews, gs_stream_t stream)
{
    using namespace gs;
    if (!check_params(n, sh_degree, sh_dtype, means, log_scales, quats, opacity_logits, sh)) return GS_ERR_ARG;
    Batch b;
    if (!gs_host::make_batch(views, nviews, &b)) return GS_ERR_ARG;
    for (int i = 0; i < nviews && n > 0; ++i) {
        const ViewDev& v = b.v[i];
        if (!v.splats || !v.radii || !v.rects || !v.tiles) {
            gs_host::set_error("gs_project: null output pointer");
            return GS_ERR_ARG;
        }
        if (((reinterpret_cast<uintptr_t>(v.splats) | reinterpret_cast<uintptr_t>(v.rects)) & 15) != 0) {
            gs_host::set_error("gs_project: splats and rects must be 16-byte aligned");
            return GS_ERR_ARG;
        }
    }
    if (n == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GS_DISPATCH_DEG_DT(sh_degree, sh_dtype, launch_project, n, means, log_scales, quats, opacity_logits, sh, b, st);
}

int32_t gs_project_bwd(int32_t n, int32_t sh_degree, int32_t sh_dtype, const float* means, const float* log_scales,
                       const float* quats, const float* opacity_logits, const void* sh, const GsCamera* cam,
                       const GsDilation* dil, const int32_t* tiles_touched, const float* grad2d, float* d_means,
                       float* d_log_scales, float* d_quats, float* d_opacity_logits, float* d_sh, float* pos_acc,
                       float* col_acc, int32_t* count, gs_stream_t stream)
{
    using namespace gs;
    if (!check_params(n, sh_degree, sh_dtype, means, log_scales, quats, opacity_logits, sh)) return GS_ERR_ARG;
    Cam c;
    Dil d;
    if (!gs_host::make_cam(cam, &c) || !gs_host::make_dil(cam, dil, &d)) return GS_ERR_ARG;
    if (n > 0 && (!tiles_touched || !grad2d || !d_means || !d_log_scales || !d_quats || !d_opacity_logits || !d_sh)) {
        gs_host::set_error("gs_project_bwd: null pointer");
        return GS_ERR_ARG;
    }
    if ((pos_acc == nullptr) != (col_acc == nullptr) || (pos_acc == nullptr) != (count == nullptr)) {
        gs_host::set_error("gs_project_bwd: pos_acc, col_acc and count must be all null or all set");
        return GS_ERR_ARG;
    }
    if (n > 0 && (((reinterpret_cast<uintptr_t>(grad2d) | reinterpret_cast<uintptr_t>(d_quats)) & 15) != 0)) {
        gs_host::set_error("gs_project_bwd: grad2d and d_quats must be 16-byte aligned");
        return GS_ERR_ARG;
    }
    if (n == 0) return GS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GS_DISPATCH_DEG_DT(sh_degree, sh_dtype, launch_project_bwd, n, means, log_scales, quats, opacity_logits, sh, c,
                       d, tiles_touched, grad2d, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, pos_acc,
                       col_acc, count, st);
}

int32_t gs_project_bwd_adam(int32_t n, int32_t sh_degree, int32_t sh_dtype, const void* sh_store, const GsCamera* cam,
                            const GsDilation* dil, const int32_t* tiles_touched, const float* grad2d,
                            const GsAdamParams* adam, float* pos_acc, float* col_acc, int32_t* count,
                            float* const* grads_out, gs_stream_t stream)
{
    if (!cam || !dil) { gs_host::set_error("gs_project_bwd_adam: camera or dilation is null"); return GS_ERR_ARG; }
    GsView v{};
    v.cam = *cam;
    v.dil = *dil;
    v.tiles_touched = const_cast<int32_t*>(tiles_touched);
    v.grad2d = const_cast<float*>(grad2d);
    return gs_project_bwd_adam_batch(n, sh_degree, sh_dtype, sh_store, &v, 1, adam, pos_acc, col_acc, count,
                                     grads_out, stream);
}

// The fused pass of gs_project_bwd_adam(_batch), and with next (one view, dense
// Adam) the next step's projection of the updated parameters.
static int32_t project_bwd_adam(int32_t n, int32_t sh_degree, int32_t sh_dtype, const void* sh_store,
                                const GsView* views, int32_t nviews, const GsAdamParams* adam, float* pos_acc,
                                float* col_acc, int32_t* count, float* const* grads_out, const GsView* next,
                                gs_stream_t stream)
{
    using namespace gs;
    if (!adam) { gs_host::set_error("gs_project_bwd_adam: adam is null"); return GS_ERR_ARG; }
    if (!check_params(n, sh_degree, sh_dtype, adam->param[0], adam->param[1], adam->param[2], adam->param[3],
                      sh_store))
        return GS_ERR_ARG;
    Batch b;
    if (!gs_host::make_batch(views, nviews, &b)) return GS_ERR_ARG;
    Batch nb{};
    if (next) {
        if (nviews != 1 || adam->sparse) {
            gs_host::set_error("gs_project_bwd_adam: the next view's projection needs one view and dense Adam");
            return GS_ERR_ARG;
        }
        if (!gs_host::make_batch(next, 1, &nb)) return GS_ERR_ARG;
        const ViewDev& v = nb.v[0];
        if (n > 0 && (!v.splats || !v.radii || !v.rects || !v.tiles ||
                      (reinterpret_cast<uintptr_t>(v.splats) & 15) != 0 ||
                      (reinterpret_cast<uintptr_t>(v.rects) & 15) != 0)) {
            gs_host::set_error("gs_project_bwd_adam: the next view needs 16-byte aligned splats and rects, radii "
                               "and tiles_touched");
            return GS_ERR_ARG;
        }
    }
    if (n > 0) {
        for (int t = 0; t < 5; ++t)
            if ((!adam->param[t] && t < 4) || !adam->m[t] || !adam->v[t]) {
                gs_host::set_error("gs_project_bwd_adam: null parameter or moment pointer");
                return GS_ERR_ARG;
            }
        uintptr_t al = reinterpret_cast<uintptr_t>(adam->param[2]) | reinterpret_cast<uintptr_t>(adam->m[2]) |
                       reinterpret_cast<uintptr_t>(adam->v[2]);
        if (grads_out && grads_out[2]) al |= reinterpret_cast<uintptr_t>(grads_out[2]);
        for (int i = 0; i < nviews; ++i) {
            if (!b.v[i].tiles || !b.v[i].grad2d) {
                gs_host::set_error("gs_project_bwd_adam: null tiles_touched or grad2d");
                return GS_ERR_ARG;
            }
            al |= reinterpret_cast<uintptr_t>(b.v[i].grad2d);
        }
        if ((al & 15) != 0) {
            gs_host::set_error("gs_project_bwd_adam: grad2d and the quaternion tensors must be 16-byte aligned");
            return GS_ERR_ARG;
        }
    }
    if ((pos_acc == nullptr) != (col_acc == nullptr) || (pos_acc == nullptr) != (count == nullptr)) {
        gs_host::set_error("gs_project_bwd_adam: pos_acc, col_acc and count must be all null or all set");
        return GS_ERR_ARG;
    }
    if ((!adam->bias_dev && adam->step < 1) || !(adam->beta1 >= 0.0f && adam->beta1 < 1.0f) ||
        !(adam->beta2 >= 0.0f && adam->beta2 < 1.0f) || !(adam->eps >= 0.0f) ||
        (adam->sh_shadow && (adam->sh_shadow_dtype < GS_DTYPE_F32 || adam->sh_shadow_dtype > GS_DTYPE_F16))) {
        gs_host::set_error("gs_project_bwd_adam: need step >= 1, 0 <= beta < 1, eps >= 0, a valid shadow dtype");
        return GS_ERR_ARG;
    }
    // no FP32 SH parameter: the SH is sh_store itself (stochastic rounding when it is BF16/FP16)
    const bool lowp = adam->param[4] == nullptr && sh_dtype != GS_DTYPE_F32;
    if (lowp && adam->sh_shadow) {
        gs_host::set_error("gs_project_bwd_adam: SH kept only in sh_store (param[4] NULL) takes no sh_shadow");
        return GS_ERR_ARG;
    }
    if (n == 0) return GS_OK;
    AdamDev a{};
    for (int t = 0; t < 5; ++t) {
        a.p[t] = adam->param[t];
        a.m[t] = adam->m[t];
        a.v[t] = adam->v[t];
        a.lr[t] = adam->lr[t];
        a.gout[t] = grads_out ? grads_out[t] : nullptr;
    }
    a.b1 = adam->beta1; a.b2 = adam->beta2; a.eps = adam->eps;
    if (adam->bias_dev) {
        a.bias = adam->bias_dev;
    } else {
        a.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)adam->beta1, (double)adam->step)));
        a.inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)adam->beta2, (double)adam->step)));
    }
    a.sparse = adam->sparse;
    a.shadow = adam->sh_shadow;
    a.shadow_dtype = adam->sh_shadow_dtype;
    if (!a.p[4] && !lowp) a.p[4] = static_cast<float*>(const_cast<void*>(sh_store));
    a.lowp = lowp ? 1 : 0;
    a.sr_seed = adam->sr_seed;
    a.step = adam->step;
    a.step_dev = adam->step_dev;
    const ViewDev* nv = next ? &nb.v[0] : nullptr;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    GS_DISPATCH_DEG_DT(sh_degree, sh_dtype, launch_project_bwd_adam, n, sh_store, b, a, pos_acc, col_acc, count, nv,
                       st);
}

int32_t gs_project_bwd_adam_batch(int32_t n, int32_t sh_degree, int32_t sh_dtype, const void* sh_store,
                                  const GsView* views, int32_t nviews, const GsAdamParams* adam, float* pos_acc,
                                  float* col_acc, int32_t* count, float* const* grads_out, gs_stream_t stream)
{
    return project_bwd_adam(n, sh_degree, sh_dtype, sh_store, views, nviews, adam, pos_acc, col_acc, count,
                            grads_out, nullptr, stream);
}

int32_t gs_project_bwd_adam_next(int32_t n, int32_t sh_degree, int32_t sh_dtype, const void* sh_store,
                                 const GsCamera* cam, const GsDilation* dil, const int32_t* tiles_touched,
                                 const float* grad2d, const GsAdamParams* adam, float* pos_acc, float* col_acc,
                                 int32_t* count, float* const* grads_out, const GsView* next, gs_stream_t stream)
{
    if (!cam || !dil || !next) {
        gs_host::set_error("gs_project_bwd_adam_next: camera, dilation or next view is null");
        return GS_ERR_ARG;
    }
    GsView v{};
    v.cam = *cam;
    v.dil = *dil;
    v.tiles_touched = const_cast<int32_t*>(tiles_touched);
    v.grad2d = const_cast<float*>(grad2d);
    return project_bwd_adam(n, sh_degree, sh_dtype, sh_store, &v, 1, adam, pos_acc, col_acc, count, grads_out, next,
                            stream);
}

int32_t gs_adam_advance(int32_t* step_dev, float beta1, float beta2, float* bias_dev, gs_stream_t stream)
{
    if (!step_dev || !bias_dev || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f)) {
        gs_host::set_error("gs_adam_advance: need device step and bias pointers and 0 <= beta < 1");
        return GS_ERR_ARG;
    }
    gs::launch(gs::k_adam_advance, 1, 1, 0, reinterpret_cast<cudaStream_t>(stream), step_dev, beta1, beta2, bias_dev);
    return gs_host::check_launch("gs_adam_advance");
}

int32_t gs_densify_stats(int32_t n, const int32_t* tiles_touched, const float* grad2d, float* pos_acc,
                         float* col_acc, int32_t* count, gs_stream_t stream)
{
    if (n < 0) { gs_host::set_error("n must be >= 0"); return GS_ERR_ARG; }
    if (n > 0 && (!tiles_touched || !grad2d || !pos_acc || !col_acc || !count)) {
        gs_host::set_error("gs_densify_stats: null pointer");
        return GS_ERR_ARG;
    }
    if (n > 0 && (reinterpret_cast<uintptr_t>(grad2d) & 15) != 0) {
        gs_host::set_error("gs_densify_stats: grad2d must be 16-byte aligned");
        return GS_ERR_ARG;
    }
    if (n == 0) return GS_OK;
    gs::launch(gs::k_densify, (n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream), n, tiles_touched,
               reinterpret_cast<const float4*>(grad2d), pos_acc, col_acc, count);
    return gs_host::check_launch("gs_densify_stats");
}

}  // extern "C"
