// gs_ssim.cu -- SSIM (the structural-similarity index of Wang et al. 2004 that
// the paper reports beside PSNR, Sec. 4 metrics) of the rendered lattice image
// against the hr target sampled at the same pixels, its gradient, and the
// L1 + D-SSIM loss of the 3DGS fitting the method builds on.
//
// Per channel, at every lattice pixel p: the Gaussian-window sums (11 x 11,
// sigma 1.5, weights summing to 1) m_x, m_y, E_xx, E_yy, E_xy, then
//   SSIM_p = (2 m_x m_y + C1)(2 (E_xy - m_x m_y) + C2)
//            / ((m_x^2 + m_y^2 + C1)(E_xx - m_x^2 + E_yy - m_y^2 + C2)),
// C1 = 0.01^2, C2 = 0.03^2. Mode 0 ("valid") averages the pixels whose window
// lies inside the image; mode 1 ("same") all pixels, with zeros outside.
//
// Two tiled passes, each a separable window sum through shared memory: the
// forward computes the five sums, SSIM and its partial derivatives in
// (m_x, E_xx, E_xy) per pixel (into the workspace); the backward spreads the
// partials back over each window (the same symmetric filter) and chains them
// through dE_xx/dx = 2x and dE_xy/dx = y. Memory-bound: 24 B in and 36 B of
// partials out per pixel, then 36 + 24 B in and 12 B out.
#include "gs_common.cuh"

namespace gs {
namespace {

constexpr int kR = 5;                    // window radius: 11 taps
constexpr int kTaps = 2 * kR + 1;
constexpr int kTW = 32, kTH = 16;        // output pixels of a CTA
constexpr int kIW = kTW + 2 * kR, kIH = kTH + 2 * kR;
constexpr int kSsimThreads = 256;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// The normalised 1-D window (sigma 1.5), computed once per CTA.
__device__ __forceinline__ void window_weights(float* w)
{
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < kTaps; ++i) {
            const float r = (float)(i - kR);
            w[i] = expf(-r * r / (2.0f * 1.5f * 1.5f));
            s += w[i];
        }
        for (int i = 0; i < kTaps; ++i) w[i] /= s;
    }
    __syncthreads();
}

struct Lattice {
    int w, h;          // lattice image
    int d, ox, oy;     // hr pixel of lattice (u, v): (d u + ox, d v + oy)
    int width;         // hr width (target row stride)
    int mode;          // 0 valid, 1 same
    int target_dtype;  // GS_TARGET_F32 or GS_TARGET_U8
    float inv_n;       // 1 / (3 * pixels averaged)
    float inv_p3;      // 1 / (3 * lattice pixels): the L1 mean
};

__device__ __forceinline__ bool counted(const Lattice& L, int u, int v)
{
    return L.mode == 1 ? true : (u >= kR && u < L.w - kR && v >= kR && v < L.h - kR);
}

__device__ __forceinline__ float target_at(const Lattice& L, const void* t, int u, int v, int c)
{
    const int64_t i = ((int64_t)(L.d * v + L.oy) * L.width + (L.d * u + L.ox)) * 3 + c;
    return L.target_dtype == GS_TARGET_U8 ? target_value<GS_TARGET_U8>(t, i) : target_value<GS_TARGET_F32>(t, i);
}

// Forward: per channel, the window sums of the CTA's output tile, SSIM and its
// partials (scaled by the mean's 1/N) into part[pix][c][0..2] (zero for a
// pixel the mean leaves out); sums of SSIM and |x - y| into acc[0], acc[1].
__global__ void __launch_bounds__(kSsimThreads)
k_ssim_fwd(Lattice L, const float* __restrict__ img, const void* __restrict__ target, float* __restrict__ part,
           double* __restrict__ acc)
{
    kernel_prologue();
    __shared__ float s_w[kTaps];
    __shared__ float s_x[kIH][kIW], s_y[kIH][kIW];
    __shared__ float s_h[5][kIH][kTW];
    __shared__ float s_red[2][kSsimThreads / 32];
    window_weights(s_w);
    const int u0 = blockIdx.x * kTW, v0 = blockIdx.y * kTH;
    float sum_s = 0.0f, sum_l1 = 0.0f;
    for (int c = 0; c < 3; ++c) {
        for (int i = threadIdx.x; i < kIH * kIW; i += kSsimThreads) {
            const int r = i / kIW, q = i % kIW;
            const int u = u0 - kR + q, v = v0 - kR + r;
            const bool in = u >= 0 && u < L.w && v >= 0 && v < L.h;
            s_x[r][q] = in ? img[((int64_t)v * L.w + u) * 3 + c] : 0.0f;
            s_y[r][q] = in ? target_at(L, target, u, v, c) : 0.0f;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kIH * kTW; i += kSsimThreads) {
            const int r = i / kTW, q = i % kTW;
            float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
            for (int k = 0; k < kTaps; ++k) {
                const float a = s_x[r][q + k], b = s_y[r][q + k], wk = s_w[k];
                mx = fmaf(wk, a, mx);
                my = fmaf(wk, b, my);
                xx = fmaf(wk, a * a, xx);
                yy = fmaf(wk, b * b, yy);
                xy = fmaf(wk, a * b, xy);
            }
            s_h[0][r][q] = mx; s_h[1][r][q] = my; s_h[2][r][q] = xx; s_h[3][r][q] = yy; s_h[4][r][q] = xy;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kTH * kTW; i += kSsimThreads) {
            const int r = i / kTW, q = i % kTW;
            const int u = u0 + q, v = v0 + r;
            if (u >= L.w || v >= L.h) continue;
            float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < kTaps; ++k) {
                const float wk = s_w[k];
#pragma unroll
                for (int j = 0; j < 5; ++j) m[j] = fmaf(wk, s_h[j][r + k][q], m[j]);
            }
            const float mx = m[0], my = m[1];
            const float a1 = 2.0f * mx * my + kC1;
            const float a2 = 2.0f * (m[4] - mx * my) + kC2;
            const float b1 = mx * mx + my * my + kC1;
            const float b2 = (m[2] - mx * mx) + (m[3] - my * my) + kC2;
            const float inv_b = 1.0f / (b1 * b2);
            const float s = a1 * a2 * inv_b;
            const int64_t pix = (int64_t)v * L.w + u;
            float* pp = part + pix * 9 + 3 * c;
            const float x = s_x[r + kR][q + kR], y = s_y[r + kR][q + kR];
            sum_l1 += fabsf(x - y);
            if (counted(L, u, v)) {
                sum_s += s;
                pp[0] = L.inv_n * ((2.0f * my * a2 - 2.0f * my * a1) * inv_b - s * (2.0f * mx / b1 - 2.0f * mx / b2));
                pp[1] = L.inv_n * (-s / b2);
                pp[2] = L.inv_n * (2.0f * a1 * inv_b);
            } else {
                pp[0] = pp[1] = pp[2] = 0.0f;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum_s += __shfl_down_sync(0xffffffffu, sum_s, o);
        sum_l1 += __shfl_down_sync(0xffffffffu, sum_l1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = sum_s;
        s_red[1][threadIdx.x >> 5] = sum_l1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kSsimThreads / 32; ++w) {
            a += (double)s_red[0][w];
            b += (double)s_red[1][w];
        }
        atomicAdd(&acc[0], a);
        atomicAdd(&acc[1], b);
    }
}

// Backward: per channel, the window sums of the three partial maps around the
// CTA's tile (the adjoint of the forward's sums: the window is symmetric), then
//   g = S(d_mx) + 2 x S(d_exx) + y S(d_exy)   (d mean SSIM / d x).
// out = ssim_scale * g + l1_scale * sign(x - y) (l1_scale 0: the SSIM gradient
// alone).
__global__ void __launch_bounds__(kSsimThreads)
k_ssim_bwd(Lattice L, const float* __restrict__ img, const void* __restrict__ target,
           const float* __restrict__ part, float ssim_scale, float l1_scale, float* __restrict__ out)
{
    kernel_prologue();
    __shared__ float s_w[kTaps];
    __shared__ float s_p[3][kIH][kIW];
    __shared__ float s_h[3][kIH][kTW];
    window_weights(s_w);
    const int u0 = blockIdx.x * kTW, v0 = blockIdx.y * kTH;
    for (int c = 0; c < 3; ++c) {
        for (int i = threadIdx.x; i < kIH * kIW; i += kSsimThreads) {
            const int r = i / kIW, q = i % kIW;
            const int u = u0 - kR + q, v = v0 - kR + r;
            const bool in = u >= 0 && u < L.w && v >= 0 && v < L.h;
            const float* pp = part + ((int64_t)v * L.w + u) * 9 + 3 * c;
#pragma unroll
            for (int j = 0; j < 3; ++j) s_p[j][r][q] = in ? pp[j] : 0.0f;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kIH * kTW; i += kSsimThreads) {
            const int r = i / kTW, q = i % kTW;
            float h0 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll
            for (int k = 0; k < kTaps; ++k) {
                const float wk = s_w[k];
                h0 = fmaf(wk, s_p[0][r][q + k], h0);
                h1 = fmaf(wk, s_p[1][r][q + k], h1);
                h2 = fmaf(wk, s_p[2][r][q + k], h2);
            }
            s_h[0][r][q] = h0; s_h[1][r][q] = h1; s_h[2][r][q] = h2;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kTH * kTW; i += kSsimThreads) {
            const int r = i / kTW, q = i % kTW;
            const int u = u0 + q, v = v0 + r;
            if (u >= L.w || v >= L.h) continue;
            float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
            for (int k = 0; k < kTaps; ++k) {
                const float wk = s_w[k];
                g0 = fmaf(wk, s_h[0][r + k][q], g0);
                g1 = fmaf(wk, s_h[1][r + k][q], g1);
                g2 = fmaf(wk, s_h[2][r + k][q], g2);
            }
            const int64_t pix = (int64_t)v * L.w + u;
            const float x = img[pix * 3 + c], y = target_at(L, target, u, v, c);
            const float g = g0 + 2.0f * x * g1 + y * g2;
            const float d = x - y;
            const float sg = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
            out[pix * 3 + c] = ssim_scale * g + l1_scale * sg;
        }
        __syncthreads();
    }
}

// Mean SSIM, and (when loss is given) L = (1 - lambda) L1 + lambda (1 - SSIM).
__global__ void k_ssim_final(const double* __restrict__ acc, Lattice L, float lambda, float* __restrict__ ssim_out,
                             float* __restrict__ loss)
{
    kernel_prologue();
    const double s = acc[0] * (double)L.inv_n;
    const double l1 = acc[1] * (double)L.inv_p3;
    if (ssim_out) *ssim_out = (float)s;
    if (loss) *loss = (float)((1.0 - (double)lambda) * l1 + (double)lambda * (1.0 - s));
}

bool make_lattice(const GsCamera* cam, const GsDilation* dil, int mode, Lattice* L)
{
    Dil d;
    if (!gs_host::make_dil(cam, dil, &d)) return false;
    if (mode != 0 && mode != 1) {
        gs_host::set_error("ssim: mode must be 0 (valid) or 1 (same)");
        return false;
    }
    if (mode == 0 && (d.w_ds < kTaps || d.h_ds < kTaps)) {
        gs_host::set_error("ssim: the valid mode needs a lattice image of at least 11 x 11 pixels");
        return false;
    }
    L->w = d.w_ds; L->h = d.h_ds; L->d = d.d; L->ox = d.ox; L->oy = d.oy; L->width = cam->width; L->mode = mode;
    const double n = mode == 0 ? (double)(d.w_ds - 2 * kR) * (d.h_ds - 2 * kR) : (double)d.w_ds * d.h_ds;
    L->inv_n = (float)(1.0 / (3.0 * n));
    L->inv_p3 = (float)(1.0 / (3.0 * (double)d.w_ds * d.h_ds));
    return true;
}

size_t ssim_ws_bytes(const Lattice& L)
{
    return 256 + (((size_t)L.w * L.h * 9 * sizeof(float) + 255) & ~size_t(255));
}

int32_t run_ssim(const GsCamera* cam, const GsDilation* dil, const float* img, const void* target,
                 int32_t target_dtype, int32_t mode, float lambda, bool loss_form, float* ssim_out, float* loss,
                 float* grad, void* workspace, size_t workspace_bytes, gs_stream_t stream)
{
    Lattice L;
    if (!make_lattice(cam, dil, mode, &L)) return GS_ERR_ARG;
    if (!img || !target || !workspace) {
        gs_host::set_error("ssim: null image, target or workspace");
        return GS_ERR_ARG;
    }
    if (target_dtype != GS_TARGET_F32 && target_dtype != GS_TARGET_U8) {
        gs_host::set_error("ssim: target_dtype must be GS_TARGET_F32 or GS_TARGET_U8");
        return GS_ERR_ARG;
    }
    L.target_dtype = target_dtype;
    if (workspace_bytes < ssim_ws_bytes(L) || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
        gs_host::set_error("ssim: workspace too small or not 256-byte aligned");
        return GS_ERR_ARG;
    }
    double* acc = static_cast<double*>(workspace);
    float* part = reinterpret_cast<float*>(static_cast<char*>(workspace) + 256);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
    const dim3 grid((L.w + kTW - 1) / kTW, (L.h + kTH - 1) / kTH);
    gs::launch(k_ssim_fwd, grid, kSsimThreads, 0, st, L, img, target, part, acc);
    if (grad) {
        // loss form: d/dx [(1 - lambda) L1 + lambda (1 - SSIM)]; metric form: d SSIM / dx
        const float ss = loss_form ? -lambda : 1.0f;
        const float l1 = loss_form ? (1.0f - lambda) * L.inv_p3 : 0.0f;
        gs::launch(k_ssim_bwd, grid, kSsimThreads, 0, st, L, img, target, part, ss, l1, grad);
    }
    gs::launch(k_ssim_final, 1, 1, 0, st, acc, L, lambda, ssim_out, loss);
    return gs_host::check_launch(loss_form ? "gs_loss_l1_dssim" : "gs_ssim");
}

}  // namespace
}  // namespace gs

extern "C" {

size_t gs_ssim_workspace_size(const GsCamera* cam, const GsDilation* dil)
{
    gs::Lattice L;
    if (!gs::make_lattice(cam, dil, 1, &L)) return 0;
    return gs::ssim_ws_bytes(L);
}

int32_t gs_ssim(const GsCamera* cam, const GsDilation* dil, const float* img, const void* target,
                int32_t target_dtype, int32_t mode, float* ssim_out, float* d_img, void* workspace,
                size_t workspace_bytes, gs_stream_t stream)
{
    if (!ssim_out) {
        gs_host::set_error("gs_ssim: null output");
        return GS_ERR_ARG;
    }
    return gs::run_ssim(cam, dil, img, target, target_dtype, mode, 0.0f, false, ssim_out, nullptr, d_img, workspace,
                        workspace_bytes, stream);
}

int32_t gs_loss_l1_dssim(const GsCamera* cam, const GsDilation* dil, const float* img, const void* target,
                         int32_t target_dtype, float lambda, int32_t mode, float* dl_dimg, float* loss, void* workspace,
                         size_t workspace_bytes, gs_stream_t stream)
{
    if (!dl_dimg || !loss || !(lambda >= 0.0f && lambda <= 1.0f)) {
        gs_host::set_error("gs_loss_l1_dssim: null output or lambda outside [0, 1]");
        return GS_ERR_ARG;
    }
    return gs::run_ssim(cam, dil, img, target, target_dtype, mode, lambda, true, nullptr, loss, dl_dimg, workspace,
                        workspace_bytes, stream);
}

}  // extern "C"
