// gs_adam.cu -- fused multi-tensor Adam step (Kingma & Ba; the optimizer the
// fitting of Sec. 4.1 runs), one launch for every parameter tensor of the
// Gaussians. Memory-bound: 4 reads + 3 writes of 4 bytes per element, moved
// with 16-byte vector accesses where the tensor allows it.
#include <cmath>

#include "gs_common.cuh"

namespace gs {
namespace {

struct AdamTensorDev {
    float* p;
    const float* g;
    float* m;
    float* v;
    void* shadow;
    int64_t numel;
    int32_t row_width;
    int32_t shadow_dtype;
    float lr;
    int32_t vec4;  // all pointers 16-byte aligned and numel % 4 == 0
    int32_t lowp;  // the parameter is `shadow` itself (BF16/FP16), rounded stochastically
    uint32_t sr;   // stream of the stochastic rounding (sr_base of the seed and the step)
};

struct AdamArgs {
    AdamTensorDev t[GS_ADAM_MAX_TENSORS];
    float b1, b2, eps, inv_bc1, inv_bc2;
    const uint8_t* row_mask;
};

__device__ __forceinline__ void adam_elem(float& p, float g, float& m, float& v, const AdamArgs& a, float lr)
{
    adam_step(p, g, m, v, a.b1, a.b2, a.eps, a.inv_bc1, a.inv_bc2, lr);
}

__device__ __forceinline__ void store_shadow(void* shadow, int dtype, int64_t e, float val)
{
    store_as(shadow, dtype, e, val);
}

__global__ void __launch_bounds__(256) k_adam(AdamArgs a)
{
    kernel_prologue();
    const AdamTensorDev& T = a.t[blockIdx.y];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (T.lowp) {
        // parameter kept only in 16 bits: FP32 update of the stored value, stochastic rounding
        uint16_t* P = reinterpret_cast<uint16_t*>(T.shadow);
        for (int64_t e = tid; e < T.numel; e += stride) {
            if (a.row_mask && !a.row_mask[e / T.row_width]) continue;
            float p = load_sh_elem(P, e, T.shadow_dtype), m = T.m[e], v = T.v[e];
            adam_elem(p, T.g[e], m, v, a, T.lr);
            P[e] = sr_round(p, sr_bits16(T.sr, (uint32_t)e), T.shadow_dtype);
            T.m[e] = m;
            T.v[e] = v;
        }
        return;
    }
    if (T.vec4) {
        const int64_t n4 = T.numel / 4;
        for (int64_t i = tid; i < n4; i += stride) {
            float4 p = reinterpret_cast<float4*>(T.p)[i];
            const float4 g = reinterpret_cast<const float4*>(T.g)[i];
            float4 m = reinterpret_cast<float4*>(T.m)[i];
            float4 v = reinterpret_cast<float4*>(T.v)[i];
            float* pp = &p.x;
            const float* gg = &g.x;
            float* mm = &m.x;
            float* vv = &v.x;
            bool any = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t e = 4 * i + k;
                if (a.row_mask && !a.row_mask[e / T.row_width]) continue;
                adam_elem(pp[k], gg[k], mm[k], vv[k], a, T.lr);
                any = true;
            }
            if (!any) continue;
            reinterpret_cast<float4*>(T.p)[i] = p;
            reinterpret_cast<float4*>(T.m)[i] = m;
            reinterpret_cast<float4*>(T.v)[i] = v;
            if (T.shadow) {
#pragma unroll
                for (int k = 0; k < 4; ++k) store_shadow(T.shadow, T.shadow_dtype, 4 * i + k, pp[k]);
            }
        }
    } else {
        for (int64_t e = tid; e < T.numel; e += stride) {
            if (a.row_mask && !a.row_mask[e / T.row_width]) continue;
            float p = T.p[e], m = T.m[e], v = T.v[e];
            adam_elem(p, T.g[e], m, v, a, T.lr);
            T.p[e] = p;
            T.m[e] = m;
            T.v[e] = v;
            if (T.shadow) store_shadow(T.shadow, T.shadow_dtype, e, p);
        }
    }
}

}  // namespace
}  // namespace gs

extern "C" {

int32_t gs_adam(const GsAdamTensor* tensors, int32_t count, float beta1, float beta2, float eps, int32_t step,
                const uint8_t* row_mask, gs_stream_t stream)
{
    using namespace gs;
    if (count < 0 || count > GS_ADAM_MAX_TENSORS || (count > 0 && !tensors)) {
        gs_host::set_error("gs_adam: count must be in 0..GS_ADAM_MAX_TENSORS");
        return GS_ERR_ARG;
    }
    if (step < 1 || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f)) {
        gs_host::set_error("gs_adam: need step >= 1, 0 <= beta < 1, eps >= 0");
        return GS_ERR_ARG;
    }
    AdamArgs a{};
    int64_t max_work = 0;
    for (int i = 0; i < count; ++i) {
        const GsAdamTensor& t = tensors[i];
        const bool lowp = !t.param && t.shadow != nullptr;
        if (t.numel < 0 || t.row_width < 1 ||
            (t.numel > 0 && ((!t.param && !lowp) || !t.grad || !t.m || !t.v)) ||
            (t.shadow && (t.shadow_dtype < GS_DTYPE_F32 || t.shadow_dtype > GS_DTYPE_F16)) ||
            (lowp && t.shadow_dtype == GS_DTYPE_F32)) {
            gs_host::set_error("gs_adam: bad tensor entry (a parameter kept only in `shadow` must be BF16/FP16)");
            return GS_ERR_ARG;
        }
        AdamTensorDev& d = a.t[i];
        d.p = t.param; d.g = t.grad; d.m = t.m; d.v = t.v; d.shadow = t.shadow;
        d.numel = t.numel; d.row_width = t.row_width; d.shadow_dtype = t.shadow_dtype; d.lr = t.lr;
        d.lowp = lowp ? 1 : 0;
        d.sr = sr_base(t.sr_seed, (uint32_t)step);
        uintptr_t al = reinterpret_cast<uintptr_t>(t.param) | reinterpret_cast<uintptr_t>(t.grad) |
                       reinterpret_cast<uintptr_t>(t.m) | reinterpret_cast<uintptr_t>(t.v);
        d.vec4 = ((al & 15) == 0) && (t.numel % 4 == 0);
        int64_t work = d.vec4 ? t.numel / 4 : t.numel;
        if (work > max_work) max_work = work;
    }
    if (count == 0 || max_work == 0) return GS_OK;
    a.b1 = beta1; a.b2 = beta2; a.eps = eps;
    a.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)step)));
    a.inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)step)));
    a.row_mask = row_mask;
    int64_t bx = (max_work + 255) / 256;
    const int64_t bmax = (int64_t)gs_host::sm_count() * 8;
    if (bx > bmax) bx = bmax;
    dim3 grid((unsigned)bx, (unsigned)count);
    gs::launch(k_adam, grid, 256, 0, reinterpret_cast<cudaStream_t>(stream), a);
    return gs_host::check_launch("gs_adam");
}

}  // extern "C"
