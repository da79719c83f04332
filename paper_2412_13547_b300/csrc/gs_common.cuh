// gs_common.cuh -- device-side helpers shared by the turbogs kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <utility>

#include "../../include/turbogs.h"

namespace gs {

// ---------------------------------------------------------------------------
// Launches. Every kernel of the library goes through gs::launch, which allows
// programmatic dependent launch: the kernel may be scheduled while its
// predecessor on the stream is still draining, and its first statement,
// kernel_prologue(), waits for that predecessor to complete with its memory
// visible (griddepcontrol.wait; a no-op when the predecessor was no kernel or
// was launched without the attribute) before anything is read or written.
// The prologue then lets the kernel's own successor be scheduled. Stream order
// and memory visibility are those of ordinary launches (each kernel starts
// its work only after every earlier one on the stream has completed); what
// goes is the idle gap between consecutive kernels, which for the chain of
// short binning kernels was about 8% of the stage. A kernel launched this way
// without the prologue would race its predecessor: every __global__ of the
// library begins with it (a CPU test checks the sources).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kernel_prologue()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(std::forward<Args>(args))...);
}

// An ordinary launch (no programmatic dependent launch) for the projection
// backward kernels, which follow the blend backward: launched early, their
// CTAs took up the SMs while the blend backward drained, and the step was
// 0.15 ms slower (2.60 instead of 2.44 ms at 4K). An SM changes its L1 /
// shared-memory split only when it is idle; the likely cause is that the
// streaming pass then ran in the blend's shared-memory-heavy split, with less
// L1 for the parameter rows it reads twice. The kernels keep the prologue (a
// no-op without the attribute).
template <typename... KArgs, typename... Args>
inline void launch_serial(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(std::forward<Args>(args))...);
}

// ---------------------------------------------------------------------------
// Constants of the method (Sec. 3 Eq. 2 early-stop rule; Sec. 3.1 low-pass).
// ---------------------------------------------------------------------------
constexpr float kLowPass = 0.3f;          // px^2 added to the 2D covariance diagonal
constexpr float kDiscFloor = 0.1f;        // floor of the eigenvalue discriminant
constexpr float kAlphaMax = 0.99f;        // alpha clamp
constexpr float kAlphaMin = 1.0f / 255.0f;  // alpha skip threshold
constexpr float kTStop = 1e-4f;           // stop before transmittance drops below
constexpr float kClampFov = 1.3f;         // Jacobian clamp, x the half field of view

// Device copies of the camera and dilation, passed by value to kernels.
struct Cam {
    float R[9];
    float T[3];
    float fx, fy, cx, cy;
    int width, height;
    float z_near;
    float lim_x, lim_y;   // clamp of t_x/t_z, t_y/t_z in the Jacobian
    float ccx, ccy, ccz;  // camera centre in world space, -R^T T
};

// Downsampled grid of a dilation. The blend works on tiles of `tile` pixels
// (tiles_x x tiles_y); the binning on tiles of tile << shift (bin_tiles_x x
// bin_tiles_y), whose lists each blend tile filters down to its own.
struct Dil {
    int d, ox, oy, mode, tile;
    int w_ds, h_ds, tiles_x, tiles_y;
    int shift, bin_tiles_x, bin_tiles_y;
};

// Binning tile of a blend tile.
__device__ __forceinline__ int bin_tile_of(const Dil& dil, int tile)
{
    const int tx = tile % dil.tiles_x, ty = tile / dil.tiles_x;
    return (ty >> dil.shift) * dil.bin_tiles_x + (tx >> dil.shift);
}

// One view of a batch, as the kernels see it.
struct ViewDev {
    Cam cam;
    Dil dil;
    float4* splats;
    int* radii;
    int4* rects;
    int* tiles;
    const uint32_t* ids;
    const uint2* ranges;
    float* img;
    float* t_final;
    uint32_t* last;
    const void* target;
    int target_dtype;  // GS_TARGET_F32 or GS_TARGET_U8
    float* dl;
    float4* grad2d;
    float* loss;
    uint32_t* keys;  // depth sort keys (nullable)
    int tile_begin;  // first global tile id of this view in the batch
};

// Element i of a target image as FP32: the value itself, or an 8-bit value t
// as t * (1/255) with 1/255 rounded to FP32.
constexpr float kInv255 = 1.0f / 255.0f;
template <int TD>
__device__ __forceinline__ float target_value(const void* t, int64_t i)
{
    if constexpr (TD == GS_TARGET_U8) return __fmul_rn((float)static_cast<const uint8_t*>(t)[i], kInv255);
    else return static_cast<const float*>(t)[i];
}

struct Batch {
    ViewDev v[GS_MAX_VIEWS];
    int nviews;
    int total_tiles;
};

// View of a global tile id (tiles numbered view by view).
__device__ __forceinline__ int view_of_tile(const Batch& b, int gt)
{
    int v = 0;
    for (int i = 1; i < b.nviews; ++i)
        if (b.v[i].tile_begin <= gt) v = i;
    return v;
}

// ---------------------------------------------------------------------------
// Float-float arithmetic (error-free transformations with FMA). Used to carry
// the hr image-plane centre with ~1e-6 px error at 4K, where plain FP32 loses
// ~1e-3 px and the steep edge of a small splat turns that into a visible error.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b)  // |a| >= |b|
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ ff two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, lo);
}

// sum_k a_k * b_k + c, accumulated in float-float
__device__ __forceinline__ ff ff_dot3_add(float a0, float b0, float a1, float b1, float a2, float b2,
                                          float c)
{
    ff acc = two_prod(a0, b0);
    acc = ff_add(acc, two_prod(a1, b1));
    acc = ff_add(acc, two_prod(a2, b2));
    acc = ff_add(acc, ff{c, 0.0f});
    return acc;
}

// a / b as float-float given rb ~ 1 / b.hi (a few ulp): the leading quotient's
// remainder is exact through the FMA, so the pair stays accurate to ~2^-46.
__device__ __forceinline__ ff ff_div_rcp(ff a, ff b, float rb)
{
    float q = __fmul_rn(a.hi, rb);
    float r = __fmaf_rn(-q, b.hi, a.hi);
    r = __fadd_rn(r, __fsub_rn(a.lo, __fmul_rn(q, b.lo)));
    float q2 = __fmul_rn(r, rb);
    return two_sum(q, q2);
}

// f * (u.hi + u.lo) + c as float-float (f, c exact floats)
__device__ __forceinline__ ff ff_affine(float f, ff u, float c)
{
    ff p = two_prod(f, u.hi);
    ff s = two_sum(p.hi, c);
    float lo = __fadd_rn(__fadd_rn(s.lo, p.lo), __fmul_rn(f, u.lo));
    return two_sum(s.hi, lo);
}

// Accurate a*d - b*c (Kahan's algorithm with FMA).
__device__ __forceinline__ float det2(float a, float b, float c, float d)
{
    float w = __fmul_rn(b, c);
    float e = __fmaf_rn(-b, c, w);
    float f = __fmaf_rn(a, d, -w);
    return __fadd_rn(f, e);
}

// ---------------------------------------------------------------------------
// The per-entry blend arithmetic, with rounding pinned by intrinsics so the
// forward pass and the backward replay take identical skip/clamp decisions.
// ---------------------------------------------------------------------------
// 2^x on the SFU (ex2.approx, flush to zero): with the conic pre-scaled by
// log2(e), G = exp(power) = 2^(power log2 e) is one SFU operation.
__device__ __forceinline__ float exp2_sfu(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two FP32 values in one 64-bit register pair, for the paired FP32
// instructions of sm_100 and later (add/sub/mul/fma.rn.f32x2): one instruction
// does the arithmetic of two pixels, each element rounded exactly as the
// scalar instruction would round it.
struct f32x2 {
    unsigned long long v;
};
__device__ __forceinline__ f32x2 pk(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpk(f32x2 a, float& x, float& y)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
}
__device__ __forceinline__ float pk_sum(f32x2 a)
{
    float x, y;
    unpk(a, x, y);
    return x + y;
}
// -(x + y) of the two halves, one add with both operands negated.
__device__ __forceinline__ float pk_sum_neg(f32x2 a)
{
    float x, y;
    unpk(a, x, y);
    return -x - y;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

constexpr float kLog2e = 1.44269504088896340736f;  // log2(e)
constexpr float kLn2 = 0.693147180559945309417f;    // ln(2) = 1 / log2(e)

constexpr float kLog2AlphaMin = -7.99435343685885793f;  // log2(1/255)

// The conic (A, B, C) and opacity o of a staged record as the terms of the
// base-2 logarithm of the splat's alpha: (a, b, c) = log2(e) (-A/2, -B, -C/2)
// and l = log2(o), so that
//   e2 = a dx^2 + b dx dy + c dy^2 + l = log2(o G),  G = exp(-(A dx^2 + C dy^2)/2 - B dx dy),
// and the alpha before the clamp is 2^e2. The alpha gates are then comparisons
// of e2: G <= 1 is e2 <= l, alpha >= 1/255 is e2 >= log2(1/255).
__device__ __forceinline__ float4 conic_exp2(float4 co)
{
    return make_float4(__fmul_rn(co.x, -0.5f * kLog2e), __fmul_rn(co.y, -kLog2e), __fmul_rn(co.z, -0.5f * kLog2e),
                       __log2f(co.w));
}

// e2 at pixel offset (dx, dy), in two parts: the terms of dx alone (a dx^2 + l
// and b dx, shared by the pixels of one column) and the rest per pixel. Every
// kernel evaluates it this way, rounding pinned with intrinsics, so the forward
// and the backward replay take the same gate decisions.
struct SplatRow {
    float adx2, bdx;
};

__device__ __forceinline__ SplatRow splat_row(float dx, float4 s)
{
    return SplatRow{__fadd_rn(__fmul_rn(s.x, __fmul_rn(dx, dx)), s.w), __fmul_rn(s.y, dx)};
}

__device__ __forceinline__ float splat_power(SplatRow r, float dy, float c)
{
    return __fmaf_rn(r.bdx, dy, __fmaf_rn(c, __fmul_rn(dy, dy), r.adx2));
}

// The gate of one pixel on e2 (above): the splat's Gaussian factor at most 1 and
// alpha at least 1/255.
__device__ __forceinline__ bool splat_gate(float e2, float l)
{
    return !(e2 > l) && !(e2 < kLog2AlphaMin);
}

// ---------------------------------------------------------------------------
// Real spherical harmonics up to degree 3 (Condon-Shortley phase, index
// l*l + l + m), written as Cartesian polynomials of the unit direction. The
// normalisation constants follow from sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!).
// ---------------------------------------------------------------------------
constexpr float kPi = 3.14159265358979323846f;

struct ShConst {
    float k0, k1, k2a, k2b, k2c, k3a, k3b, k3c, k3d, k3e;
};

__device__ __forceinline__ ShConst sh_const()
{
    ShConst c;
    c.k0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
    c.k1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
    c.k2a = 1.0925484305920792f;   // sqrt(15/pi)/2
    c.k2b = 0.31539156525252005f;  // sqrt(5/pi)/4
    c.k2c = 0.5462742152960396f;   // sqrt(15/pi)/4
    c.k3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
    c.k3b = 2.890611442640554f;    // sqrt(105/pi)/2
    c.k3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
    c.k3d = 0.3731763325901154f;   // sqrt(7/pi)/4
    c.k3e = 1.445305721320277f;    // sqrt(105/pi)/4
    return c;
}

// Basis values Y[0..(deg+1)^2) at the unit direction (x, y, z).
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y)
{
    // every operation rounded explicitly (no contraction left to the compiler), so the
    // forward projection and every backward pass that recomputes the colour agree bit for
    // bit, down to the clamp of a colour channel at zero
    const ShConst c = sh_const();
    Y[0] = c.k0;
    if (deg < 1) return;
    Y[1] = __fmul_rn(-c.k1, y);
    Y[2] = __fmul_rn(c.k1, z);
    Y[3] = __fmul_rn(-c.k1, x);
    if (deg < 2) return;
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    Y[4] = __fmul_rn(__fmul_rn(c.k2a, x), y);
    Y[5] = __fmul_rn(__fmul_rn(-c.k2a, y), z);
    Y[6] = __fmul_rn(c.k2b, __fsub_rn(__fsub_rn(__fmul_rn(2.0f, zz), xx), yy));
    Y[7] = __fmul_rn(__fmul_rn(-c.k2a, x), z);
    Y[8] = __fmul_rn(c.k2c, __fsub_rn(xx, yy));
    if (deg < 3) return;
    const float xx3 = __fmul_rn(3.0f, xx), yy3 = __fmul_rn(3.0f, yy);
    const float t4 = __fsub_rn(__fsub_rn(__fmul_rn(4.0f, zz), xx), yy);
    Y[9] = __fmul_rn(__fmul_rn(-c.k3a, y), __fsub_rn(xx3, yy));
    Y[10] = __fmul_rn(__fmul_rn(__fmul_rn(c.k3b, x), y), z);
    Y[11] = __fmul_rn(__fmul_rn(-c.k3c, y), t4);
    Y[12] = __fmul_rn(__fmul_rn(c.k3d, z), __fsub_rn(__fsub_rn(__fmul_rn(2.0f, zz), xx3), yy3));
    Y[13] = __fmul_rn(__fmul_rn(-c.k3c, x), t4);
    Y[14] = __fmul_rn(__fmul_rn(c.k3e, z), __fsub_rn(xx, yy));
    Y[15] = __fmul_rn(__fmul_rn(-c.k3a, x), __fsub_rn(xx, yy3));
}

// Gradient of sum_k w_k Y_k(x, y, z) with respect to (x, y, z), for weights w.
__device__ __forceinline__ void sh_basis_vjp(int deg, float x, float y, float z, const float* w,
                                             float& gx, float& gy, float& gz)
{
    const ShConst c = sh_const();
    gx = gy = gz = 0.0f;
    if (deg < 1) return;
    gx += -c.k1 * w[3];
    gy += -c.k1 * w[1];
    gz += c.k1 * w[2];
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    gx += c.k2a * y * w[4] - 2.0f * c.k2b * x * w[6] - c.k2a * z * w[7] + 2.0f * c.k2c * x * w[8];
    gy += c.k2a * x * w[4] - c.k2a * z * w[5] - 2.0f * c.k2b * y * w[6] - 2.0f * c.k2c * y * w[8];
    gz += -c.k2a * y * w[5] + 4.0f * c.k2b * z * w[6] - c.k2a * x * w[7];
    if (deg < 3) return;
    gx += -6.0f * c.k3a * x * y * w[9] + c.k3b * y * z * w[10] + 2.0f * c.k3c * x * y * w[11]
          - 6.0f * c.k3d * x * z * w[12] - c.k3c * (4.0f * zz - 3.0f * xx - yy) * w[13]
          + 2.0f * c.k3e * x * z * w[14] - 3.0f * c.k3a * (xx - yy) * w[15];
    gy += -3.0f * c.k3a * (xx - yy) * w[9] + c.k3b * x * z * w[10]
          - c.k3c * (4.0f * zz - xx - 3.0f * yy) * w[11] - 6.0f * c.k3d * y * z * w[12]
          + 2.0f * c.k3c * x * y * w[13] - 2.0f * c.k3e * y * z * w[14] + 6.0f * c.k3a * x * y * w[15];
    gz += c.k3b * x * y * w[10] - 8.0f * c.k3c * y * z * w[11]
          + c.k3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12] - 8.0f * c.k3c * x * z * w[13]
          + c.k3e * (xx - yy) * w[14];
}

// One Adam update (Kingma & Ba, bias-corrected; inv_bc = 1 / (1 - beta^step)),
// rounding pinned with intrinsics so every kernel that applies it agrees bit
// for bit.
__device__ __forceinline__ void adam_step(float& p, float g, float& m, float& v, float b1, float b2, float eps,
                                          float inv_bc1, float inv_bc2, float lr)
{
    m = __fmaf_rn(b1, m, __fmul_rn(1.0f - b1, g));
    v = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(1.0f - b2, g), g));
    const float mhat = __fmul_rn(m, inv_bc1);
    const float vhat = __fmul_rn(v, inv_bc2);
    // sqrt(vhat) and the division through the SFU's approximate reciprocal
    // square root and reciprocal: a few ulp on the step, no branches
    const float root = vhat > 0.0f ? __fmul_rn(vhat, rsqrtf(vhat)) : 0.0f;
    p = __fsub_rn(p, __fdividef(__fmul_rn(lr, mhat), __fadd_rn(root, eps)));
}

__device__ __forceinline__ void store_as(void* dst, int dtype, int64_t e, float val)
{
    if (dtype == GS_DTYPE_BF16) reinterpret_cast<__nv_bfloat16*>(dst)[e] = __float2bfloat16_rn(val);
    else if (dtype == GS_DTYPE_F16) reinterpret_cast<__half*>(dst)[e] = __float2half_rn(val);
    else reinterpret_cast<float*>(dst)[e] = val;
}

// The value store_as keeps for val, as FP32 (round to nearest for BF16/FP16).
__device__ __forceinline__ float stored_value(int dtype, float val)
{
    if (dtype == GS_DTYPE_BF16) return __bfloat162float(__float2bfloat16_rn(val));
    if (dtype == GS_DTYPE_F16) return __half2float(__float2half_rn(val));
    return val;
}

// Four consecutive values stored as one vector in the given dtype: 8 bytes for
// BF16/FP16 at element e (e a multiple of 4 and the array 8-byte aligned), 16
// bytes for FP32.
__device__ __forceinline__ void store4_as(void* dst, int dtype, int64_t e, float4 v)
{
    if (dtype == GS_DTYPE_BF16) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        reinterpret_cast<uint2*>(dst)[e >> 2] =
            make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
    } else if (dtype == GS_DTYPE_F16) {
        const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        reinterpret_cast<uint2*>(dst)[e >> 2] =
            make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
    } else {
        reinterpret_cast<float4*>(dst)[e >> 2] = v;
    }
}

// ---------------------------------------------------------------------------
// Stochastic rounding of FP32 values to BF16/FP16 storage (for parameters kept
// only in the low-precision type: an update smaller than half a step of that
// type still moves the stored value, by a whole step with the matching
// probability, so the expected stored value follows the FP32 update).
// ---------------------------------------------------------------------------

// Counter-based generator: the PCG hash of Jarzynski and Olano ("Hash
// Functions for GPU Rendering", JCGT 9(3), 2020): one step of the 32-bit LCG
// of PCG, then PCG's RXS-M-XS output permutation.
__host__ __device__ __forceinline__ uint32_t pcg_hash(uint32_t v)
{
    const uint32_t state = v * 747796405u + 2891336453u;
    const uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}

// Stream of one optimizer step. Elements 2k and 2k + 1 draw the low and the
// high 16 bits of pcg_hash(base + k).
__host__ __device__ __forceinline__ uint32_t sr_base(uint32_t seed, uint32_t step)
{
    return pcg_hash(pcg_hash(seed) ^ step);
}

__device__ __forceinline__ uint32_t sr_bits16(uint32_t base, uint32_t e)
{
    const uint32_t h = pcg_hash(base + (e >> 1));
    return (e & 1u) ? (h >> 16) : (h & 0xffffu);
}

// x rounded to the BF16 neighbour away from zero when the 16 random bits r are
// below the FP32 bits it drops (its position between the two neighbours, in
// units of 2^-16 of a BF16 step), else toward zero. Non-finite: nearest.
__device__ __forceinline__ uint16_t sr_bf16(float x, uint32_t r)
{
    const uint32_t b = __float_as_uint(x);
    if ((b & 0x7f800000u) == 0x7f800000u) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return (uint16_t)((b >> 16) + ((b & 0xffffu) > r ? 1u : 0u));
}

// The same rule for FP16, in integer arithmetic on x's bits. In FP16's normal
// range the pattern toward zero keeps the top 10 of x's 23 mantissa bits and
// the 13 it drops are x's position in units of 2^-13 of the step (<< 3: units
// of 2^-16). Below it (FP16 subnormals and zero, steps of 2^-24) the position
// comes from |x| 2^24 = m + f (m the subnormal mantissa; the scaling by a power
// of two and the difference are exact). Magnitudes from 2^16 saturate at the
// largest finite value, as does rounding up from it; non-finite: nearest.
__device__ __forceinline__ uint16_t sr_f16(float x, uint32_t r)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t sign = (b >> 16) & 0x8000u;
    const uint32_t ex = (b >> 23) & 0xffu;
    if (ex - 113u <= 29u) {
        const uint32_t h = sign | ((ex - 112u) << 10) | ((b >> 13) & 0x3ffu);
        const uint32_t pos = (b & 0x1fffu) << 3;
        return (uint16_t)(h + ((pos > r && (h & 0x7fffu) != 0x7bffu) ? 1u : 0u));
    }
    if (ex < 113u) {
        const float y = __fmul_rn(fabsf(x), 16777216.0f);
        const uint32_t m = __float2uint_rz(y);
        const uint32_t pos = __float2uint_rz(__fmul_rn(__fsub_rn(y, (float)m), 65536.0f));
        return (uint16_t)((sign | m) + (pos > r ? 1u : 0u));
    }
    if (ex == 255u) return __half_as_ushort(__float2half_rn(x));
    return (uint16_t)(sign | 0x7bffu);
}

__device__ __forceinline__ uint16_t sr_round(float x, uint32_t r, int dtype)
{
    return dtype == GS_DTYPE_BF16 ? sr_bf16(x, r) : sr_f16(x, r);
}

// SH storage conversions
__device__ __forceinline__ float load_sh_elem(const void* base, int64_t idx, int dtype)
{
    if (dtype == GS_DTYPE_F32) return reinterpret_cast<const float*>(base)[idx];
    if (dtype == GS_DTYPE_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[idx]);
    return __half2float(reinterpret_cast<const __half*>(base)[idx]);
}

// Unit quaternion (w, x, y, z) -> row-major rotation matrix.
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float* R)
{
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
    R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
}

}  // namespace gs

// Host-side helpers shared by the API translation units.
namespace gs_host {
void set_error(const char* msg);
int32_t check_launch(const char* what);
bool make_cam(const GsCamera* in, gs::Cam* out);
bool make_dil(const GsCamera* cam, const GsDilation* in, gs::Dil* out);
// Fills the device view table from the caller's; checks cameras and dilations
// (one tile size for all views).
bool make_batch(const GsView* views, int nviews, gs::Batch* out);
// Streaming multiprocessors of the current device (read once per device; 148
// if the query fails), for the grids sized to whole waves.
int sm_count();
}  // namespace gs_host
