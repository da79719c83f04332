// gs_api.cu -- error state, argument checks and small host helpers of the C ABI.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "gs_common.cuh"

namespace {
thread_local char g_err[512] = "";
}

namespace gs_host {

void set_error(const char* msg)
{
    std::snprintf(g_err, sizeof(g_err), "%s", msg);
}

int sm_count()
{
    constexpr int kMaxDevices = 64;
    static int cached[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return 148;
    }
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 148;
        }
        cached[dev] = n;
    }
    return cached[dev];
}

int32_t check_launch(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        std::snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

bool make_cam(const GsCamera* in, gs::Cam* out)
{
    if (!in) { set_error("camera is null"); return false; }
    if (in->width <= 0 || in->height <= 0 || !(in->fx > 0.0f) || !(in->fy > 0.0f)) {
        set_error("camera: width, height, fx and fy must be positive");
        return false;
    }
    for (int i = 0; i < 9; ++i) out->R[i] = in->R[i];
    for (int i = 0; i < 3; ++i) out->T[i] = in->T[i];
    out->fx = in->fx; out->fy = in->fy; out->cx = in->cx; out->cy = in->cy;
    out->width = in->width; out->height = in->height; out->z_near = in->z_near;
    out->lim_x = (float)(gs::kClampFov * 0.5 * (double)in->width / (double)in->fx);
    out->lim_y = (float)(gs::kClampFov * 0.5 * (double)in->height / (double)in->fy);
    // camera centre -R^T T, evaluated in double
    double c[3];
    for (int j = 0; j < 3; ++j)
        c[j] = -((double)in->R[j] * in->T[0] + (double)in->R[3 + j] * in->T[1] + (double)in->R[6 + j] * in->T[2]);
    out->ccx = (float)c[0]; out->ccy = (float)c[1]; out->ccz = (float)c[2];
    return true;
}

bool make_dil(const GsCamera* cam, const GsDilation* in, gs::Dil* out)
{
    if (!in || !cam) { set_error("dilation or camera is null"); return false; }
    if (in->d < 1 || in->d > 64 || in->ox < 0 || in->ox >= in->d || in->oy < 0 || in->oy >= in->d) {
        set_error("dilation: need 1 <= d <= 64 and 0 <= ox, oy < d");
        return false;
    }
    if (in->tile != 8 && in->tile != 16 && in->tile != 32) {
        set_error("dilation: tile must be 8, 16 or 32");
        return false;
    }
    if (in->center_mode != 0 && in->center_mode != 1) {
        set_error("dilation: center_mode must be 0 or 1");
        return false;
    }
    if (cam->width <= in->ox || cam->height <= in->oy) {
        set_error("dilation: offset outside the image");
        return false;
    }
    if (in->bin_shift < 0 || in->bin_shift > 2) {
        set_error("dilation: bin_shift must be 0, 1 or 2");
        return false;
    }
    out->d = in->d; out->ox = in->ox; out->oy = in->oy; out->mode = in->center_mode; out->tile = in->tile;
    out->w_ds = (cam->width - in->ox + in->d - 1) / in->d;
    out->h_ds = (cam->height - in->oy + in->d - 1) / in->d;
    out->tiles_x = (out->w_ds + in->tile - 1) / in->tile;
    out->tiles_y = (out->h_ds + in->tile - 1) / in->tile;
    out->shift = in->bin_shift;
    const int step = 1 << in->bin_shift;
    out->bin_tiles_x = (out->tiles_x + step - 1) / step;
    out->bin_tiles_y = (out->tiles_y + step - 1) / step;
    return true;
}

bool make_batch(const GsView* views, int nviews, gs::Batch* out)
{
    if (!views || nviews < 1 || nviews > GS_MAX_VIEWS) {
        set_error("batch: need 1 <= nviews <= GS_MAX_VIEWS and a view table");
        return false;
    }
    out->nviews = nviews;
    int tiles = 0;
    for (int i = 0; i < nviews; ++i) {
        const GsView& in = views[i];
        gs::ViewDev& v = out->v[i];
        if (!make_cam(&in.cam, &v.cam) || !make_dil(&in.cam, &in.dil, &v.dil)) return false;
        if (v.dil.tile != out->v[0].dil.tile) {
            set_error("batch: all views must use the same tile size");
            return false;
        }
        v.splats = reinterpret_cast<float4*>(in.splats);
        v.radii = in.radii;
        v.rects = reinterpret_cast<int4*>(in.rects);
        v.tiles = in.tiles_touched;
        v.ids = in.sorted_ids;
        v.ranges = reinterpret_cast<const uint2*>(in.ranges);
        v.img = in.img;
        v.t_final = in.t_final;
        v.last = in.last;
        v.target = in.target;
        v.target_dtype = in.target_dtype;
        if (in.target_dtype != GS_TARGET_F32 && in.target_dtype != GS_TARGET_U8) {
            set_error("view: target_dtype must be GS_TARGET_F32 or GS_TARGET_U8");
            return false;
        }
        v.dl = in.dl_dimg;
        v.grad2d = reinterpret_cast<float4*>(in.grad2d);
        v.loss = in.loss;
        v.keys = in.depth_keys;
        v.tile_begin = tiles;
        tiles += v.dil.tiles_x * v.dil.tiles_y;
    }
    out->total_tiles = tiles;
    return true;
}

}  // namespace gs_host

extern "C" {

int32_t gs_version(void) { return 100; }

const char* gs_last_error(void) { return g_err; }

int32_t gs_grid(const GsCamera* cam, const GsDilation* dil, int32_t* w_ds, int32_t* h_ds,
                int32_t* tiles_x, int32_t* tiles_y)
{
    gs::Dil d;
    if (!gs_host::make_dil(cam, dil, &d)) return GS_ERR_ARG;
    if (w_ds) *w_ds = d.w_ds;
    if (h_ds) *h_ds = d.h_ds;
    if (tiles_x) *tiles_x = d.tiles_x;
    if (tiles_y) *tiles_y = d.tiles_y;
    return GS_OK;
}

int32_t gs_bin_grid(const GsCamera* cam, const GsDilation* dil, int32_t* bin_tiles_x, int32_t* bin_tiles_y)
{
    gs::Dil d;
    if (!gs_host::make_dil(cam, dil, &d)) return GS_ERR_ARG;
    if (bin_tiles_x) *bin_tiles_x = d.bin_tiles_x;
    if (bin_tiles_y) *bin_tiles_y = d.bin_tiles_y;
    return GS_OK;
}

}  // extern "C"
