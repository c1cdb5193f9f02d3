// Multi-view cluster frame (the paper's multiview organizer, Sec. 3.2): the real
// view of one camera at full resolution, and below it the 2 x n_side views of its
// neighbourhood along the camera arc, each box-downscaled by `scale` and tiled
// `scale` per row.  One fused resize + copy pass over the output frame.
#include "common.h"

namespace fvv {
namespace {

constexpr int kMaxSide = 64; // views per side that fit the kernel's pointer table

struct SideTable {
    const float *v[2 * kMaxSide];
};

// One thread per output pixel.  Rows [0, H): the centre view; rows [H, H + R·H/s):
// tile k = (row block) x s + (column block), view k of the arc, pixel = the s x s
// box average (summed row by row, left to right, then scaled by 1 / s^2).
__global__ void stitch_kernel(const float *center, const SideTable tab, int n_views, int H, int W, int s, int out_h,
                              float *out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)out_h * W) return;
    const int x = (int)(idx % W), y = (int)(idx / W);
    float *o = out + idx * 3;
    if (y < H) {
        const float *c = center + ((size_t)y * W + x) * 3;
        o[0] = __ldg(c); o[1] = __ldg(c + 1); o[2] = __ldg(c + 2);
        return;
    }
    const int th = H / s, tw = W / s;
    const int ty = (y - H) / th, tx = x / tw, k = ty * s + tx;
    if (k >= n_views) { o[0] = o[1] = o[2] = 0.f; return; }
    const int sy = ((y - H) - ty * th) * s, sx = (x - tx * tw) * s;
    const float *src = tab.v[k];
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int dy = 0; dy < s; ++dy) {
        const float *row = src + ((size_t)(sy + dy) * W + sx) * 3;
        for (int dx = 0; dx < s; ++dx) {
            a0 += __ldg(row + 3 * dx);
            a1 += __ldg(row + 3 * dx + 1);
            a2 += __ldg(row + 3 * dx + 2);
        }
    }
    const float inv = 1.f / (float)(s * s);
    o[0] = a0 * inv; o[1] = a1 * inv; o[2] = a2 * inv;
}

} // namespace
} // namespace fvv

using namespace fvv;

extern "C" int fvv_stitch_cluster(const float *center, const float *const *side_views, int n_side, int H, int W,
                                  int scale, float *out, void *stream) {
    clear_error();
    if (!center || !side_views || !out) { set_error("NULL argument"); return FVV_EINVAL; }
    if (n_side < 1 || n_side > kMaxSide || scale < 1 || H < 1 || W < 1 || H % scale || W % scale) {
        set_error("stitch: need 1 <= n_side <= %d, scale >= 1 dividing H and W", kMaxSide);
        return FVV_ESHAPE;
    }
    SideTable tab{};
    for (int i = 0; i < 2 * n_side; ++i) {
        if (!side_views[i]) { set_error("stitch: side view %d is NULL", i); return FVV_EINVAL; }
        tab.v[i] = side_views[i];
    }
    const int rows = (2 * n_side + scale - 1) / scale;
    const int out_h = H + rows * (H / scale);
    const long long n = (long long)out_h * W;
    stitch_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(center, tab, 2 * n_side, H, W, scale,
                                                                                out_h, out);
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}
