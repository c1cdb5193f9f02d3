// Memory-bound stages of the VINet forward: frame pyramid, VIBlock input
// assembly (upsample + backward warp), Eq. 2 residual update, final warp +
// blend (Eq. 1), context warps for the refinement U-Net, and the residual output.
//
// Sampling conventions (the paper leaves them open; one reading, used throughout):
//  * backward warp: out(x, y) = I(x + F_x, y + F_y), bilinear, pixel centres at
//    integer indices; the sample point is split as x + floor(F_x) and weight
//    F_x - floor(F_x); taps clamp to the border (zero mode) or wrap (circular);
//  * x2 upsampling: fine pixel X samples coarse coordinate X/2 - 1/4 (half-pixel
//    centres), taps clamp or wrap; flow values are doubled;
//  * stage images and the flow pyramid are box averages.
// All coordinates, weights, flows and mask logits are FP32.
#include <cstring>

#include "common.h"
#include "kernels.h"
#include "sampling.h"

namespace fvv {

namespace {

template <typename T> __device__ __forceinline__ T to_store(float v);
template <> __device__ __forceinline__ float to_store<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 to_store<bf16>(float v) { return __float2bfloat16_rn(v); }

// Store the N values of one pixel.  FP32 layouts are dense (cs = N).  The bf16
// layouts keep cs a multiple of 8 so that every pixel is 16-byte aligned and is
// written with 16-byte stores; only the first round_up(N, 8) channels are written:
// the channels above stay at the zeros the buffer was cleared to when allocated.
template <int N> __device__ __forceinline__ void store_px(float *dst, const float (&v)[N], int cs) {
    for (int c = 0; c < cs; ++c) dst[c] = c < N ? v[c] : 0.f;
}
template <int N> __device__ __forceinline__ void store_px(bf16 *dst, const float (&v)[N], int) {
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 8) {
        __nv_bfloat162 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int c = c0 + 2 * j;
            h[j] = __floats2bfloat162_rn(c < N ? v[c] : 0.f, c + 1 < N ? v[c + 1] : 0.f);
        }
        uint4 u;
        memcpy(&u, h, 16);
        *reinterpret_cast<uint4 *>(dst + c0) = u;
    }
}

// ---------------------------------------------------------------------------
// a0: zero-pad each camera frame to Hp x Wp and build its 1/2 box level.
// One thread per 2x2 block (= one pixel of the 1/2 level).
__global__ void prep_cams_kernel(const float *const *cams, int n_cams, const int *ncam_dev, int H, int W, int Hp,
                                 int Wp, float4 *img0, float4 *img1) {
    n_cams = dev_count(ncam_dev, n_cams);
    int h2 = Hp / 2, w2 = Wp / 2;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n_cams * h2 * w2) return;
    int x2 = idx % w2;
    long long r = idx / w2;
    int y2 = r % h2, c = r / h2;
    const float *src = cams[c];
    float s[3] = {0.f, 0.f, 0.f};
    size_t P0 = (size_t)Hp * Wp;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        int y = 2 * y2 + dy;
        float v[6];
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            int x = 2 * x2 + dx;
            bool in = y < H && x < W;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) v[3 * dx + ch] = in ? __ldg(src + ((size_t)y * W + x) * 3 + ch) : 0.f;
        }
        float4 *d = img0 + (size_t)c * P0 + (size_t)y * Wp + 2 * x2;
        d[0] = make_float4(v[0], v[1], v[2], 0.f);
        d[1] = make_float4(v[3], v[4], v[5], 0.f);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) s[ch] += v[ch] + v[3 + ch];
    }
    img1[(size_t)c * (P0 / 4) + (size_t)y2 * w2 + x2] = make_float4(s[0] * 0.25f, s[1] * 0.25f, s[2] * 0.25f, 0.f);
}

// a0: the 1/4 level as the 2x2 box average of the 1/2 level (= the 4x4 box).
__global__ void box_quarter_kernel(const float4 *img1, int n_cams, const int *ncam_dev, int h2, int w2,
                                   float4 *img2) {
    n_cams = dev_count(ncam_dev, n_cams);
    int h4 = h2 / 2, w4 = w2 / 2;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n_cams * h4 * w4) return;
    int x = idx % w4;
    long long r = idx / w4;
    int y = r % h4, c = r / h4;
    const float4 *s = img1 + (size_t)c * h2 * w2;
    size_t p00 = (size_t)(2 * y) * w2 + 2 * x, p10 = p00 + w2;
    float4 a = s[p00], b = s[p00 + 1], d = s[p10], e = s[p10 + 1];
    img2[idx] = make_float4((a.x + b.x + d.x + e.x) * 0.25f, (a.y + b.y + d.y + e.y) * 0.25f,
                            (a.z + b.z + d.z + e.z) * 0.25f, 0.f);
}

// a2 input: [I_l/4, I_r/4, t] (7 channels, zero-padded to cs).
template <typename T>
__global__ void vib0_input_kernel(const float4 *img2, const ViewTab vt, int nv, int h, int w, T *x, int cs) {
    nv = dev_count(vt.n, nv);
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long P = (long long)h * w;
    if (idx >= (long long)nv * P) return;
    int v = idx / P;
    long long p = idx % P;
    const float4 L = __ldg(img2 + (size_t)vt.cam_l[v] * P + p);
    const float4 R = __ldg(img2 + (size_t)vt.cam_r[v] * P + p);
    float vals[7] = {L.x, L.y, L.z, R.x, R.y, R.z, vt.t[v]};
    store_px(x + (size_t)idx * cs, vals, cs);
}

// Pixel of this thread in a grid of 32 x 8 tiles (blocks of 256 threads): the taps of a
// tile's bilinear gathers overlap in rows as well as columns, so they share L1 lines.
__device__ __forceinline__ bool tile_pixel(int h, int w, int &X, int &Y) {
    const int tiles_x = (w + 31) / 32;
    X = (int)(blockIdx.x % tiles_x) * 32 + (int)(threadIdx.x & 31);
    Y = (int)(blockIdx.x / tiles_x) * 8 + (int)(threadIdx.x >> 5);
    return X < w && Y < h;
}

// a3: stage s input [I_l, I_r, W_l, W_r, M_up, F_up(4), t] (18 ch, zero-padded to cs)
// at the stage grid h x w, from the previous stage's flow/mask FMp (h/2 x w/2 x 5).
// One thread per pixel walks the views: views of one camera pair gather the same
// image neighbourhoods, which then come from L1/L2 instead of DRAM once per view.
template <typename T, bool CIRC>
__global__ void stage_input_kernel(const float4 *imgs, const float *FMp, const ViewTab vt, int nv,
                                   int h, int w, T *x, int cs) {
    nv = dev_count(vt.n, nv);
    const long long P = (long long)h * w;
    int X, Y;
    if (!tile_pixel(h, w, X, Y)) return;
    const int p = Y * w + X;
    for (int v = 0; v < nv; ++v) {
    const long long idx = v * P + p;
    const float *fm = FMp + (size_t)v * (P / 4) * 5;
    Taps u = up_taps_t<CIRC>(X, Y, h / 2, w / 2);
    float up[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) up[c] = bilerp(fm, 5, c, u);
#pragma unroll
    for (int c = 0; c < 4; ++c) up[c] *= 2.f;
    const float4 *L = imgs + (size_t)vt.cam_l[v] * P;
    const float4 *R = imgs + (size_t)vt.cam_r[v] * P;
    Taps tl = warp_taps_t<CIRC>(X, Y, up[0], up[1], h, w);
    Taps tr = warp_taps_t<CIRC>(X, Y, up[2], up[3], h, w);
    const float4 lc = __ldg(L + p), rc = __ldg(R + p);
    const float3 wl = bilerp_rgb(L, tl), wr = bilerp_rgb(R, tr);
    float vals[18] = {lc.x, lc.y, lc.z, rc.x, rc.y, rc.z, wl.x, wl.y, wl.z, wr.x, wr.y, wr.z};
    vals[12] = up[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) vals[13 + c] = up[c];
    vals[17] = vt.t[v];
    store_px(x + (size_t)idx * cs, vals, cs);
    }
}

// Eq. 2: F^s, M^s = up(F^{s-1}) x2, up(M^{s-1}) + Res^s  (in place on res).
__global__ void residual_kernel(const float *FMp, float *res, int nv, const int *nv_dev, int h, int w, int circ) {
    nv = dev_count(nv_dev, nv);
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long P = (long long)h * w;
    if (idx >= (long long)nv * P) return;
    int v = idx / P;
    int p = idx % P;
    int X = p % w, Y = p / w;
    const float *fm = FMp + (size_t)v * (P / 4) * 5;
    Taps u = up_taps(X, Y, h / 2, w / 2, circ);
    float *r = res + (size_t)idx * 5;
#pragma unroll
    for (int c = 0; c < 5; ++c) r[c] += bilerp(fm, 5, c, u) * (c < 4 ? 2.f : 1.f);
}

// a5 (Eq. 1): I_l->m, I_r->m by the final flows, M = sigmoid(logit), blend.
// Writes the refinement input [I_l->m, I_r->m] (zero-padded to cs) and I_blend.
// One thread per pixel walks the views (image taps shared across views stay in cache).
template <typename T, bool CIRC>
__global__ void final_blend_kernel(const float4 *__restrict__ img0, const float *__restrict__ FM, const ViewTab vt,
                                   int nv, int h, int w, T *__restrict__ u0, int cs, float *__restrict__ ib) {
    nv = dev_count(vt.n, nv);
    const long long P = (long long)h * w;
    int X, Y;
    if (!tile_pixel(h, w, X, Y)) return;
    const int p = Y * w + X;
    // two views in flight per thread (their gathers overlap)
#pragma unroll 2
    for (int v = 0; v < nv; ++v) {
    const long long idx = v * P + p;
    const float *f = FM + (size_t)idx * 5;
    const float4 *L = img0 + (size_t)vt.cam_l[v] * P;
    const float4 *R = img0 + (size_t)vt.cam_r[v] * P;
    Taps tl = warp_taps_t<CIRC>(X, Y, f[0], f[1], h, w);
    Taps tr = warp_taps_t<CIRC>(X, Y, f[2], f[3], h, w);
    float M = sigmoidf_(f[4]);
    const float3 a = bilerp_rgb(L, tl), b = bilerp_rgb(R, tr);
    float vals[6] = {a.x, a.y, a.z, b.x, b.y, b.z};
    float *o = ib + (size_t)idx * 3;
    o[0] = M * a.x + (1.f - M) * b.x;
    o[1] = M * a.y + (1.f - M) * b.y;
    o[2] = M * a.z + (1.f - M) * b.z;
    store_px(u0 + (size_t)idx * cs, vals, cs);
    }
}

// Bilinear sample of 8 consecutive channels (bf16 storage, 16-byte loads).
__device__ __forceinline__ void bilerp8(const bf16 *img, int cs, int c0, const Taps &t, float (&o)[8]) {
    const int offs[4] = {t.o00, t.o01, t.o10, t.o11};
    float a[4][8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint4 u = __ldg(reinterpret_cast<const uint4 *>(img + (size_t)offs[k] * cs + c0));
        __nv_bfloat162 hh[4];
        memcpy(hh, &u, 16);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float2 f = __bfloat1622float2(hh[j]);
            a[k][2 * j] = f.x;
            a[k][2 * j + 1] = f.y;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
        o[j] = (1.f - t.ly) * ((1.f - t.lx) * a[0][j] + t.lx * a[1][j]) + t.ly * ((1.f - t.lx) * a[2][j] + t.lx * a[3][j]);
}
__device__ __forceinline__ void bilerp8(const float *img, int cs, int c0, const Taps &t, float (&o)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = bilerp(img, cs, c0 + j, t);
}
__device__ __forceinline__ void store8(float *d, const float (&v)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) d[j] = v[j];
}
__device__ __forceinline__ void store8(bf16 *d, const float (&v)[8]) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    uint4 u;
    memcpy(&u, h, 16);
    *reinterpret_cast<uint4 *>(d) = u;
}

// a6: flow pyramid level k: F_k = box2(F_{k-1}) / 2 (4 channels; F_0 = the final
// flow with stride 5), then warp both cameras' context features of this level
// by F_k[0:2] / F_k[2:4] into channel slots of the U-Net level tensor.
// One thread per (pixel, group of 8 channels) walks the views (the context features
// of a camera are gathered by every view that uses it).
// (glog = log2(C / 8): groups of 8 channels per pixel; every index fits in 32 bits)
template <typename T, bool CIRC>
__global__ void ctx_warp_kernel(const float *Fprev, int fprev_cs, float *Fk, const T *ctx, int C, int glog,
                                const ViewTab vt, int nv, int h, int w,
                                T *dst, int dst_cs, int off_l, int off_r) {
    nv = dev_count(vt.n, nv);
    const int P = h * w;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= (P << glog)) return;
    const int g = gi & ((1 << glog) - 1);
    const int p = gi >> glog;
    const int X = p % w, Y = p / w;
    const int W2 = 2 * w;
    // the 2 x 2 block of the finer flow level under this pixel
    const int i00 = (2 * Y * W2 + 2 * X) * fprev_cs, i01 = i00 + fprev_cs, i10 = i00 + W2 * fprev_cs,
              i11 = i10 + fprev_cs;
    for (int v = 0; v < nv; ++v) {
    const size_t vp = (size_t)v * P + p;
    const float *fp = Fprev + (size_t)v * (P * 4) * fprev_cs;
    float F[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float s = fp[i00 + c] + fp[i01 + c] + fp[i10 + c] + fp[i11 + c];
        F[c] = s * 0.25f * 0.5f;
    }
    if (g == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) Fk[(size_t)vp * 4 + c] = F[c];
    }
    const T *cl = ctx + (size_t)vt.cam_l[v] * P * C;
    const T *cr = ctx + (size_t)vt.cam_r[v] * P * C;
    Taps tl = warp_taps_t<CIRC>(X, Y, F[0], F[1], h, w);
    Taps tr = warp_taps_t<CIRC>(X, Y, F[2], F[3], h, w);
    T *d = dst + (size_t)vp * dst_cs;
    float o[8];
    bilerp8(cl, C, g * 8, tl, o);
    store8(d + off_l + g * 8, o);
    bilerp8(cr, C, g * 8, tr, o);
    store8(d + off_r + g * 8, o);
    }
}

// a8: out = clamp(I_blend + 2 sigmoid(z) - 1, 0, 1), cropped to H x W.
__global__ void output_kernel(const float *ib, const float *z, int z_cs, int nv, const int *nv_dev, int Hp, int Wp,
                              int H, int W, float *const *outp) {
    nv = dev_count(nv_dev, nv);
    float *out = *outp;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long P = (long long)H * W;
    if (idx >= (long long)nv * P) return;
    int v = idx / P;
    int p = idx % P;
    int x = p % W, y = p / W;
    size_t q = (size_t)v * Hp * Wp + (size_t)y * Wp + x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float r = 2.f * sigmoidf_(z[q * z_cs + c]) - 1.f;
        out[(size_t)idx * 3 + c] = fminf(fmaxf(ib[q * 3 + c] + r, 0.f), 1.f);
    }
}

// Circular padding for the tensor-core convolutions (whose TMA loads can only fill out-
// of-range rows and columns with zeros): the channel window [coff, coff + chunks x 16 B)
// of every pixel of n images, copied into an (H + 2 pad) x (W + 2 pad) image whose
// border repeats the opposite edges (pixel (y, x) = input ((y - pad) mod H, (x - pad)
// mod W)).  One thread per 16-byte chunk of the padded image.
__global__ void wrap_pad_kernel(const uint8_t *__restrict__ in, int N, const int *n_dev, int H, int W, int cs_b,
                                int coff_b, int chunks, int pad, uint8_t *__restrict__ out) {
    N = dev_count(n_dev, N);
    const int Hq = H + 2 * pad, Wq = W + 2 * pad;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * Hq * Wq * chunks) return;
    const int j = (int)(idx % chunks);
    long long r = idx / chunks;
    const int x = (int)(r % Wq);
    r /= Wq;
    const int y = (int)(r % Hq), n = (int)(r / Hq);
    int sy = (y - pad) % H, sx = (x - pad) % W;
    sy += sy < 0 ? H : 0;
    sx += sx < 0 ? W : 0;
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(in + (((size_t)n * H + sy) * W + sx) * cs_b + coff_b) + j);
    reinterpret_cast<uint4 *>(out)[idx] = v;
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }
// 256-thread blocks over 32 x 8 pixel tiles (a warp = 32 pixels of one row)
inline unsigned tile_blocks(int h, int w) { return (unsigned)(((w + 31) / 32) * ((h + 7) / 8)); }

} // namespace

#define FVV_LAUNCH_CHECK() \
    do { count_launch(); FVV_CHECK_CUDA(cudaGetLastError()); } while (0)

int launch_prep_cams(const float *const *cams, int n_cams, const int *ncam_dev, int H, int W, int Hp, int Wp,
                     float4 *img0, float4 *img1, float4 *img2, cudaStream_t st) {
    long long n = (long long)n_cams * (Hp / 2) * (Wp / 2);
    prep_cams_kernel<<<blocks_for(n, 256), 256, 0, st>>>(cams, n_cams, ncam_dev, H, W, Hp, Wp, img0, img1);
    FVV_LAUNCH_CHECK();
    n = (long long)n_cams * (Hp / 4) * (Wp / 4);
    box_quarter_kernel<<<blocks_for(n, 256), 256, 0, st>>>(img1, n_cams, ncam_dev, Hp / 2, Wp / 2, img2);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

template <typename T>
int launch_vib0_input(const float4 *img2, const ViewTab &vt, int nv, int h, int w, T *x, int cs, cudaStream_t st) {
    long long n = (long long)nv * h * w;
    vib0_input_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(img2, vt, nv, h, w, x, cs);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

template <typename T>
int launch_stage_input(const float4 *imgs, const float *FMp, const ViewTab &vt, int nv, int h, int w,
                       int circ, T *x, int cs, cudaStream_t st) {
    if (circ) stage_input_kernel<T, true><<<tile_blocks(h, w), 256, 0, st>>>(imgs, FMp, vt, nv, h, w, x, cs);
    else stage_input_kernel<T, false><<<tile_blocks(h, w), 256, 0, st>>>(imgs, FMp, vt, nv, h, w, x, cs);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

int launch_residual(const float *FMp, float *res, int nv, const int *nv_dev, int h, int w, int circ,
                    cudaStream_t st) {
    long long n = (long long)nv * h * w;
    residual_kernel<<<blocks_for(n, 256), 256, 0, st>>>(FMp, res, nv, nv_dev, h, w, circ);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

template <typename T>
int launch_final_blend(const float4 *img0, const float *FM, const ViewTab &vt, int nv, int h, int w,
                       int circ, T *u0, int cs, float *ib, cudaStream_t st) {
    if (circ) final_blend_kernel<T, true><<<tile_blocks(h, w), 256, 0, st>>>(img0, FM, vt, nv, h, w, u0, cs, ib);
    else final_blend_kernel<T, false><<<tile_blocks(h, w), 256, 0, st>>>(img0, FM, vt, nv, h, w, u0, cs, ib);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

template <typename T>
int launch_ctx_warp(const float *Fprev, int fprev_cs, float *Fk, const T *ctx, int C, const ViewTab &vt,
                    int nv, int h, int w, int circ, T *dst, int dst_cs, int off_l, int off_r, cudaStream_t st) {
    long long n = (long long)h * w * (C / 8);
    int glog = 0;
    while ((8 << glog) < C) ++glog;
    if ((8 << glog) != C || 4ll * h * w * fprev_cs >= (1ll << 31) || n >= (1ll << 31)) {
        set_error("context warp: C must be 8 x a power of two, the level below 2^31 elements");
        return FVV_ESHAPE;
    }
    if (circ)
        ctx_warp_kernel<T, true><<<blocks_for(n, 256), 256, 0, st>>>(Fprev, fprev_cs, Fk, ctx, C, glog, vt, nv, h, w,
                                                                     dst, dst_cs, off_l, off_r);
    else
        ctx_warp_kernel<T, false><<<blocks_for(n, 256), 256, 0, st>>>(Fprev, fprev_cs, Fk, ctx, C, glog, vt, nv, h, w,
                                                                      dst, dst_cs, off_l, off_r);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

int launch_wrap_pad(const void *in, int N, const int *n_dev, int H, int W, int cs_bytes, int coff_bytes, int bytes,
                    int pad, void *out, cudaStream_t st) {
    if (cs_bytes % 16 || coff_bytes % 16 || bytes % 16 || ((uintptr_t)in % 16) || ((uintptr_t)out % 16)) {
        set_error("circular pad: pixel stride, offset and width must be multiples of 16 bytes");
        return FVV_EINVAL;
    }
    const long long n = (long long)N * (H + 2 * pad) * (W + 2 * pad) * (bytes / 16);
    wrap_pad_kernel<<<blocks_for(n, 256), 256, 0, st>>>((const uint8_t *)in, N, n_dev, H, W, cs_bytes, coff_bytes,
                                                        bytes / 16, pad, (uint8_t *)out);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

int launch_output(const float *ib, const float *z, int z_cs, int nv, const int *nv_dev, int Hp, int Wp, int H, int W,
                  float *const *outp, cudaStream_t st) {
    long long n = (long long)nv * H * W;
    output_kernel<<<blocks_for(n, 256), 256, 0, st>>>(ib, z, z_cs, nv, nv_dev, Hp, Wp, H, W, outp);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

#define INST(T)                                                                                          \
    template int launch_vib0_input<T>(const float4 *, const ViewTab &, int, int, int, T *, int, cudaStream_t); \
    template int launch_stage_input<T>(const float4 *, const float *, const ViewTab &, int, int, int, int, T *, \
                                       int, cudaStream_t);                                              \
    template int launch_final_blend<T>(const float4 *, const float *, const ViewTab &, int, int, int, int, T *, \
                                       int, float *, cudaStream_t);                                     \
    template int launch_ctx_warp<T>(const float *, int, float *, const T *, int, const ViewTab &, int, int, int, \
                                    int, T *, int, int, int, cudaStream_t);
INST(float)
INST(bf16)
#undef INST

} // namespace fvv
