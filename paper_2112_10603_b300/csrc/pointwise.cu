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
#include "common.h"
#include "kernels.h"

namespace fvv {

namespace {

template <typename T> __device__ __forceinline__ T to_store(float v);
template <> __device__ __forceinline__ float to_store<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 to_store<bf16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(bf16 v) { return __bfloat162float(v); }

__device__ __forceinline__ int fix_index(int i, int n, int circ) {
    if (circ) { i %= n; return i < 0 ? i + n : i; }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Bilinear tap set for a backward warp at integer pixel (x, y) with flow (fx, fy).
struct Taps { int o00, o01, o10, o11; float lx, ly; };

__device__ __forceinline__ Taps warp_taps(int x, int y, float fx, float fy, int H, int W, int circ) {
    // beyond the border every tap clamps to the same pixel; this also maps NaN
    // (fmaxf returns the other operand) to a finite value, keeping indices in range
    float lim = circ ? 16777216.f : (float)(max(H, W) + 4);
    fx = fminf(fmaxf(fx, -lim), lim);
    fy = fminf(fmaxf(fy, -lim), lim);
    float flx = floorf(fx), fly = floorf(fy);
    Taps t;
    t.lx = fx - flx;
    t.ly = fy - fly;
    int x0 = x + (int)flx, y0 = y + (int)fly;
    int xa = fix_index(x0, W, circ), xb = fix_index(x0 + 1, W, circ);
    int ya = fix_index(y0, H, circ), yb = fix_index(y0 + 1, H, circ);
    t.o00 = ya * W + xa; t.o01 = ya * W + xb; t.o10 = yb * W + xa; t.o11 = yb * W + xb;
    return t;
}

template <typename T>
__device__ __forceinline__ float bilerp(const T *img, int cs, int c, const Taps &t) {
    float a = to_f(img[(size_t)t.o00 * cs + c]), b = to_f(img[(size_t)t.o01 * cs + c]);
    float d = to_f(img[(size_t)t.o10 * cs + c]), e = to_f(img[(size_t)t.o11 * cs + c]);
    return (1.f - t.ly) * ((1.f - t.lx) * a + t.lx * b) + t.ly * ((1.f - t.lx) * d + t.lx * e);
}

// x2 upsampling taps of fine pixel (Y, X) on a coarse h x w grid.
__device__ __forceinline__ Taps up_taps(int X, int Y, int h, int w, int circ) {
    Taps t;
    int x0 = (X >> 1) - ((X & 1) ? 0 : 1), y0 = (Y >> 1) - ((Y & 1) ? 0 : 1);
    t.lx = (X & 1) ? 0.25f : 0.75f;
    t.ly = (Y & 1) ? 0.25f : 0.75f;
    int xa = fix_index(x0, w, circ), xb = fix_index(x0 + 1, w, circ);
    int ya = fix_index(y0, h, circ), yb = fix_index(y0 + 1, h, circ);
    t.o00 = ya * w + xa; t.o01 = ya * w + xb; t.o10 = yb * w + xa; t.o11 = yb * w + xb;
    return t;
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

// ---------------------------------------------------------------------------
// a0: zero-pad each camera frame to Hp x Wp and build its 1/2 and 1/4 box pyramid.
// One thread per 4x4 block of the padded frame.
__global__ void prep_cams_kernel(const float *const *cams, int n_cams, int H, int W, int Hp, int Wp,
                                 float *img0, float *img1, float *img2, bf16 *img0_b16) {
    int h4 = Hp / 4, w4 = Wp / 4;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = (long long)n_cams * h4 * w4;
    if (idx >= total) return;
    int x4 = idx % w4;
    long long r = idx / w4;
    int y4 = r % h4, c = r / h4;
    const float *src = cams[c];
    float blk[4][4][3];
#pragma unroll
    for (int dy = 0; dy < 4; ++dy)
#pragma unroll
        for (int dx = 0; dx < 4; ++dx) {
            int y = y4 * 4 + dy, x = x4 * 4 + dx;
            bool in = y < H && x < W;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) blk[dy][dx][ch] = in ? __ldg(src + ((size_t)y * W + x) * 3 + ch) : 0.f;
        }
    size_t P0 = (size_t)Hp * Wp;
#pragma unroll
    for (int dy = 0; dy < 4; ++dy)
#pragma unroll
        for (int dx = 0; dx < 4; ++dx) {
            size_t p = (size_t)c * P0 + (size_t)(y4 * 4 + dy) * Wp + x4 * 4 + dx;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) img0[p * 3 + ch] = blk[dy][dx][ch];
            if (img0_b16) {
                bf16 *d = img0_b16 + p * 16;
#pragma unroll
                for (int ch = 0; ch < 16; ++ch) d[ch] = __float2bfloat16_rn(ch < 3 ? blk[dy][dx][ch] : 0.f);
            }
        }
    size_t P1 = P0 / 4;
    float s4[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int by = 0; by < 2; ++by)
#pragma unroll
        for (int bx = 0; bx < 2; ++bx) {
            size_t p = (size_t)c * P1 + (size_t)(y4 * 2 + by) * (Wp / 2) + x4 * 2 + bx;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float s = blk[2 * by][2 * bx][ch] + blk[2 * by][2 * bx + 1][ch] +
                          blk[2 * by + 1][2 * bx][ch] + blk[2 * by + 1][2 * bx + 1][ch];
                img1[p * 3 + ch] = s * 0.25f;
                s4[ch] += s;
            }
        }
    size_t p2 = (size_t)c * (P0 / 16) + (size_t)y4 * w4 + x4;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) img2[p2 * 3 + ch] = s4[ch] * 0.0625f;
}

// a2 input: [I_l/4, I_r/4, t] (7 channels, zero-padded to cs).
template <typename T>
__global__ void vib0_input_kernel(const float *img2, const ViewTab vt, int nv, int h, int w, T *x, int cs) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long P = (long long)h * w;
    if (idx >= (long long)nv * P) return;
    int v = idx / P;
    long long p = idx % P;
    const float *L = img2 + ((size_t)vt.cam_l[v] * P + p) * 3;
    const float *R = img2 + ((size_t)vt.cam_r[v] * P + p) * 3;
    T *d = x + (size_t)idx * cs;
    float vals[7] = {L[0], L[1], L[2], R[0], R[1], R[2], vt.t[v]};
    for (int c = 0; c < cs; ++c) d[c] = to_store<T>(c < 7 ? vals[c] : 0.f);
}

// a3: stage s input [I_l, I_r, W_l, W_r, M_up, F_up(4), t] (18 ch, zero-padded to cs)
// at the stage grid h x w, from the previous stage's flow/mask FMp (h/2 x w/2 x 5).
template <typename T>
__global__ void stage_input_kernel(const float *imgs, const float *FMp, const ViewTab vt, int nv,
                                   int h, int w, int circ, T *x, int cs) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long P = (long long)h * w;
    if (idx >= (long long)nv * P) return;
    int v = idx / P;
    int p = idx % P;
    int X = p % w, Y = p / w;
    const float *fm = FMp + (size_t)v * (P / 4) * 5;
    Taps u = up_taps(X, Y, h / 2, w / 2, circ);
    float up[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) up[c] = bilerp(fm, 5, c, u);
#pragma unroll
    for (int c = 0; c < 4; ++c) up[c] *= 2.f;
    const float *L = imgs + (size_t)vt.cam_l[v] * P * 3;
    const float *R = imgs + (size_t)vt.cam_r[v] * P * 3;
    Taps tl = warp_taps(X, Y, up[0], up[1], h, w, circ);
    Taps tr = warp_taps(X, Y, up[2], up[3], h, w, circ);
    float vals[18];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vals[c] = L[(size_t)p * 3 + c];
        vals[3 + c] = R[(size_t)p * 3 + c];
        vals[6 + c] = bilerp(L, 3, c, tl);
        vals[9 + c] = bilerp(R, 3, c, tr);
    }
    vals[12] = up[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) vals[13 + c] = up[c];
    vals[17] = vt.t[v];
    T *d = x + (size_t)idx * cs;
    for (int c = 0; c < cs; ++c) d[c] = to_store<T>(c < 18 ? vals[c] : 0.f);
}

// Eq. 2: F^s, M^s = up(F^{s-1}) x2, up(M^{s-1}) + Res^s  (in place on res).
__global__ void residual_kernel(const float *FMp, float *res, int nv, int h, int w, int circ) {
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
template <typename T>
__global__ void final_blend_kernel(const float *img0, const float *FM, const ViewTab vt, int nv,
                                   int h, int w, int circ, T *u0, int cs, float *ib) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long P = (long long)h * w;
    if (idx >= (long long)nv * P) return;
    int v = idx / P;
    int p = idx % P;
    int X = p % w, Y = p / w;
    const float *f = FM + (size_t)idx * 5;
    const float *L = img0 + (size_t)vt.cam_l[v] * P * 3;
    const float *R = img0 + (size_t)vt.cam_r[v] * P * 3;
    Taps tl = warp_taps(X, Y, f[0], f[1], h, w, circ);
    Taps tr = warp_taps(X, Y, f[2], f[3], h, w, circ);
    float M = sigmoidf_(f[4]);
    T *d = u0 + (size_t)idx * cs;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float a = bilerp(L, 3, c, tl), b = bilerp(R, 3, c, tr);
        d[c] = to_store<T>(a);
        d[3 + c] = to_store<T>(b);
        ib[(size_t)idx * 3 + c] = M * a + (1.f - M) * b;
    }
    for (int c = 6; c < cs; ++c) d[c] = to_store<T>(0.f);
}

// a6: flow pyramid level k: F_k = box2(F_{k-1}) / 2 (4 channels; F_0 = the final
// flow with stride 5), then warp both cameras' context features of this level
// by F_k[0:2] / F_k[2:4] into channel slots of the U-Net level tensor.
// One thread per (view, pixel, group of 8 channels).
template <typename T>
__global__ void ctx_warp_kernel(const float *Fprev, int fprev_cs, float *Fk, const T *ctx, int C,
                                const ViewTab vt, int nv, int h, int w, int circ,
                                T *dst, int dst_cs, int off_l, int off_r) {
    int groups = C / 8;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long P = (long long)h * w;
    if (idx >= (long long)nv * P * groups) return;
    int g = idx % groups;
    long long vp = idx / groups;
    int v = vp / P;
    int p = vp % P;
    int X = p % w, Y = p / w;
    const float *fp = Fprev + (size_t)v * (P * 4) * fprev_cs;
    int W2 = 2 * w;
    float F[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float s = fp[((size_t)(2 * Y) * W2 + 2 * X) * fprev_cs + c] + fp[((size_t)(2 * Y) * W2 + 2 * X + 1) * fprev_cs + c] +
                  fp[((size_t)(2 * Y + 1) * W2 + 2 * X) * fprev_cs + c] + fp[((size_t)(2 * Y + 1) * W2 + 2 * X + 1) * fprev_cs + c];
        F[c] = s * 0.25f * 0.5f;
    }
    if (g == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) Fk[(size_t)vp * 4 + c] = F[c];
    }
    const T *cl = ctx + (size_t)vt.cam_l[v] * P * C;
    const T *cr = ctx + (size_t)vt.cam_r[v] * P * C;
    Taps tl = warp_taps(X, Y, F[0], F[1], h, w, circ);
    Taps tr = warp_taps(X, Y, F[2], F[3], h, w, circ);
    T *d = dst + (size_t)vp * dst_cs;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int c = g * 8 + j;
        d[off_l + c] = to_store<T>(bilerp(cl, C, c, tl));
        d[off_r + c] = to_store<T>(bilerp(cr, C, c, tr));
    }
}

// a8: out = clamp(I_blend + 2 sigmoid(z) - 1, 0, 1), cropped to H x W.
__global__ void output_kernel(const float *ib, const float *z, int z_cs, int nv, int Hp, int Wp,
                              int H, int W, float *out) {
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

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

} // namespace

#define FVV_LAUNCH_CHECK() \
    do { count_launch(); FVV_CHECK_CUDA(cudaGetLastError()); } while (0)

int launch_prep_cams(const float *const *cams, int n_cams, int H, int W, int Hp, int Wp, float *img0,
                     float *img1, float *img2, bf16 *img0_b16, cudaStream_t st) {
    long long n = (long long)n_cams * (Hp / 4) * (Wp / 4);
    prep_cams_kernel<<<blocks_for(n, 128), 128, 0, st>>>(cams, n_cams, H, W, Hp, Wp, img0, img1, img2, img0_b16);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

template <typename T>
int launch_vib0_input(const float *img2, const ViewTab &vt, int nv, int h, int w, T *x, int cs, cudaStream_t st) {
    long long n = (long long)nv * h * w;
    vib0_input_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(img2, vt, nv, h, w, x, cs);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

template <typename T>
int launch_stage_input(const float *imgs, const float *FMp, const ViewTab &vt, int nv, int h, int w,
                       int circ, T *x, int cs, cudaStream_t st) {
    long long n = (long long)nv * h * w;
    stage_input_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(imgs, FMp, vt, nv, h, w, circ, x, cs);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

int launch_residual(const float *FMp, float *res, int nv, int h, int w, int circ, cudaStream_t st) {
    long long n = (long long)nv * h * w;
    residual_kernel<<<blocks_for(n, 256), 256, 0, st>>>(FMp, res, nv, h, w, circ);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

template <typename T>
int launch_final_blend(const float *img0, const float *FM, const ViewTab &vt, int nv, int h, int w,
                       int circ, T *u0, int cs, float *ib, cudaStream_t st) {
    long long n = (long long)nv * h * w;
    final_blend_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(img0, FM, vt, nv, h, w, circ, u0, cs, ib);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

template <typename T>
int launch_ctx_warp(const float *Fprev, int fprev_cs, float *Fk, const T *ctx, int C, const ViewTab &vt,
                    int nv, int h, int w, int circ, T *dst, int dst_cs, int off_l, int off_r, cudaStream_t st) {
    long long n = (long long)nv * h * w * (C / 8);
    ctx_warp_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(Fprev, fprev_cs, Fk, ctx, C, vt, nv, h, w, circ,
                                                           dst, dst_cs, off_l, off_r);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

int launch_output(const float *ib, const float *z, int z_cs, int nv, int Hp, int Wp, int H, int W, float *out,
                  cudaStream_t st) {
    long long n = (long long)nv * H * W;
    output_kernel<<<blocks_for(n, 256), 256, 0, st>>>(ib, z, z_cs, nv, Hp, Wp, H, W, out);
    FVV_LAUNCH_CHECK();
    return FVV_OK;
}

#define INST(T)                                                                                          \
    template int launch_vib0_input<T>(const float *, const ViewTab &, int, int, int, T *, int, cudaStream_t); \
    template int launch_stage_input<T>(const float *, const float *, const ViewTab &, int, int, int, int, T *, \
                                       int, cudaStream_t);                                              \
    template int launch_final_blend<T>(const float *, const float *, const ViewTab &, int, int, int, int, T *, \
                                       int, float *, cudaStream_t);                                     \
    template int launch_ctx_warp<T>(const float *, int, float *, const T *, int, const ViewTab &, int, int, int, \
                                    int, T *, int, int, int, cudaStream_t);
INST(float)
INST(bf16)
#undef INST

} // namespace fvv
