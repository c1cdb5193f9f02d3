// Sampling helpers shared by the memory-bound kernels and the fused conv epilogues.
//
// Conventions (the paper leaves them open; one reading, used everywhere):
//  * backward warp: out(x, y) = I(x + F_x, y + F_y), bilinear, pixel centres at
//    integer indices; the sample point is split as x + floor(F_x) and weight
//    F_x - floor(F_x); taps clamp to the border (zero mode) or wrap (circular);
//  * x2 upsampling: fine pixel X samples coarse coordinate X/2 - 1/4 (half-pixel
//    centres), taps clamp or wrap; flow values are doubled by the caller.
#pragma once
#include "common.h"

namespace fvv {

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(bf16 v) { return __bfloat162float(v); }

__device__ __forceinline__ int fix_index(int i, int n, int circ) {
    if (circ) { i %= n; return i < 0 ? i + n : i; }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Bilinear tap set: four pixel indices (row-major in the sampled grid) + weights.
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

// The same taps with the padding mode fixed at compile time (no per-index branch).
template <bool CIRC> __device__ __forceinline__ int fix_index_t(int i, int n) {
    if (CIRC) { i %= n; return i < 0 ? i + n : i; }
    return min(max(i, 0), n - 1);
}
template <bool CIRC> __device__ __forceinline__ Taps warp_taps_t(int x, int y, float fx, float fy, int H, int W) {
    const float lim = CIRC ? 16777216.f : (float)(max(H, W) + 4);
    fx = fminf(fmaxf(fx, -lim), lim);
    fy = fminf(fmaxf(fy, -lim), lim);
    const float flx = floorf(fx), fly = floorf(fy);
    Taps t;
    t.lx = fx - flx;
    t.ly = fy - fly;
    const int x0 = x + (int)flx, y0 = y + (int)fly;
    const int xa = fix_index_t<CIRC>(x0, W), xb = fix_index_t<CIRC>(x0 + 1, W);
    const int ya = fix_index_t<CIRC>(y0, H), yb = fix_index_t<CIRC>(y0 + 1, H);
    t.o00 = ya * W + xa; t.o01 = ya * W + xb; t.o10 = yb * W + xa; t.o11 = yb * W + xb;
    return t;
}
template <bool CIRC> __device__ __forceinline__ Taps up_taps_t(int X, int Y, int h, int w) {
    Taps t;
    const int x0 = (X >> 1) - ((X & 1) ? 0 : 1), y0 = (Y >> 1) - ((Y & 1) ? 0 : 1);
    t.lx = (X & 1) ? 0.25f : 0.75f;
    t.ly = (Y & 1) ? 0.25f : 0.75f;
    const int xa = fix_index_t<CIRC>(x0, w), xb = fix_index_t<CIRC>(x0 + 1, w);
    const int ya = fix_index_t<CIRC>(y0, h), yb = fix_index_t<CIRC>(y0 + 1, h);
    t.o00 = ya * w + xa; t.o01 = ya * w + xb; t.o10 = yb * w + xa; t.o11 = yb * w + xb;
    return t;
}

template <typename T>
__device__ __forceinline__ float bilerp(const T *img, int cs, int c, const Taps &t) {
    float a = to_f(img[(size_t)t.o00 * cs + c]), b = to_f(img[(size_t)t.o01 * cs + c]);
    float d = to_f(img[(size_t)t.o10 * cs + c]), e = to_f(img[(size_t)t.o11 * cs + c]);
    return (1.f - t.ly) * ((1.f - t.lx) * a + t.lx * b) + t.ly * ((1.f - t.lx) * d + t.lx * e);
}

// Frame pyramid levels hold one float4 (R, G, B, 0) per pixel: one 16-byte load per
// bilinear tap.  Same arithmetic, channel by channel, as bilerp().
__device__ __forceinline__ float3 bilerp_rgb(const float4 *img, const Taps &t) {
    float4 a = __ldg(img + t.o00), b = __ldg(img + t.o01), d = __ldg(img + t.o10), e = __ldg(img + t.o11);
    const float wx0 = 1.f - t.lx, wy0 = 1.f - t.ly;
    float3 r;
    r.x = wy0 * (wx0 * a.x + t.lx * b.x) + t.ly * (wx0 * d.x + t.lx * e.x);
    r.y = wy0 * (wx0 * a.y + t.lx * b.y) + t.ly * (wx0 * d.y + t.lx * e.y);
    r.z = wy0 * (wx0 * a.z + t.lx * b.z) + t.ly * (wx0 * d.z + t.lx * e.z);
    return r;
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

} // namespace fvv
