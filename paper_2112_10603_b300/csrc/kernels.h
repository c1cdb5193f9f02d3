// Kernel launchers (one per kernel family); all return FVV_OK or an FVV_E* code.
#pragma once
#include "common.h"

namespace fvv {

// Per-view lookup table in device memory: cameras of the view's pair and its t.
// n: the device count words {views, cameras} of a launch captured for a size bucket
// (NULL: the launch's own counts are exact).
struct ViewTab {
    const int *cam_l;
    const int *cam_r;
    const float *t;
    const int *n = nullptr;
};

// Items a kernel launched for up to n of them actually processes: the device count
// word *d (graph replay for a size bucket: the call's count, uploaded before the
// launch), else n.
__device__ __forceinline__ int dev_count(const int *d, int n) { return d ? min(__ldg(d), n) : n; }

// FP32 SIMT implicit-GEMM conv / convT (weights packed by pack_simt).
int launch_conv_simt(const ConvArgs &a, bool in_bf16, bool out_bf16, cudaStream_t st);
// direct kernel for a 3 -> 16 channel conv read from FP32 (ContextNet's first layer)
int launch_conv_c3(const ConvArgs &a, bool out_bf16, cudaStream_t st);
void pack_simt(int kind, int Ci, int Co, const float *w, float *dst);

// Frame pyramid levels (img0 = padded frame, img1 = 1/2, img2 = 1/4 box levels):
// one float4 (R, G, B, 0) per pixel.  bf16 stage inputs (x, u0) are written only
// up to the last 8-channel group holding data; the padding channels above are
// zeros from the allocation-time clear.
int launch_prep_cams(const float *const *cams, int n_cams, const int *ncam_dev, int H, int W, int Hp, int Wp,
                     float4 *img0, float4 *img1, float4 *img2, cudaStream_t st);
template <typename T>
int launch_vib0_input(const float4 *img2, const ViewTab &vt, int nv, int h, int w, T *x, int cs, cudaStream_t st);
template <typename T>
int launch_stage_input(const float4 *imgs, const float *FMp, const ViewTab &vt, int nv, int h, int w, int circ,
                       T *x, int cs, cudaStream_t st);
int launch_residual(const float *FMp, float *res, int nv, const int *nv_dev, int h, int w, int circ,
                    cudaStream_t st);
template <typename T>
int launch_final_blend(const float4 *img0, const float *FM, const ViewTab &vt, int nv, int h, int w, int circ,
                       T *u0, int cs, float *ib, cudaStream_t st);
template <typename T>
int launch_ctx_warp(const float *Fprev, int fprev_cs, float *Fk, const T *ctx, int C, const ViewTab &vt, int nv,
                    int h, int w, int circ, T *dst, int dst_cs, int off_l, int off_r, cudaStream_t st);
int launch_output(const float *ib, const float *z, int z_cs, int nv, const int *nv_dev, int Hp, int Wp, int H, int W,
                  float *const *outp, cudaStream_t st);
// Circular padding of a channel window (`bytes` per pixel from byte `coff_bytes` of pixels
// `cs_bytes` apart) into a compact (H + 2 pad) x (W + 2 pad) image with wrapped borders.
int launch_wrap_pad(const void *in, int N, const int *n_dev, int H, int W, int cs_bytes, int coff_bytes, int bytes,
                    int pad, void *out, cudaStream_t st);

} // namespace fvv
