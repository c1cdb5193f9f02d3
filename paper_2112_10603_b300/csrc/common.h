// Internal definitions shared by the library's translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "fvv.h"

namespace fvv {

// Thread-local error message (fvv_last_error).
void set_error(const char *fmt, ...);
void clear_error();

#define FVV_CHECK_CUDA(call)                                                              \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ::fvv::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return FVV_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

#define FVV_TRY(expr)               \
    do {                            \
        int rc_ = (expr);           \
        if (rc_ != FVV_OK) return rc_; \
    } while (0)

typedef __nv_bfloat16 bf16;

// A tensor of N images, H x W pixels, each pixel `cs` elements apart; the view
// starts at channel `coff` of each pixel.  Element type given by the kernel.
struct TView {
    void *p;
    int N, H, W, cs, coff;
};

enum LayerKind { K_CONV = 0, K_CONVT = 1 };

// One convolution launch (3x3 pad 1 stride 1/2, or 4x4 stride-2 transposed).
struct ConvArgs {
    const void *in;
    int in_cs, in_coff;
    void *out;
    int out_cs, out_coff;
    const void *w;      // packed weights (layout depends on the kernel)
    const float *bias;  // Co floats
    int N, H, W;        // input images and size
    int Ci, Co, Ho, Wo; // Ho, Wo = output size
    int kind, stride, relu, circ;
    const int *n_dev;   // device count of images actually run (graph replay of a size bucket), or NULL
};

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Launch counter for the last run (fvv_interp_last_launches).
extern thread_local int g_launches;
inline void count_launch(int n = 1) { g_launches += n; }

} // namespace fvv
