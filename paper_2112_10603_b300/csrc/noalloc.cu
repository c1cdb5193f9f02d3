// fvv_layer_noalloc: one Table-3 layer on caller buffers without any device
// allocation.
//
// Who needs it: callers that may not call cudaMalloc themselves or through us —
// a host application that owns a fixed device-memory budget and forbids other
// allocations, a real-time frame loop that cannot afford the device-wide
// synchronisation an allocation can cause, or a plug-in running inside another
// framework's memory pool.  They cannot create an fvv_interp handle (create
// allocates the weights and the workspace), so this entry point takes the
// layer's weights straight from the caller, in the weight blob's own layout.
//
// The FP32 convolution kernel wants its weights repacked into [phase][K][C_out]
// rows.  That repacked copy is the only scratch memory the call needs; it lives in
// a fixed file-scope device array (g_noalloc_w, 4 MiB: the largest layer of
// Table 3, RefineNet's d0 with 512 x 128 x 16 weights).  Every GPU that loads the
// library holds this array until the process exits.  The CUDA runtime loads this
// file's module lazily: the first call on a device loads it, which is when the driver
// creates the array on that device (an allocation the driver makes, and one that may
// synchronise the device), and that call also looks up the array's address.  Calls
// after the first on a device allocate nothing.
#include <mutex>

#include "interp.h"

namespace fvv {

namespace {

constexpr size_t kNoallocMaxWeights = (size_t)1 << 20;
static __device__ __align__(256) float g_noalloc_w[kNoallocMaxWeights];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_w on the current device.  In host code the symbol
// name is only a host-side stand-in, so the address is looked up once per device
// (with that device current) and cached.
int noalloc_scratch(float **out) {
    int dev = -1;
    FVV_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("fvv_layer_noalloc: device ordinal %d not supported", dev);
        return FVV_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_w);
        if (e != cudaSuccess || !p) {
            set_error("fvv_layer_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return FVV_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return FVV_OK;
}

// Weights from the blob layout (conv [Co][Ci][3][3], convT [Ci][Co][4][4]) to the
// FP32 GEMM rows: conv (tap, ci) x co; convT (phase, tap, ci) x co, where phase
// (py, px) and tap (ty, tx) select kernel row ky = 1 + 2 ty (py = 0) or 2 ty
// (py = 1), and likewise the column.
__global__ void noalloc_repack_kernel(const float *w, int convt, int Ci, int Co, float *dst) {
    long long total = (long long)(convt ? 16 : 9) * Ci * Co;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int co = i % Co;
    long long r = i / Co;
    int ci = r % Ci;
    int g = r / Ci; // tap (conv) or phase * 4 + tap (convT)
    float v;
    if (!convt) {
        v = w[((size_t)co * Ci + ci) * 9 + g];
    } else {
        int phase = g >> 2, tap = g & 3;
        int py = phase >> 1, px = phase & 1, ty = tap >> 1, tx = tap & 1;
        int ky = py == 0 ? 1 + 2 * ty : 2 * ty, kx = px == 0 ? 1 + 2 * tx : 2 * tx;
        v = w[((size_t)ci * Co + co) * 16 + ky * 4 + kx];
    }
    dst[i] = v;
}

} // namespace

} // namespace fvv

using namespace fvv;

extern "C" int fvv_layer_noalloc(int layer, const float *w, const float *b, const float *in, int in_cs, int in_coff,
                                 int n, int H, int W, float *out, int out_cs, int out_coff, void *stream) {
    clear_error();
    if (layer < 0 || layer >= kNumLayers || !w || !b || !in || !out) {
        set_error("fvv_layer_noalloc: bad layer index or NULL pointer");
        return FVV_EINVAL;
    }
    const LayerDef &L = kLayers[layer];
    const size_t nw = (size_t)L.ci * L.co * (L.kind == K_CONV ? 9 : 16);
    if (nw > kNoallocMaxWeights) {
        set_error("fvv_layer_noalloc: layer %s has %zu weights, the fixed scratch holds %zu", L.name, nw,
                  kNoallocMaxWeights);
        return FVV_ESHAPE;
    }
    if (n < 1 || H < 1 || W < 1 || in_coff < 0 || out_coff < 0 || in_cs < in_coff + L.ci || out_cs < out_coff + L.co) {
        set_error("fvv_layer_noalloc: layer %s: bad sizes", L.name);
        return FVV_ESHAPE;
    }
    if (L.kind == K_CONV && L.stride == 2 && (H % 2 || W % 2)) {
        set_error("fvv_layer_noalloc: stride-2 layer %s needs even H, W", L.name);
        return FVV_ESHAPE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the scratch address below is the current device's; a stream of another device
    // would have the kernels read and write that device's copy of the array
    int cur = -1, sdev = -1;
    FVV_CHECK_CUDA(cudaGetDevice(&cur));
    FVV_CHECK_CUDA(cudaStreamGetDevice(st, &sdev));
    if (sdev != cur) {
        set_error("fvv_layer_noalloc: stream belongs to device %d, current device is %d", sdev, cur);
        return FVV_EINVAL;
    }
    float *scratch = nullptr;
    FVV_TRY(noalloc_scratch(&scratch));
    noalloc_repack_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(w, L.kind == K_CONVT, L.ci, L.co, scratch);
    FVV_CHECK_CUDA(cudaGetLastError());
    ConvArgs a{};
    a.in = in; a.in_cs = in_cs; a.in_coff = in_coff;
    a.out = out; a.out_cs = out_cs; a.out_coff = out_coff;
    a.w = scratch;
    a.bias = b;
    a.N = n; a.H = H; a.W = W; a.Ci = L.ci; a.Co = L.co;
    a.kind = L.kind; a.stride = L.stride; a.relu = L.relu; a.circ = 0;
    if (L.kind == K_CONV) { a.Ho = (H - 1) / L.stride + 1; a.Wo = (W - 1) / L.stride + 1; }
    else { a.Ho = 2 * H; a.Wo = 2 * W; }
    if (layer == kCtx) return launch_conv_c3(a, false, st);
    return launch_conv_simt(a, false, false, st);
}
