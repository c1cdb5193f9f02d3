// Network executor: layer table, packed weights, workspace and the layer schedule.
#pragma once
#include <map>
#include <vector>

#include "common.h"
#include "kernels.h"

namespace fvv {

struct LayerDef {
    const char *name;
    int kind, ci, co, stride, relu;
};

constexpr int kNumLayers = 51;
extern const LayerDef kLayers[kNumLayers];
// first layer index of each sub-network
constexpr int kVib0 = 0, kVib1 = 10, kVib2 = 20, kCtx = 30, kRef = 38;

size_t blob_floats();

// Fused epilogues of the tensor-core convolutions.
enum { EPI_STORE = 0, EPI_RESID = 1, EPI_OUTPUT = 2 };
struct TcEpi {
    int mode = EPI_STORE;
    const float *fm_prev = nullptr; // EPI_RESID: previous stage F, M (half grid, 5 ch FP32)
    const float *ib = nullptr;      // EPI_OUTPUT: I_blend on the padded grid (3 ch FP32)
    float *const *final_out_ref = nullptr; // EPI_OUTPUT: device slot holding the cropped n x crop_h x crop_w x 3 output
    int crop_h = 0, crop_w = 0;
};

// Packed weights of one layer for the tensor-core kernels.
struct TcWeights {
    void *w = nullptr;      // device, [phase*taps][Co_pad][Ci_pad] bf16 (or fp8) K-major
    float *scale = nullptr; // FP8: per-output-channel dequantisation scale
    alignas(64) unsigned char map[128] = {}; // host CUtensorMap of w (B operand)
    alignas(64) unsigned char map3[128] = {};     // same, box of 3 consecutive taps (grouped halo stages)
    // folded column taps: per row tap ky one slice of kxf_n rows (kx * G + j, G = output
    // columns per tap), [3][kxf_n][Ci_pad]; map_k boxes the 3 row taps of one channel block
    void *wk = nullptr;
    alignas(64) unsigned char map_k[128] = {};
    int kxf_n = 0;
    // per-tap stride-2 input convs: wcopies copies of w side by side ([copies][taps]...),
    // CTAs read copy blockIdx % wcopies (spreads the hot weight lines over more of L2)
    void *wrep = nullptr;
    alignas(64) unsigned char map_rep[128] = {};
    int wcopies = 1;
    int ci_pad = 0, co_pad = 0;
};

} // namespace fvv

struct fvv_interp {
    int H = 0, W = 0, Hp = 0, Wp = 0;
    fvv_opts o{};
    // weights
    float *w32 = nullptr;    // SIMT-packed FP32 weights, all layers
    float *bias = nullptr;   // all biases
    size_t w_off[fvv::kNumLayers] = {}, b_off[fvv::kNumLayers] = {};
    fvv::TcWeights tc[fvv::kNumLayers];
    // per-camera buffers
    float4 *img0 = nullptr, *img1 = nullptr, *img2 = nullptr; // (R, G, B, 0) per pixel
    void *ctx[4] = {}, *ctxt = nullptr;
    // per-view buffers
    void *xb = nullptr, *xb0 = nullptr, *ta = nullptr, *ma = nullptr, *mb = nullptr;
    float *fm[3] = {}, *ib = nullptr, *fk[4] = {}, *z = nullptr;
    void *u[5] = {};
    // view table and camera pointer table (device) + pinned host staging
    int *d_cam_l = nullptr, *d_cam_r = nullptr;
    float *d_t = nullptr;
    const float **d_cams = nullptr;
    char *h_stage = nullptr;
    cudaEvent_t stage_done = nullptr;
    // staging for host-buffer calls: slot 0 is d_in/d_out; the pipelined calls alternate
    // between two slots, copies on their own streams so a copy-out overlaps the next forward
    float *d_in = nullptr, *d_out = nullptr;
    struct HostSlot {
        float *d_in = nullptr, *d_out = nullptr;
        cudaEvent_t in_ready = nullptr, fwd_done = nullptr, out_done = nullptr;
        long long ticket = -1; // the call that used the slot last
    };
    HostSlot hs[2];
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    long long host_calls = 0;
    int *d_err = nullptr; // device error word written by bounded waits
    // fault injection (fvv_interp_inject_stall): armed for the next fvv_interp_layer call,
    // live (stall_now) only during that call, so no captured graph ever holds it
    long long stall_cycles = 0, stall_now = 0;
    size_t dev_bytes = 0;
    int last_launches = 0;
    std::vector<void *> allocs;
    // per-layer event timing (fvv_interp_profile)
    struct ProfRec { int layer; double flops; cudaEvent_t a, b; };
    bool profiling = false;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    // output pointer slot read by the last kernel (so a captured graph serves any buffer)
    float **d_outp = nullptr;
    // CUDA graphs, one per view-count bucket (and cached-frames flag), captured on cap_stream;
    // d_cnt = {views, cameras} of the current call, read by every kernel of a bucket graph
    struct Graph { cudaGraphExec_t exec; int launches; };
    std::map<long long, Graph> graphs;
    int *d_cnt = nullptr;
    bool counts_live = false; // set while a bucket graph is captured
    // circular mode on the tensor-core path: each conv's input window with a wrapped border
    void *cpad = nullptr;
    size_t cpad_bytes = 0;
    long long graph_captures = 0;
    cudaStream_t cap_stream = nullptr;
    // ContextNet runs on its own stream beside the VIBlocks (forked after the frame pyramid,
    // joined before RefineNet's context warps); in a captured graph: two branches
    cudaStream_t ctx_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // tile rectangle per layer: log2 of the tile width (-1: fewest-tiles default);
    // tile_force >= 0 overrides every layer (used while autotuning)
    signed char tile_tw[fvv::kNumLayers];
    int tile_force = -1;
    // set by the server while the frames (and so the pyramid and ContextNet features
    // already in this handle's workspace) are those of its previous run
    int skip_cams = 0;
    // FP8 (E4M3) path for the 256-channel VIB convs: weights with per-output-channel
    // scales s_w, activations with per-tensor scales s_a from calibration
    fvv::TcWeights tc8[fvv::kNumLayers];
    std::vector<float> s_w[fvv::kNumLayers];  // host copy of the weight scales
    float s_a[fvv::kNumLayers] = {};          // input scale of each FP8 layer
    float q_out[fvv::kNumLayers] = {};        // 1 / s_a of the consumer (producers of FP8 inputs)
    float *q_acc[fvv::kNumLayers] = {};       // device: s_a * s_w[co]
    float *d_amax = nullptr;                  // device: max |output| per layer while calibrating
    int fp8_ready = 0, calibrating = 0;
    // recursive t mode: generated intermediate views
    float *rec_buf = nullptr;
    int rec_cap = 0;
};

namespace fvv {
int interp_forward(fvv_interp *h, int n_cams, int nv, cudaStream_t st);
int dalloc(fvv_interp *h, void **p, size_t bytes);
int tc_prepare(fvv_interp *h, const float *blob);
int tc_conv(fvv_interp *h, int layer, const void *in, int in_cs, int in_coff, int N, int Hin, int Win,
            void *out, int out_cs, int out_coff, bool out_f32, cudaStream_t st, const TcEpi *epi = nullptr);
// VIBlock s > 0: the stage input (x2 upsampled F, M of the previous stage, both frames
// warped, the frames, t) computed by the loader of the block's first conv (c0) itself;
// out: the c0 output (bf16, or E4M3 for an FP8 consumer), out_cs = 128
bool stage_conv_layer(const fvv_interp *h, int layer);
// RefineNet's output conv with the network output fused (csrc/out_conv.cu): whether the
// dedicated kernel takes this call, and its launch (in: n x hp x wp x 16 bf16; ib: I_blend
// on the padded grid; out_ref: device slot holding the cropped output pointer)
bool out_conv_ok(const fvv_interp *h, int layer, int in_cs, int n, int hp, int wp, int crop_h, int crop_w);
int tc_out_conv(fvv_interp *h, int layer, const void *in, int n, int hp, int wp, const float *ib,
                float *const *out_ref, int crop_h, int crop_w, const int *n_dev, cudaStream_t st);
// RefineNet d3 (all-phase transposed conv 64 -> 16, column taps folded into N;
// csrc/convt_fold.cu): whether the dedicated kernel takes this call, and its launch
// (in: n x hin x win pixels of in_cs bf16 channels, the first 64 used; out: bf16,
// n x 2 hin x 2 win x 16)
bool convt_fold_ok(const fvv_interp *h, int layer, int in_cs, int in_coff, int out_cs, int out_coff, bool out_f32);
int tc_convt_fold(fvv_interp *h, int layer, const void *in, int in_cs, int n, int hin, int win, void *out,
                  const int *n_dev, cudaStream_t st);
// VIBlock t1 with the Eq. 2 update fused, rows walked down 120-pixel strips
// (csrc/t1_fold.cu): whether the dedicated kernel takes this call, and its launch
// (in: n x hin x win x 128 bf16; fm_prev: F^{s-1}, M^{s-1} on the same grid, 5 FP32;
// out: F^s, M^s, n x 2 hin x 2 win x 5 FP32)
bool vib_t1_ok(const fvv_interp *h, int layer, int in_cs, int in_coff, int n, int hin, int win, int out_cs,
               int out_coff, bool out_f32);
int tc_vib_t1(fvv_interp *h, int layer, const void *in, int n, int hin, int win, const float *fm_prev, float *out,
              const int *n_dev, cudaStream_t st);
int tc_stage_conv(fvv_interp *h, int layer, const float4 *imgs, const float *fm_prev, const ViewTab &vt, int nv,
                  int hs, int ws, int circ, void *out, int out_cs, cudaStream_t st);
bool tc_all_phases(int layer); // transposed conv run as one 3x3 conv over all 4 phases
bool tc_kxf_layer(int layer);   // column taps folded into N (tiles of 120 pixels)
// FP8 layers: every VIBlock conv with 128 or 256 input channels -- c1 (128 -> 256,
// stride 2), the six 256 -> 256 convs m0-m5, t0 (256 -> 128 transposed) and t1 (128 -> 5
// transposed, all phases); their producers are the layer before (c0 .. t0) and write
// E4M3 codes.
inline bool fp8_layer(int li) { return li < kCtx && li % 10 >= 1; }
// border (pixels) of the wrapped copies the tensor-core convs read in circular mode: even,
// so that the stride-2 pixel-pair maps stay aligned to pairs
constexpr int kCircPad = 2;
// Device count word a conv layer's launch reads while a size-bucket graph is captured:
// cameras for ContextNet's layers, views for every other layer; NULL otherwise.
inline const int *count_word(const fvv_interp *h, int li) {
    if (!h->counts_live) return nullptr;
    return h->d_cnt + (li >= kCtx && li < kCtx + 8 ? 1 : 0);
}
inline bool feeds_fp8(int li) { return li < kCtx && li % 10 <= 8; }
} // namespace fvv
