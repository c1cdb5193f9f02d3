// Tensor-core convolutions: tcgen05 BF16 implicit GEMM, FP32 accumulation in TMEM.
//
// GEMM view of a Table-3 layer: M = output pixels (128 per tile, a TH x TW
// rectangle of one image), N = C_out (one tile, <= 256), K = taps x C_in.
// K is walked in blocks of one tap x CK channels; for every block TMA copies
//   A: the input patch of the tile shifted by the tap (tiled 4-D map over
//      [N][H][W][C]; out-of-range rows/columns arrive as zeros = conv padding),
//   B: the tap's [C_out][CK] weight slice,
// into 128B/64B/32B-swizzled shared memory, and one thread issues CK/16
// tcgen05.mma (M=128, N=C_out, K=16).
//   * stride-2 conv: the input is viewed as pixel pairs [N][H/2][2][W/2][2C]
//     (5-D map), so tap (ky, kx) is a plain box at (pair column ox-1 or ox,
//     half = kx!=1, row pair oy-1 or oy, row parity = ky!=1);
//   * 4x4 stride-2 transposed conv: 4 output phases, each a 2x2-tap conv on the
//     input grid (phase p: taps read rows q - t (p=0) or q + 1 - t (p=1)); with few
//     output channels all 4 phases at once as one 3x3 conv (MODE_T3, N = 4 C_out);
//   * E4M3 operands (kind::f8f6f4, K = 32 per MMA) for the FP8 layers.
// Halo tiles, grouped stages, the stride-2 pair halo and the TMA-store epilogue are
// described at the kernel template below.
// Warp roles: warp 0 = TMA producer, warp 1 = MMA issuer (+ TMEM owner),
// warps 2-5 = epilogue (TMEM -> registers -> bias, ReLU, BF16/FP32 -> global).
// The accumulator is double-buffered in TMEM so the epilogue of one tile runs
// under the main loop of the next; CTAs loop over tiles (persistent grid).
// Every mbarrier wait is bounded: on expiry the kernel records an error code in
// global memory, tells the other roles to stop, drains and frees TMEM, returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <cstring>
#include <vector>

#include "interp.h"
#include "sampling.h"
#include "tc_ptx.h"
#include "tc_wait.h"

namespace fvv {

namespace {

// MODE_T3: a transposed conv with few output channels computed for all 4 output
// phases at once as a 3x3 conv over the input grid with N = 4 x C_out (phase-major
// columns; each phase's weights are zero on the 5 taps it does not use).
enum { MODE_S1 = 0, MODE_S2 = 1, MODE_T = 2, MODE_T3 = 3 };
constexpr int kThreads = 192;

// Unsigned division by a divisor fixed at launch, as a multiply-high and shifts
// (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994,
// the round-up method for N = 32): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) with t = mulhi(m, n); exact for
// every 32-bit n.
struct FastDiv {
    uint32_t d = 1, m = 1, s1 = 0, s2 = 0;
    FastDiv() = default;
    explicit FastDiv(uint32_t div) : d(div) {
        uint32_t l = 0;
        while ((1ull << l) < div) ++l;
        m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
        s1 = l < 1 ? l : 1;
        s2 = l > 1 ? l - 1 : 0;
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        const uint32_t t = __umulhi(m, n);
        return (t + ((n - t) >> s1)) >> s2;
    }
};

struct TcParams {
    int mode;
    int n_img, gh, gw;      // GEMM grid (conv: output size; convT: input size)
    int th_log, tw_log;     // tile = (1 << th_log) x (1 << tw_log) = 128 pixels
    int tiles_y, tiles_x, num_tiles;
    FastDiv fdx, fdy;       // division by tiles_x, tiles_y
    FastDiv fdco;           // division by co (the phase of an all-phase transposed conv's column)
    int nck_log;            // log2 of the channel blocks per tap (a power of two)
    int nck;                // channel blocks per tap
    int taps;               // 9 (conv, MODE_T3) or 4 (convT phase)
    int in_cs, in_coff;     // input pixel stride / channel offset (elements)
    int co;                 // real output channels (per phase in MODE_T3)
    int relu, out_f32, vec_ok;
    void *out;
    int out_cs, out_coff, out_h, out_w;
    const float *bias;
    int *err;
    TcEpi epi;
    // FP8 (E4M3) operands: the accumulator is in units of s_a * s_w[co]
    const float *acc_scale; // per output channel, NULL for BF16 operands
    int out_fp8;            // store E4M3 codes of value * out_q (saturating)
    float out_q;
    float *amax;            // calibration: running max |output| (NULL: off)
    int tma_store;          // epilogue stages each warp's 32 rows in shared memory, TMA stores them
    int kxf;                // column taps folded into N: tiles of kKxfTile output pixels of one row
    int wcopies;            // per-tap stride-2 path: weight copies (CTA b reads copy b % wcopies)
    const int *n_dev;       // device count of images actually run (graph replay of a size bucket), or NULL
    int ipad;               // circular mode: the input carries a wrapped border of ipad pixels (A coordinates
                            // shift by ipad pixels, ipad / 2 pixel pairs on the stride-2 maps); 0 otherwise
    long long stall_cycles; // fault injection (tests): > 0 makes the MMA warp wait on a barrier
                            // nothing signals, for at most this many cycles, then abort
};

// Column taps folded into N (3x3 stride-1 convs and the all-phase transposed convs with
// few output channels): the weight slice of row tap ky holds the three column taps
// side by side (N = 3 G, G = output columns per tap), so ONE MMA per K step covers all
// three and the A operand is fetched a third as often.  Row r of the accumulator is then
// the partial sum of input pixel r for every column tap; output pixel r sums tap 0 of
// row r - 1, tap 1 of row r and tap 2 of row r + 1 -- neighbouring TMEM lanes, i.e.
// neighbouring threads of an epilogue warp (warp shuffles).  Each warp's 32 rows are
// loaded as their own box of 32 input pixels, overlapping the next warp's by 2, so a
// warp never needs another warp's rows: lanes 1..30 produce outputs, 120 per tile.
constexpr int kKxfTile = 120;

// 16 values times q as E4M3 codes (paired conversions, RNE, saturating), value j in byte j
__device__ __forceinline__ uint4 e4m3x16(const float (&v)[16], float q) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * k] * q, v[4 * k + 1] * q), __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi =
            __nv_cvt_float2_to_fp8x2(make_float2(v[4 * k + 2] * q, v[4 * k + 3] * q), __NV_SATFINITE, __NV_E4M3);
        w[k] = lo | (hi << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ uint8_t to_e4m3(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

struct __align__(16) Bars { // (16: the staged biases that follow it are read as float4)
    uint64_t full[16], empty[16], tmem_full[2], tmem_empty[2], drain;
    uint64_t never; // signalled by nothing: the fault-injection wait
    uint32_t tmem_base;
    int abort;
};


// Tile t of a launch.  The 4 output phases of a per-phase transposed conv are the
// innermost index: the four tiles of one pixel region run on neighbouring CTAs at the
// same time and share its input in L2 (phase-major order streamed the whole input from
// DRAM once per phase when it exceeds L2); with a grid that is a multiple of 4 every
// persistent CTA also keeps one phase, i.e. one set of weight slices.
__device__ __forceinline__ void tile_coords(const TcParams &p, int t, int &phase, int &n, int &y0, int &x0) {
    const bool t4 = p.mode == MODE_T;
    phase = t4 ? t & 3 : 0;
    const uint32_t r = t4 ? (uint32_t)t >> 2 : (uint32_t)t;
    const uint32_t r1 = p.fdx.div(r), r2 = p.fdy.div(r1);
    const int tx = (int)(r - r1 * (uint32_t)p.tiles_x), ty = (int)(r1 - r2 * (uint32_t)p.tiles_y);
    n = (int)r2;
    y0 = ty << p.th_log;
    x0 = p.kxf ? tx * kKxfTile : tx << p.tw_log;
}

// Eq. 2 update of a 4-phase transposed conv with 5 outputs (the VIB t1 layer): the
// pixel (gy, gx) of the half grid owns the 4 fine pixels (2 gy + py, 2 gx + px); their
// x2 upsampling reads the 3x3 neighbourhood of (gy, gx) in the previous stage's F, M,
// fetched into nb before the accumulator is ready.  row32: the warp's lanes hold 32
// consecutive pixels of one row (each lane loads its own column, neighbours by shuffle).
__device__ __forceinline__ void resid_nb(const TcParams &p, int n, int gy, int gx, int lane, bool row32,
                                         float (&nb)[3][3][5]) {
    const int h2 = p.gh, w2 = p.gw;
    const float *fm = p.epi.fm_prev + (size_t)n * h2 * w2 * 5;
    if (row32) {
        const int xc = min(max(gx, 0), w2 - 1);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int yy = min(max(gy + a - 1, 0), h2 - 1);
            const float *src = fm + ((size_t)yy * w2 + xc) * 5;
#pragma unroll
            for (int k = 0; k < 5; ++k) nb[a][1][k] = __ldg(src + k);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                nb[a][0][k] = __shfl_up_sync(0xffffffffu, nb[a][1][k], 1);
                nb[a][2][k] = __shfl_down_sync(0xffffffffu, nb[a][1][k], 1);
            }
        if (lane == 0 || lane == 31) {
            const int b = lane == 0 ? 0 : 2;
            const int xx = lane == 0 ? max(xc - 1, 0) : min(xc + 1, w2 - 1);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int yy = min(max(gy + a - 1, 0), h2 - 1);
#pragma unroll
                for (int k = 0; k < 5; ++k) nb[a][b][k] = __ldg(fm + ((size_t)yy * w2 + xx) * 5 + k);
            }
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                int yy = min(max(gy + a - 1, 0), h2 - 1), xx = min(max(gx + b - 1, 0), w2 - 1);
                const float *src = fm + ((size_t)yy * w2 + xx) * 5;
#pragma unroll
                for (int k = 0; k < 5; ++k) nb[a][b][k] = __ldg(src + k);
            }
    }
}

// F^s, M^s = up(F^{s-1}) x 2, up(M^{s-1}) + Res^s for accumulator column col (phase
// col / 5, channel col % 5) of a pixel whose neighbourhood is nb
__device__ __forceinline__ float resid_value(const float (&nb)[3][3][5], int col, float acc, float sc, float bias) {
    const int pj = col / 5, co = col % 5, py = pj >> 1, px = pj & 1;
    const float ly = py ? 0.25f : 0.75f, lx = px ? 0.25f : 0.75f;
    float up = (1.f - ly) * ((1.f - lx) * nb[py][px][co] + lx * nb[py][px + 1][co]) +
               ly * ((1.f - lx) * nb[py + 1][px][co] + lx * nb[py + 1][px + 1][co]);
    return acc * sc + bias + up * (co < 4 ? 2.f : 1.f);
}
// Bias and dequantisation scale (1 without) of output channel co: from the copies staged in
// shared memory (SB: sb, ss are their shared addresses), or from global memory.
template <bool SB> __device__ __forceinline__ float bias_of(const TcParams &p, uint32_t sb, int co) {
    return SB ? ptx::lds_f32(sb + 4 * co) : __ldg(p.bias + co);
}
template <bool SB> __device__ __forceinline__ float scale_of(const TcParams &p, uint32_t ss, int co) {
    return SB ? ptx::lds_f32(ss + 4 * co) : (p.acc_scale ? __ldg(p.acc_scale + co) : 1.f);
}
// Biases and scales of 16 consecutive output channels co0 .. co0 + 15 (co0 a multiple of
// 16): from the staged copies as four 16-byte broadcast loads each (SB), the scales only
// for E4M3 layers (F8; 1 without); else through the scalar paths above.
template <bool SB, int F8>
__device__ __forceinline__ void bias_scale16(const TcParams &p, uint32_t sb, uint32_t ss, int co0, float (&b)[16],
                                             float (&sc)[16]) {
    if (SB) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = ptx::lds_v4f(sb + 4 * (co0 + 4 * k));
            b[4 * k] = v.x; b[4 * k + 1] = v.y; b[4 * k + 2] = v.z; b[4 * k + 3] = v.w;
            if (F8) {
                const float4 w = ptx::lds_v4f(ss + 4 * (co0 + 4 * k));
                sc[4 * k] = w.x; sc[4 * k + 1] = w.y; sc[4 * k + 2] = w.z; sc[4 * k + 3] = w.w;
            } else {
                sc[4 * k] = sc[4 * k + 1] = sc[4 * k + 2] = sc[4 * k + 3] = 1.f;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            b[j] = bias_of<SB>(p, sb, co0 + j);
            sc[j] = scale_of<SB>(p, ss, co0 + j);
        }
    }
}
template <bool SB>
__device__ __forceinline__ void resid_store(const TcParams &p, uint32_t sb, uint32_t ss, const float (&nb)[3][3][5],
                                            int n, int gy, int gx, int col, float acc) {
    const int pj = col / 5, co = col % 5, py = pj >> 1, px = pj & 1;
    size_t pix = ((size_t)n * p.out_h + 2 * gy + py) * p.out_w + 2 * gx + px;
    ((float *)p.out)[pix * p.out_cs + p.out_coff + co] =
        resid_value(nb, col, acc, scale_of<SB>(p, ss, co), bias_of<SB>(p, sb, co));
}

// One output element of the epilogue (scalar path): bias, ReLU, then store, or
// the fused Eq. 2 update.
template <bool SB>
__device__ __forceinline__ void epi_elem(const TcParams &p, uint32_t sb, uint32_t ss, int n, int oy, int ox, int co,
                                         float acc) {
    float x = acc * scale_of<SB>(p, ss, co) + bias_of<SB>(p, sb, co);
    if (p.relu) x = fmaxf(x, 0.f);
    if (p.amax) atomicMax(reinterpret_cast<int *>(p.amax), __float_as_int(fabsf(x)));
    size_t pix = ((size_t)n * p.out_h + oy) * p.out_w + ox;
    if (p.epi.mode == EPI_RESID) {
        // F^s, M^s = up(F^{s-1}) x 2, up(M^{s-1}) + Res^s; previous stage on the half grid
        int h2 = p.out_h / 2, w2 = p.out_w / 2;
        const float *fm = p.epi.fm_prev + (size_t)n * h2 * w2 * 5;
        Taps u = up_taps(ox, oy, h2, w2, 0);
        x += bilerp(fm, 5, co, u) * (co < 4 ? 2.f : 1.f);
        ((float *)p.out)[pix * p.out_cs + p.out_coff + co] = x;
    } else if (p.out_f32) {
        ((float *)p.out)[pix * p.out_cs + p.out_coff + co] = x;
    } else if (p.out_fp8) {
        ((uint8_t *)p.out)[pix * p.out_cs + p.out_coff + co] = to_e4m3(x * p.out_q);
    } else {
        ((bf16 *)p.out)[pix * p.out_cs + p.out_coff + co] = __float2bfloat16_rn(x);
    }
}

// MT = 128-pixel row blocks per tile (1 or 2): with MT = 2 each weight slice in
// shared memory feeds two MMAs (two accumulators), halving weight traffic per FLOP.
// The accumulators are double-buffered (ACCB = 2) when TMEM has room.
template <int BN, int MT> struct AccCfg {
    static constexpr int ACCB = 2 * MT * BN <= 512 ? 2 : 1;
    static constexpr int COLS_USED = ACCB * MT * BN;
    static constexpr uint32_t TMEM_COLS =
        COLS_USED <= 32 ? 32 : (COLS_USED <= 64 ? 64 : (COLS_USED <= 128 ? 128 : (COLS_USED <= 256 ? 256 : 512)));
};

// F8 = 1: E4M3 operands (kind::f8f6f4, K = 32 per MMA), else BF16 (kind::f16, K = 16);
// either way one MMA consumes 32 bytes of every operand row.
// HALO = 1 (stride-1 3x3 taps, MT x 128-pixel tiles, 32/64/128-byte rows): one TMA box of
// MT image rows x 130 pixels per (row tap ky, channel block) serves the three column
// taps kx, whose A operands start 0, 1, 2 rows into each 130-row block; A boxes
// (STAGES ring) and B slices (STAGES_B ring) are pipelined separately.  K order is
// (ky, block, kx) on both paths.  With MT = 2 each weight slice feeds two MMAs.
// TS = 1: shared-memory staging for the TMA-store epilogue (used when p.tma_store).
// GRP = 2: the same with the nine weight slices of a one-block layer resident in shared
// memory (loaded once per CTA); a stage is the A box alone.
// GRP = 1 (halo, small N): one stage holds a (row tap, channel block)'s A box AND its
// three weight slices, so the MMA thread syncs once per 3 x (row bytes / 32) MMAs.
// S2H = 1 (stride-2 3x3 conv whose input pixel is one channel block of 16 or 32 channels):
// the tile is one row of 128 output pixels; per row tap ky ONE box of 129 pixel PAIRS
// (the 5-D pair view, pair rows of 64 or 128 bytes) feeds the three column taps: kx = 1
// reads the even pixel of pairs 1..128, kx = 0 / 2 the odd pixel of pairs 0..127 / 1..128
// (descriptor start +1 row and/or + one pixel's bytes).  The nine weight slices stay
// resident in shared memory (loaded once per CTA).  K order (ky, kx, k) as on the
// per-tap path.
// KXF = number of channel blocks (0: off): column taps folded into N (kKxfTile), on the
// resident-weight grouped path (GRP = 2): a stage is the four 32-pixel boxes of one
// (row tap, channel block), the weights are 3 x KXF folded slices of N rows.
template <int BN, int CK, int MT, int STAGES, int CTAS, int F8, int HALO = 0, int STAGES_B = STAGES, int TS = 0,
          int GRP = 0, int S2H = 0, int KXF = 0>
__global__ void __launch_bounds__(kThreads, CTAS)
conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmC, const TcParams p) {
    constexpr int ES = F8 ? 1 : 2;                 // operand element bytes
    constexpr int ROW_BYTES = CK * ES;
    constexpr uint32_t A_BYTES = S2H ? 129 * 2 * ROW_BYTES
                                     : (HALO && !KXF ? 130 * MT * ROW_BYTES : 128 * MT * ROW_BYTES),
                       B_BYTES = BN * ROW_BYTES;
    constexpr int HROW = 130; // pixels per row of a halo box
    constexpr int NB = 3;     // weight slices (column taps) per halo box
    constexpr uint32_t A_STRIDE = (A_BYTES + 1023) & ~1023u, B_STRIDE = (B_BYTES + 1023) & ~1023u;
    static_assert(!HALO || STAGES + STAGES_B <= 16, "halo config");
    // (BN % 8 == 0: each weight slice of a grouped box starts on a swizzle-pattern boundary)
    static_assert(!GRP || (HALO && BN % 8 == 0), "grouped stages run on the halo path");
    static_assert(!S2H || (!HALO && !GRP && MT == 1 && !F8 && STAGES < 16 && BN % 8 == 0 &&
                           (ROW_BYTES == 32 || ROW_BYTES == 64)),
                  "stride-2 pair halo: one 16/32-channel block, pair rows of 64/128 bytes");
    static_assert(!KXF || (GRP == 2 && MT == 1 && !TS && KXF <= 2), "folded column taps: resident grouped stages");
    // S2H / GRP == 2: the resident weight slices (KXF: 3 folded slices per channel block)
    constexpr uint32_t BR_STRIDE = ((KXF ? 3 * KXF : 9) * B_BYTES + 1023) & ~1023u;
    // grouped stage: A box + the row tap's 3 weight slices, loaded as ONE box of 3 taps
    // (slice kx at kx * B_BYTES; every B_BYTES here is a multiple of the swizzle atom)
    constexpr uint32_t G_STRIDE = GRP == 2 ? A_STRIDE : A_STRIDE + ((3 * B_BYTES + 1023) & ~1023u);
    constexpr int ACCB = AccCfg<BN, MT>::ACCB;
    constexpr uint32_t TMEM_COLS = AccCfg<BN, MT>::TMEM_COLS;
    constexpr uint32_t IDESC = F8 ? ptx::make_idesc(128, BN, 0, 0) : ptx::make_idesc(128, BN, 1, 1);

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * (GRP ? G_STRIDE : A_STRIDE);
    // epilogue staging: per epilogue warp two buffers of 32 rows x STG_ROW bytes
    constexpr uint32_t STG_ROW = BN * 2 < 128 ? BN * 2 : 128, STG_BYTES = 32 * STG_ROW;
    // staging buffers per epilogue warp: two (a chunk is staged while the previous one's
    // store reads), one for the two-row-block tiles, whose operand stages are larger
    constexpr int NSB = MT == 2 ? 1 : 2;
    uint8_t *stg = sB + (GRP == 1 ? 0u : (S2H || GRP == 2 ? BR_STRIDE : (HALO ? STAGES_B : STAGES) * B_STRIDE));
    // KXF: per epilogue warp the Eq. 2 outputs of its 30 pixels, two fine rows of 60 x 5
    // floats, staged so that the warp stores whole rows
    constexpr uint32_t KST_BYTES = KXF ? 4 * 2 * 300 * 4 : 0;
    // the output conv (N = 16, resident weights): a ring of NIB tiles of I_blend (128 pixels x
    // 3 floats), bulk-copied by the producer with the tile's A boxes, so that the epilogue
    // reads it from shared memory instead of waiting for global loads on every tile;
    // barriers full / empty[STAGES + 1 + slot]
    constexpr int NIB = BN == 16 && GRP == 2 && !TS && !KXF ? 4 : 0;
    constexpr uint32_t IB_SLOT = 128 * 3 * 4;
    static_assert(STAGES + 1 + NIB <= 16, "barrier slots");
    float *const ibs = (float *)(stg + (TS ? 4 * NSB * STG_BYTES : KST_BYTES));
    Bars *bars = (Bars *)(stg + (TS ? 4 * NSB * STG_BYTES : KST_BYTES) + NIB * IB_SLOT);
    // the layer's biases and dequantisation scales (1 without) for output channels co < BN,
    // staged once per CTA for the TMA-store epilogue of the one- and two-CTA kernels
    // (measured: 2-3 % faster there; the four-CTA kernels, capped at 80 registers, spilled
    // with it, and the per-thread-store epilogue of the all-phase d3 got slower)
    constexpr bool SB = TS && CTAS <= 2;
    float *const sbias_p = (float *)(bars + 1);
    volatile int *abort = &bars->abort;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        // halo: full/empty[0, STAGES) = A ring, [STAGES, STAGES + STAGES_B) = B ring
        // S2H: full[STAGES] = the resident weights
        for (int s = 0; s < (HALO && !GRP ? STAGES + STAGES_B : STAGES + (S2H || GRP == 2 ? 1 : 0)); ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_full[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_empty[a]), 128);
        }
        for (int i = 0; i < NIB; ++i) {
            ptx::mbar_init(ptx::smem_u32(&bars->full[STAGES + 1 + i]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->empty[STAGES + 1 + i]), 4); // one arrive per epilogue warp
        }
        ptx::mbar_init(ptx::smem_u32(&bars->drain), 1);
        ptx::mbar_init(ptx::smem_u32(&bars->never), 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
        ptx::fence_proxy_async_smem();
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        if (TS && p.tma_store) ptx::prefetch_tmap(&tmC);
    }
    for (int i = threadIdx.x; SB && i < BN; i += kThreads) {
        sbias_p[i] = i < p.co ? __ldg(p.bias + i) : 0.f;
        sbias_p[BN + i] = i < p.co && p.acc_scale ? __ldg(p.acc_scale + i) : 1.f;
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(&bars->tmem_base), TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    const int kblocks = p.taps * p.nck;
    const int ip = p.ipad, pp = p.ipad >> 1; // circular mode: A coordinates in the wrapped-border input
    // I_blend ring live: the output conv's fused residual output on one-row 128-pixel tiles
    // (bulk copies: 16-byte aligned rows, so the image base 16-byte aligned and its width a multiple of 4)
    const bool ibr = NIB && p.epi.mode == EPI_OUTPUT && p.th_log == 0 && p.tw_log == 7 &&
                     ((uintptr_t)p.epi.ib & 15) == 0 && (p.out_w & 3) == 0;
    // images actually run: a launch captured for a size bucket reads the call's count
    const int n_img = p.n_dev ? min(__ldg(p.n_dev), p.n_img) : p.n_img;
    const int num_tiles = p.n_dev ? n_img * p.tiles_y * p.tiles_x * (p.mode == MODE_T ? 4 : 1) : p.num_tiles;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0 && S2H) {
            const uint32_t fw = ptx::smem_u32(&bars->full[STAGES]);
            ptx::mbar_arrive_expect_tx(fw, 9 * B_BYTES);
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) // taps 3ky .. 3ky + 2 per box
                ptx::tma_load_3d(ptx::smem_u32(sB) + ky * 3 * B_BYTES, &tmB, fw, 0, 0, ky * 3);
            int s = 0;
            uint32_t ph_bit = 0;
            long long issued = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < num_tiles && !*abort && !stop; t += gridDim.x) {
                int ph, n, y0, x0;
                tile_coords(p, t, ph, n, y0, x0);
                for (int ky = 0; ky < 3; ++ky) {
                    if (!wait_bar(ptx::smem_u32(&bars->empty[s]), ph_bit ^ 1, abort, p.err, 1)) { stop = true; break; }
                    const uint32_t fs = ptx::smem_u32(&bars->full[s]);
                    ptx::mbar_arrive_expect_tx(fs, A_BYTES);
                    // input row 2 y0 + ky - 1 = (row pair, parity) (y0 - 1, 1), (y0, 0), (y0, 1);
                    // pairs x0 - 1 .. x0 + 127 (both pixels of each)
                    ptx::tma_load_5d(ptx::smem_u32(sA + s * A_STRIDE), &tmA, fs, 0, x0 - 1 + pp, ky != 1 ? 1 : 0,
                                     y0 - (ky == 0 ? 1 : 0) + pp, n);
                    ++issued;
                    if (++s == STAGES) { s = 0; ph_bit ^= 1; }
                }
            }
            if (*abort || stop) {
                // let every copy still in flight land before the CTA exits
                long long t0 = clock64();
                while (!ptx::mbar_try_wait(fw, 0) && clock64() - t0 < kWaitCycles) {}
                for (int i = 0; i < STAGES && i < issued; ++i) {
                    long long k = issued - 1 - i;
                    t0 = clock64();
                    while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->full[k % STAGES]), (uint32_t)((k / STAGES) & 1)) &&
                           clock64() - t0 < kWaitCycles) {}
                }
            }
        } else if (lane == 0 && GRP) {
            const uint32_t fw = ptx::smem_u32(&bars->full[STAGES]); // GRP == 2: resident weights
            if (KXF) {
                // channel block c: the folded slices of row taps 0..2 in one box
                ptx::mbar_arrive_expect_tx(fw, 3 * KXF * B_BYTES);
#pragma unroll
                for (int c = 0; c < KXF; ++c)
                    ptx::tma_load_3d(ptx::smem_u32(sB) + c * 3 * B_BYTES, &tmB, fw, c * CK, 0, 0);
            } else if (GRP == 2) {
                ptx::mbar_arrive_expect_tx(fw, 9 * B_BYTES);
#pragma unroll
                for (int ky = 0; ky < 3; ++ky) // taps 3ky .. 3ky + 2 per box
                    ptx::tma_load_3d(ptx::smem_u32(sB) + ky * 3 * B_BYTES, &tmB, fw, 0, 0, ky * 3);
            }
            int s = 0;
            uint32_t ph_bit = 0;
            long long issued = 0, ib_issued = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < num_tiles && !*abort && !stop; t += gridDim.x) {
                int ph, n, y0, x0;
                tile_coords(p, t, ph, n, y0, x0);
                if (ibr) {
                    // this tile's I_blend row segment (the padded grid is a multiple of 16 wide)
                    const int slot = (int)(ib_issued % NIB);
                    if (!wait_bar(ptx::smem_u32(&bars->empty[STAGES + 1 + slot]),
                                  (uint32_t)((ib_issued / NIB) & 1) ^ 1u, abort, p.err, 1)) { stop = true; break; }
                    const uint32_t bytes = (uint32_t)min(128, p.gw - x0) * 12u;
                    const uint32_t fi = ptx::smem_u32(&bars->full[STAGES + 1 + slot]);
                    ptx::mbar_arrive_expect_tx(fi, bytes);
                    ptx::bulk_load(ptx::smem_u32(ibs + slot * 384),
                                   p.epi.ib + (((size_t)n * p.out_h + y0) * p.out_w + x0) * 3, bytes, fi);
                    ++ib_issued;
                }
                for (int ky = 0; ky < 3 && !stop; ++ky)
                    for (int c = 0; c < p.nck; ++c) {
                        if (!wait_bar(ptx::smem_u32(&bars->empty[s]), ph_bit ^ 1, abort, p.err, 1)) { stop = true; break; }
                        const uint32_t fs = ptx::smem_u32(&bars->full[s]);
                        ptx::mbar_arrive_expect_tx(fs, GRP == 2 ? A_BYTES : A_BYTES + 3 * B_BYTES);
                        const uint32_t base = ptx::smem_u32(sA + s * G_STRIDE);
                        if (KXF) { // epilogue warp q's rows: input pixels x0 - 1 + 30 q .. + 31
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                ptx::tma_load_4d(base + q * 32 * ROW_BYTES, &tmA, fs, p.in_coff + c * CK,
                                                 x0 - 1 + 30 * q + ip, y0 + ky - 1 + ip, n);
                        } else {
                            ptx::tma_load_4d(base, &tmA, fs, p.in_coff + c * CK, x0 - 1 + ip, y0 + ky - 1 + ip, n);
                        }
                        if (GRP == 1)
                            ptx::tma_load_3d(base + A_STRIDE, &tmB, fs, c * CK, 0, ky * 3); // taps ky*3 .. ky*3+2
                        ++issued;
                        if (++s == STAGES) { s = 0; ph_bit ^= 1; }
                    }
            }
            if (*abort || stop) {
                // let every copy still in flight land before the CTA exits
                if (GRP == 2) {
                    long long t0 = clock64();
                    while (!ptx::mbar_try_wait(fw, 0) && clock64() - t0 < kWaitCycles) {}
                }
                for (int i = 0; i < NIB && i < ib_issued; ++i) {
                    const long long k = ib_issued - 1 - i;
                    long long t0 = clock64();
                    while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->full[STAGES + 1 + k % NIB]),
                                               (uint32_t)((k / NIB) & 1)) &&
                           clock64() - t0 < kWaitCycles) {}
                }
                for (int i = 0; i < STAGES && i < issued; ++i) {
                    long long k = issued - 1 - i;
                    long long t0 = clock64();
                    while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->full[k % STAGES]), (uint32_t)((k / STAGES) & 1)) &&
                           clock64() - t0 < kWaitCycles) {}
                }
            }
        } else if (lane == 0 && HALO) {
            int sa = 0, sb = 0;
            uint32_t pa = 0, pb = 0;
            long long issued_a = 0, issued_b = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < num_tiles && !*abort && !stop; t += gridDim.x) {
                int ph, n, y0, x0;
                tile_coords(p, t, ph, n, y0, x0);
                // boxes in K order (ky, channel block)
                const int ngroups = 3 * p.nck;
                for (int grp = 0; grp < ngroups && !stop; ++grp) {
                        const int ky = grp >> p.nck_log, c = grp & (p.nck - 1);
                        if (!wait_bar(ptx::smem_u32(&bars->empty[sa]), pa ^ 1, abort, p.err, 1)) { stop = true; break; }
                        uint32_t fa = ptx::smem_u32(&bars->full[sa]);
                        ptx::mbar_arrive_expect_tx(fa, A_BYTES);
                        ptx::tma_load_4d(ptx::smem_u32(sA + sa * A_STRIDE), &tmA, fa, p.in_coff + c * CK, x0 - 1 + ip,
                                         y0 + ky - 1 + ip, n);
                        ++issued_a;
                        if (++sa == STAGES) { sa = 0; pa ^= 1; }
                        for (int kx = 0; kx < NB; ++kx) {
                            const int slot = STAGES + sb;
                            if (!wait_bar(ptx::smem_u32(&bars->empty[slot]), pb ^ 1, abort, p.err, 1)) { stop = true; break; }
                            uint32_t fbb = ptx::smem_u32(&bars->full[slot]);
                            ptx::mbar_arrive_expect_tx(fbb, B_BYTES);
                            ptx::tma_load_3d(ptx::smem_u32(sB + sb * B_STRIDE), &tmB, fbb, c * CK, 0, ky * 3 + kx);
                            ++issued_b;
                            if (++sb == STAGES_B) { sb = 0; pb ^= 1; }
                        }
                }
            }
            if (*abort || stop) {
                // let every copy still in flight land before the CTA exits
                for (int s = 0; s < STAGES && s < issued_a; ++s) {
                    long long k = issued_a - 1 - s;
                    long long t0 = clock64();
                    while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->full[k % STAGES]), (uint32_t)((k / STAGES) & 1)) &&
                           clock64() - t0 < kWaitCycles) {}
                }
                for (int s = 0; s < STAGES_B && s < issued_b; ++s) {
                    long long k = issued_b - 1 - s;
                    long long t0 = clock64();
                    while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->full[STAGES + k % STAGES_B]),
                                               (uint32_t)((k / STAGES_B) & 1)) &&
                           clock64() - t0 < kWaitCycles) {}
                }
            }
        } else if (lane == 0) {
            int stage = 0;
            uint32_t phase_bit = 0;
            long long issued = 0;
            for (int t = blockIdx.x; t < num_tiles && !*abort; t += gridDim.x) {
                int ph, n, y0, x0;
                tile_coords(p, t, ph, n, y0, x0);
                for (int kb = 0; kb < kblocks; ++kb) {
                    if (!wait_bar(ptx::smem_u32(&bars->empty[stage]), phase_bit ^ 1, abort, p.err, 1)) break;
                    int tap = kb >> p.nck_log, c0 = (kb & (p.nck - 1)) * CK;
                    uint32_t fb = ptx::smem_u32(&bars->full[stage]);
                    ptx::mbar_arrive_expect_tx(fb, A_BYTES + B_BYTES);
                    uint32_t da = ptx::smem_u32(sA + stage * A_STRIDE), db = ptx::smem_u32(sB + stage * B_STRIDE);
                    if (p.mode == MODE_S1 || p.mode == MODE_T3) {
                        // K order (ky, channel block, kx): the same as the halo path
                        const int ky = (kb >> p.nck_log) / 3, r = kb - ((ky * 3) << p.nck_log), kx = r % 3;
                        c0 = (r / 3) * CK;
                        tap = ky * 3 + kx;
                        ptx::tma_load_4d(da, &tmA, fb, p.in_coff + c0, x0 + kx - 1 + ip, y0 + ky - 1 + ip, n);
                        ptx::tma_load_3d(db, &tmB, fb, c0, 0, tap);
                    } else if (p.mode == MODE_S2) {
                        int ky = tap / 3, kx = tap - 3 * (tap / 3);
                        int half = kx == 1 ? 0 : 1, rpar = ky == 1 ? 0 : 1;
                        ptx::tma_load_5d(da, &tmA, fb, half * p.in_cs + p.in_coff + c0, x0 - (kx == 0 ? 1 : 0) + pp,
                                         rpar, y0 - (ky == 0 ? 1 : 0) + pp, n);
                        ptx::tma_load_3d(db, &tmB, fb, c0, 0,
                                         tap + (p.wcopies > 1 ? 9 * (int)(blockIdx.x % (unsigned)p.wcopies) : 0));
                    } else {
                        // K order (channel block, tap)
                        tap = kb & 3;
                        c0 = (kb >> 2) * CK;
                        int py = ph >> 1, px = ph & 1, ty = tap >> 1, tx = tap & 1;
                        int dy = py == 0 ? -ty : 1 - ty, dx = px == 0 ? -tx : 1 - tx;
                        ptx::tma_load_4d(da, &tmA, fb, p.in_coff + c0, x0 + dx + ip, y0 + dy + ip, n);
                        ptx::tma_load_3d(db, &tmB, fb, c0, 0, ph * 4 + tap);
                    }
                    ++issued;
                    if (++stage == STAGES) { stage = 0; phase_bit ^= 1; }
                }
            }
            if (*abort) {
                // let every copy still in flight land before the CTA exits
                for (int s = 0; s < STAGES && issued > 0; ++s) {
                    long long k = issued - 1 - s;
                    if (k < 0) break;
                    int st = (int)(k % STAGES);
                    uint32_t par = (uint32_t)((k / STAGES) & 1);
                    long long t0 = clock64();
                    while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->full[st]), par) && clock64() - t0 < kWaitCycles) {}
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        // fault injection: a wait that runs out (nothing arrives on `never`) records
        // code 6 and raises the abort flag before any MMA is issued; the producer then
        // stops and lets its copies land, the epilogue warps leave, TMEM is freed
        if (lane == 0 && p.stall_cycles > 0)
            wait_bar(ptx::smem_u32(&bars->never), 0, abort, p.err, 6, p.stall_cycles);
        if (lane == 0 && S2H) {
            int s = 0;
            uint32_t ph_bit = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool issued_any = false;
            bool ok = wait_bar(ptx::smem_u32(&bars->full[STAGES]), 0, abort, p.err, 3); // resident weights
            ptx::tc_fence_after();
            const uint32_t bw = ptx::smem_u32(sB);
            for (int t = blockIdx.x; ok && t < num_tiles && !*abort; t += gridDim.x) {
                if (!wait_bar(ptx::smem_u32(&bars->tmem_empty[acc]), acc_phase ^ 1, abort, p.err, 2)) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem + acc * BN;
                for (int ky = 0; ky < 3; ++ky) {
                    if (!wait_bar(ptx::smem_u32(&bars->full[s]), ph_bit, abort, p.err, 3)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const uint32_t a0 = ptx::smem_u32(sA + s * A_STRIDE);
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
                        const uint32_t b0 = bw + (ky * 3 + kx) * B_BYTES;
                        // output pixel j reads input pixel 2j + kx - 1: pair j + (kx == 0 ? 0 : 1) of the
                        // box, odd pixel (second ROW_BYTES of the pair row) unless kx == 1
                        const uint32_t ak = a0 + (kx == 0 ? 0u : 2u * ROW_BYTES) + (kx == 1 ? 0u : (uint32_t)ROW_BYTES);
#pragma unroll
                        for (int k = 0; k < ROW_BYTES / 32; ++k) {
                            const uint64_t bd = ptx::smem_desc(b0 + k * 32, ROW_BYTES);
                            const uint64_t ad = ptx::smem_desc(ak + k * 32, 2 * ROW_BYTES);
                            ptx::mma_bf16(d, ad, bd, IDESC, (ky | kx | k) != 0);
                        }
                    }
                    issued_any = true;
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[s]));
                    if (++s == STAGES) { s = 0; ph_bit ^= 1; }
                }
                if (!ok) break;
                ptx::mma_commit(ptx::smem_u32(&bars->tmem_full[acc]));
                if (++acc == ACCB) { acc = 0; acc_phase ^= 1; }
            }
            if (*abort && issued_any) {
                ptx::mma_commit(ptx::smem_u32(&bars->drain));
                long long t0 = clock64();
                while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->drain), 0) && clock64() - t0 < kWaitCycles) {}
            }
        } else if (lane == 0 && GRP) {
            int s = 0;
            uint32_t ph_bit = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool issued_any = false;
            // GRP == 2: the resident weight slices (one channel block: group g = row tap ky)
            const bool wok = GRP != 2 || wait_bar(ptx::smem_u32(&bars->full[STAGES]), 0, abort, p.err, 3);
            ptx::tc_fence_after();
            for (int t = blockIdx.x; wok && t < num_tiles && !*abort; t += gridDim.x) {
                if (!wait_bar(ptx::smem_u32(&bars->tmem_empty[acc]), acc_phase ^ 1, abort, p.err, 2)) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem + acc * (MT * BN);
                bool ok = true;
                uint32_t accumulate = 0;
                for (int g = 0; g < 3 * p.nck; ++g) { // (ky, channel block) in K order
                    if (!wait_bar(ptx::smem_u32(&bars->full[s]), ph_bit, abort, p.err, 3)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const uint32_t a0 = ptx::smem_u32(sA + s * G_STRIDE);
                    if (KXF) {
                        // the folded slice of (row tap ky, channel block c): all three column taps
                        const int ky = g / KXF, c = g - ky * KXF;
                        const uint32_t b0 = ptx::smem_u32(sB) + (c * 3 + ky) * B_BYTES;
#pragma unroll
                        for (int k = 0; k < ROW_BYTES / 32; ++k) {
                            const uint64_t bd = ptx::smem_desc(b0 + k * 32, ROW_BYTES);
                            const uint64_t ad = ptx::smem_desc(a0 + k * 32, ROW_BYTES);
                            if (F8) ptx::mma_f8(d, ad, bd, IDESC, accumulate | (uint32_t)k);
                            else ptx::mma_bf16(d, ad, bd, IDESC, accumulate | (uint32_t)k);
                        }
                        accumulate = 1;
                    }
#pragma unroll
                    for (int kx = 0; kx < (KXF ? 0 : 3); ++kx) {
                        const uint32_t b0 = GRP == 2 ? ptx::smem_u32(sB) + (g * 3 + kx) * B_BYTES
                                                     : a0 + A_STRIDE + kx * B_BYTES;
#pragma unroll
                        for (int k = 0; k < ROW_BYTES / 32; ++k) {
                            uint64_t bd = ptx::smem_desc(b0 + k * 32, ROW_BYTES);
#pragma unroll
                            for (int m = 0; m < MT; ++m) {
                                uint64_t ad = ptx::smem_desc(a0 + (m * 130 + kx) * ROW_BYTES + k * 32, ROW_BYTES);
                                if (F8) ptx::mma_f8(d + m * BN, ad, bd, IDESC, accumulate | (uint32_t)k);
                                else ptx::mma_bf16(d + m * BN, ad, bd, IDESC, accumulate | (uint32_t)k);
                            }
                        }
                        accumulate = 1;
                    }
                    issued_any = true;
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[s]));
                    if (++s == STAGES) { s = 0; ph_bit ^= 1; }
                }
                if (!ok) break;
                ptx::mma_commit(ptx::smem_u32(&bars->tmem_full[acc]));
                if (++acc == ACCB) { acc = 0; acc_phase ^= 1; }
            }
            if (*abort && issued_any) {
                ptx::mma_commit(ptx::smem_u32(&bars->drain));
                long long t0 = clock64();
                while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->drain), 0) && clock64() - t0 < kWaitCycles) {}
            }
        } else if (lane == 0 && HALO) {
            int sa = 0, sb = 0;
            uint32_t pa = 0, pb = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool issued_any = false;
            for (int t = blockIdx.x; t < num_tiles && !*abort; t += gridDim.x) {
                if (!wait_bar(ptx::smem_u32(&bars->tmem_empty[acc]), acc_phase ^ 1, abort, p.err, 2)) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem + acc * (MT * BN);
                bool ok = true;
                uint32_t accumulate = 0;
                const int ngroups = 3 * p.nck;
                for (int grp = 0; grp < ngroups && ok; ++grp) {
                        if (!wait_bar(ptx::smem_u32(&bars->full[sa]), pa, abort, p.err, 3)) { ok = false; break; }
                        ptx::tc_fence_after();
                        const uint32_t a0 = ptx::smem_u32(sA + sa * A_STRIDE);
                        for (int kx = 0; kx < NB; ++kx) {
                            if (!wait_bar(ptx::smem_u32(&bars->full[STAGES + sb]), pb, abort, p.err, 3)) { ok = false; break; }
                            ptx::tc_fence_after();
                            const uint32_t b0 = ptx::smem_u32(sB + sb * B_STRIDE);
                            // column tap kx: the 128 output pixels read box rows kx .. kx + 127.
                            // The swizzle follows address bits, so a start 1-2 rows into
                            // the swizzle atom needs no base-offset field.
#pragma unroll
                            for (int k = 0; k < ROW_BYTES / 32; ++k) {
                                uint64_t bd = ptx::smem_desc(b0 + k * 32, ROW_BYTES);
#pragma unroll
                                for (int m = 0; m < MT; ++m) {
                                    const int row0 = m * HROW + kx; // row block m, column tap kx
                                    uint64_t ad = ptx::smem_desc(a0 + row0 * ROW_BYTES + k * 32, ROW_BYTES);
                                    if (F8) ptx::mma_f8(d + m * BN, ad, bd, IDESC, accumulate | (uint32_t)k);
                                    else ptx::mma_bf16(d + m * BN, ad, bd, IDESC, accumulate | (uint32_t)k);
                                }
                            }
                            accumulate = 1;
                            issued_any = true;
                            ptx::mma_commit(ptx::smem_u32(&bars->empty[STAGES + sb]));
                            if (++sb == STAGES_B) { sb = 0; pb ^= 1; }
                        }
                        if (!ok) break;
                        ptx::mma_commit(ptx::smem_u32(&bars->empty[sa]));
                        if (++sa == STAGES) { sa = 0; pa ^= 1; }
                }
                if (!ok) break;
                ptx::mma_commit(ptx::smem_u32(&bars->tmem_full[acc]));
                if (++acc == ACCB) { acc = 0; acc_phase ^= 1; }
            }
            if (*abort && issued_any) {
                ptx::mma_commit(ptx::smem_u32(&bars->drain));
                long long t0 = clock64();
                while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->drain), 0) && clock64() - t0 < kWaitCycles) {}
            }
        } else if (lane == 0) {
            int stage = 0;
            uint32_t phase_bit = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool issued_any = false;
            for (int t = blockIdx.x; t < num_tiles && !*abort; t += gridDim.x) {
                if (!wait_bar(ptx::smem_u32(&bars->tmem_empty[acc]), acc_phase ^ 1, abort, p.err, 2)) break;
                ptx::tc_fence_after();
                uint32_t d = tmem + acc * (MT * BN);
                bool ok = true;
                for (int kb = 0; kb < kblocks; ++kb) {
                    if (!wait_bar(ptx::smem_u32(&bars->full[stage]), phase_bit, abort, p.err, 3)) { ok = false; break; }
                    ptx::tc_fence_after();
                    uint32_t a0 = ptx::smem_u32(sA + stage * A_STRIDE), b0 = ptx::smem_u32(sB + stage * B_STRIDE);
#pragma unroll
                    for (int k = 0; k < ROW_BYTES / 32; ++k) {
                        uint64_t bd = ptx::smem_desc(b0 + k * 32, ROW_BYTES);
#pragma unroll
                        for (int m = 0; m < MT; ++m) {
                            uint64_t ad = ptx::smem_desc(a0 + m * 128 * ROW_BYTES + k * 32, ROW_BYTES);
                            if (F8) ptx::mma_f8(d + m * BN, ad, bd, IDESC, (kb | k) != 0);
                            else ptx::mma_bf16(d + m * BN, ad, bd, IDESC, (kb | k) != 0);
                        }
                    }
                    issued_any = true;
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[stage]));
                    if (++stage == STAGES) { stage = 0; phase_bit ^= 1; }
                }
                if (!ok) break;
                ptx::mma_commit(ptx::smem_u32(&bars->tmem_full[acc]));
                if (++acc == ACCB) { acc = 0; acc_phase ^= 1; }
            }
            if (*abort && issued_any) {
                // wait (bounded) for the MMAs already issued before TMEM is freed
                ptx::mma_commit(ptx::smem_u32(&bars->drain));
                long long t0 = clock64();
                while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->drain), 0) && clock64() - t0 < kWaitCycles) {}
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const uint32_t sbias = ptx::smem_u32(bars + 1), sscale = sbias + 4 * BN; // staged biases, scales
        const int q = warp & 3;           // TMEM lane quarter this warp may access
        const int row = q * 32 + lane;    // tile row = accumulator lane
        int acc = 0;
        uint32_t acc_phase = 0;
        uint32_t scnt = 0;                // staged chunks of this warp (buffer = scnt % NSB)
        const uint32_t stg_warp = ptx::smem_u32(stg) + (uint32_t)(q * NSB * STG_BYTES);
        const int tw = 1 << p.tw_log;
        const int dy = row >> p.tw_log, dx = row & (tw - 1);
        float *const kst = KXF ? (float *)stg + q * 600 : nullptr; // folded taps: Eq. 2 staging
        float r_bias[5], r_sc[5]; // folded taps, Eq. 2: bias and dequantisation scale of F, M
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            r_bias[k] = KXF && p.epi.mode == EPI_RESID ? __ldg(p.bias + k) : 0.f;
            r_sc[k] = KXF && p.epi.mode == EPI_RESID && p.acc_scale ? __ldg(p.acc_scale + k) : 1.f;
        }
        // fused network output (N = 16 tiles): the cropped output buffer and the 3 biases
        float *const out_final = BN == 16 && p.epi.mode == EPI_OUTPUT ? *p.epi.final_out_ref : nullptr;
        float obias[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) obias[j] = BN == 16 && p.epi.mode == EPI_OUTPUT ? __ldg(p.bias + j) : 0.f;
        long long tk = -1; // this CTA's tile count (I_blend ring slot / phase)
        for (int t = blockIdx.x; t < num_tiles && !*abort; t += gridDim.x) {
            ++tk;
            int ph, n, y0, x0;
            tile_coords(p, t, ph, n, y0, x0);
            int gy = y0 + dy, gx = x0 + dx;
            bool valid = gy < p.gh && gx < p.gw;
            uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + acc * (MT * BN);
            if (KXF) {
                // folded column taps: this lane's row is input pixel x0 - 1 + 30 q + lane; lanes
                // 1..30 sum tap 0 of the lane before, tap 1 of their own and tap 2 of the next
                const int G = p.mode == MODE_T3 ? 4 * p.co : p.co; // accumulator columns per tap
                const int kgx = x0 - 1 + 30 * q + lane;
                const bool kvalid = lane >= 1 && lane <= 30 && kgx < p.gw && y0 < p.gh;
                const bool resid = p.epi.mode == EPI_RESID;
                float nb[3][3][5];
                if (resid) resid_nb(p, n, y0, kgx, lane, true, nb);
                if (!wait_bar(ptx::smem_u32(&bars->tmem_full[acc]), acc_phase, abort, p.err, 4)) break;
                ptx::tc_fence_after();
                // (j0 unrolled over the BN / 3 columns a tap can have: static register indices)
#pragma unroll
                for (int j0 = 0; j0 < BN / 3; j0 += 16) {
                    if (j0 >= G) break;
                    // 4-column loads: G is a multiple of 4, so every load starts on a
                    // multiple of its own width
                    uint32_t ra[16], rb[16], rc[16];
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < 16; u += 4) {
                        ra[u] = ra[u + 1] = ra[u + 2] = ra[u + 3] = 0u;
                        rb[u] = rb[u + 1] = rb[u + 2] = rb[u + 3] = 0u;
                        rc[u] = rc[u + 1] = rc[u + 2] = rc[u + 3] = 0u;
                        if (j0 + u < G) {
                            ptx::tmem_ld4(tbase + j0 + u, ra + u);
                            ptx::tmem_ld4(tbase + G + j0 + u, rb + u);
                            ptx::tmem_ld4(tbase + 2 * G + j0 + u, rc + u);
                        }
                    }
                    ptx::tmem_ld_wait();
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float left = __shfl_up_sync(0xffffffffu, __uint_as_float(ra[j]), 1);
                        const float right = __shfl_down_sync(0xffffffffu, __uint_as_float(rc[j]), 1);
                        v[j] = left + __uint_as_float(rb[j]) + right;
                    }
                    if (!kvalid) continue;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = j0 + j;
                        if (col >= G) break;
                        if (resid) {
                            // fine pixel (2 y0 + py, 2 kgx + px), channel co -> staging row py
                            const int pj = col / 5, co = col % 5;
                            kst[(pj >> 1) * 300 + (2 * (lane - 1) + (pj & 1)) * 5 + co] =
                                resid_value(nb, col, v[j], r_sc[co], r_bias[co]);
                        } else if (p.mode == MODE_T3) {
                            const int pj = (int)p.fdco.div((uint32_t)col), co = col - pj * p.co;
                            epi_elem<SB>(p, sbias, sscale, n, 2 * y0 + (pj >> 1), 2 * kgx + (pj & 1), co, v[j]);
                        } else {
                            epi_elem<SB>(p, sbias, sscale, n, y0, kgx, col, v[j]);
                        }
                    }
                }
                if (resid) {
                    // the warp's two fine rows, 2 x 30 pixels x 5 channels each, as whole
                    // 128-byte lines (F, M are dense: C = 5, no channel offset)
                    __syncwarp();
                    const int gx0 = x0 + 30 * q; // pixel of lane 1
#pragma unroll
                    for (int py = 0; py < 2; ++py) {
                        float *dst = (float *)p.out + (((size_t)n * p.out_h + 2 * y0 + py) * p.out_w + 2 * gx0) * 5;
                        for (int i = lane; i < 300; i += 32)
                            if (2 * gx0 + i / 5 < p.out_w) dst[i] = kst[py * 300 + i];
                    }
                    __syncwarp();
                }
            } else if (MT == 1 && BN == 32 && p.epi.mode == EPI_RESID) {
                // Eq. 2 update of a 4-phase transposed conv with 5 outputs (the VIB
                // t1 layer): this pixel q of the half grid owns the 4 fine pixels
                // (2q + phase); their x2 upsampling reads the 3x3 neighbourhood of q
                // in the previous stage's F, M, fetched before the accumulator is ready.
                float nb[3][3][5];
                resid_nb(p, n, gy, gx, lane, p.tw_log >= 5, nb);
                if (!wait_bar(ptx::smem_u32(&bars->tmem_full[acc]), acc_phase, abort, p.err, 4)) break;
                ptx::tc_fence_after();
#pragma unroll
                for (int c = 0; c < 32; c += 16) {
                    uint32_t r[16];
                    __syncwarp();
                    ptx::tmem_ld16(tbase + c, r);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c + j < 20 && valid) resid_store<SB>(p, sbias, sscale, nb, n, gy, gx, c + j, __uint_as_float(r[j]));
                }
            } else {
            if (!wait_bar(ptx::smem_u32(&bars->tmem_full[acc]), acc_phase, abort, p.err, 4)) break;
            ptx::tc_fence_after();
            const int ncols = p.mode == MODE_T3 ? 4 * p.co : p.co; // columns that hold outputs
            const float *ibt = nullptr; // this tile's I_blend in the ring
            if (ibr) {
                if (!wait_bar(ptx::smem_u32(&bars->full[STAGES + 1 + tk % NIB]), (uint32_t)((tk / NIB) & 1), abort, p.err,
                              4)) break;
                ibt = ibs + (tk % NIB) * 384;
            }
            if (TS && p.tma_store) {
            // Each warp writes its 32 rows chunk by chunk (STG_ROW bytes of channels per
            // row) into a swizzled staging buffer and one lane stores the box with TMA
            // (rows outside the output are clipped by the tensor map).  bf16 or E4M3.
            // A chunk is min(BN, 64) (bf16) or min(BN, 128) (E4M3) columns; for the 4-phase
            // transposed conv (MODE_T3) it is one phase's C_out columns, stored through
            // the pixel-pair map at that phase's row and column parity.
            const int oes = p.out_fp8 ? 1 : 2;
            // (staged stores of the 4-phase convT exist for N = 128 only; other tiles compile without them)
            const bool t3 = BN == 128 && p.mode == MODE_T3;
            const int chn = t3 ? p.co : (BN * oes < 128 ? BN : 128 / oes), chb = chn * oes;
            const int ncol = t3 ? 4 * p.co : BN;
            constexpr int LDB = BN >= 64 ? (CTAS <= 2 ? 4 : 2) : (BN == 32 ? 2 : 1); // divides chn / 16
            const uint32_t swm = chb == 128 ? 7u : (chb == 64 ? 3u : 1u);
#pragma unroll 1
            for (int m = 0; m < MT; ++m) {
                const int rb = m * 128 + q * 32, rm = rb + lane;
                const int gy = y0 + (rm >> p.tw_log), gx = x0 + (rm & (tw - 1));
                const bool valid = gy < p.gh && gx < p.gw;
                const int by = y0 + (rb >> p.tw_log), bx = x0 + (rb & (tw - 1));
                const uint32_t tb = tbase + m * BN;
#pragma unroll 1
                for (int k0 = 0; k0 < ncol; k0 += chn) {
                    // the buffer staged two chunks ago must have been read by its store
                    // the buffer's previous store (NSB chunks ago) must have been read
                    if (lane == 0) ptx::bulk_wait_read<NSB - 1>();
                    __syncwarp();
                    const uint32_t sbuf = stg_warp + (scnt % NSB) * STG_BYTES;
                    // bias, ReLU, conversion and swizzled staging of columns c .. c + 15
                    // (output channels cc .. cc + 15)
                    auto stage16 = [&](int c, int cc, const uint32_t(&r)[16]) {
                        float v[16], bq[16], sq[16];
                        bias_scale16<SB, F8>(p, sbias, sscale, cc, bq, sq);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float a = __uint_as_float(r[j]) * sq[j] + bq[j];
                            v[j] = p.relu ? fmaxf(a, 0.f) : a;
                        }
                        if (p.amax && valid) { // calibration only
                            float vmax = 0.f;
#pragma unroll
                            for (int j = 0; j < 16; ++j) vmax = fmaxf(vmax, fabsf(v[j]));
                            atomicMax(reinterpret_cast<int *>(p.amax), __float_as_int(vmax));
                        }
                        const uint32_t a0 = sbuf + lane * chb + (c - k0) * oes;
                        if (p.out_fp8) {
                            ptx::st_shared_v4(a0 ^ (((a0 >> 7) & swm) << 4), e4m3x16(v, p.out_q));
                        } else {
                            __nv_bfloat162 h[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            uint4 w0, w1;
                            memcpy(&w0, &h[0], 16);
                            memcpy(&w1, &h[4], 16);
                            const uint32_t a1 = a0 + 16;
                            ptx::st_shared_v4(a0 ^ (((a0 >> 7) & swm) << 4), w0);
                            ptx::st_shared_v4(a1 ^ (((a1 >> 7) & swm) << 4), w1);
                        }
                    };
                    if (t3) {
                        // one phase: C_out (a multiple of 32) columns, two loads per wait
#pragma unroll 1
                        for (int cb = k0; cb < k0 + chn; cb += 32) {
                            uint32_t r0[16], r1[16];
                            __syncwarp();
                            ptx::tmem_ld16(tb + cb, r0);
                            ptx::tmem_ld16(tb + cb + 16, r1);
                            ptx::tmem_ld_wait();
                            stage16(cb, cb - k0, r0);
                            stage16(cb + 16, cb + 16 - k0, r1);
                        }
                    } else {
#pragma unroll 1
                        for (int cb = k0; cb < k0 + chn; cb += 16 * LDB) {
                            // LDB accumulator loads in flight per wait (their latency overlaps)
                            uint32_t rr[LDB][16];
                            __syncwarp();
#pragma unroll
                            for (int u = 0; u < LDB; ++u) ptx::tmem_ld16(tb + cb + 16 * u, rr[u]);
                            ptx::tmem_ld_wait();
#pragma unroll
                            for (int u = 0; u < LDB; ++u) stage16(cb + 16 * u, cb + 16 * u, rr[u]);
                        }
                    }
                    ptx::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        if (p.mode == MODE_T)
                            ptx::tma_store_5d(&tmC, sbuf, (ph & 1) * p.out_cs + p.out_coff + k0, bx, ph >> 1, by, n);
                        else if (t3) // phase k0 / C_out: output row parity >> 1, column parity & 1
                            ptx::tma_store_5d(&tmC, sbuf, ((int)p.fdco.div((uint32_t)k0) & 1) * p.out_cs + p.out_coff,
                                              bx, (int)p.fdco.div((uint32_t)k0) >> 1, by, n);
                        else
                            ptx::tma_store_4d(&tmC, sbuf, p.out_coff + k0, bx, by, n);
                        ptx::bulk_commit();
                    }
                    ++scnt;
                }
            }
            } else {
#pragma unroll 1
            for (int m = 0; m < MT; ++m) {
            // row block m of the tile: accumulator m, pixel rows m * 128 + lane row
            const int rm = m * 128 + row;
            const int gy = y0 + (rm >> p.tw_log), gx = x0 + (rm & (tw - 1));
            const bool valid = gy < p.gh && gx < p.gw;
            const uint32_t tb = tbase + m * BN;
#pragma unroll 1
            for (int c = 0; c < BN; c += 16) {
                uint32_t r[16];
                __syncwarp();
                if (BN == 16 && p.epi.mode == EPI_OUTPUT) ptx::tmem_ld4(tb + c, r); // 3 output columns
                else ptx::tmem_ld16(tb + c, r);
                ptx::tmem_ld_wait();
                if (!valid || c >= ncols) continue;
                // output pixel and channel of column c (a chunk never straddles a
                // phase when C_out is a multiple of 16)
                int cph = p.mode == MODE_T3 ? (int)p.fdco.div((uint32_t)c) : ph;
                int co0 = p.mode == MODE_T3 ? c - cph * p.co : c;
                int oy = gy, ox = gx;
                if (p.mode == MODE_T || p.mode == MODE_T3) { oy = 2 * gy + (cph >> 1); ox = 2 * gx + (cph & 1); }
                if (BN == 16 && p.epi.mode == EPI_OUTPUT) {
                    // RefineNet's 16 -> 3 output conv (Sigmoid, Table 3) with the residual
                    // output: clamp(I_blend + 2 sigmoid(z) - 1, 0, 1) on the cropped grid
                    if (oy < p.epi.crop_h && ox < p.epi.crop_w) {
                        const size_t q = ((size_t)n * p.out_h + oy) * p.out_w + ox;
                        float *o = out_final + (((size_t)n * p.epi.crop_h + oy) * p.epi.crop_w + ox) * 3;
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const float z = __uint_as_float(r[j]) + obias[j];
                            // (1 + e^-z >= 1: the fast reciprocal division is within 2 ulp;
                            // the fast exponential adds ~2^-21 relative, far inside BF16)
                            const float res = __fdividef(2.f, 1.f + __expf(-z)) - 1.f;
                            const float ibv = ibt ? ibt[(ox - x0) * 3 + j] : __ldg(p.epi.ib + q * 3 + j);
                            o[j] = fminf(fmaxf(ibv + res, 0.f), 1.f);
                        }
                    }
                    continue;
                }
                if (p.epi.mode == EPI_STORE && !p.out_f32 && p.vec_ok && co0 + 16 <= p.co && (co0 & 3) == 0) {
                    float v[16], bq[16], sq[16];
                    bias_scale16<SB, F8>(p, sbias, sscale, co0, bq, sq);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float a = __uint_as_float(r[j]) * sq[j] + bq[j];
                        v[j] = p.relu ? fmaxf(a, 0.f) : a;
                    }
                    if (p.amax) { // calibration only
                        float vmax = 0.f;
#pragma unroll
                        for (int j = 0; j < 16; ++j) vmax = fmaxf(vmax, fabsf(v[j]));
                        atomicMax(reinterpret_cast<int *>(p.amax), __float_as_int(vmax));
                    }
                    size_t pix = ((size_t)n * p.out_h + oy) * p.out_w + ox;
                    if (p.out_fp8) {
                        *reinterpret_cast<uint4 *>((uint8_t *)p.out + pix * p.out_cs + p.out_coff + co0) =
                            e4m3x16(v, p.out_q);
                    } else {
                        __nv_bfloat162 h[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        uint4 w0, w1;
                        memcpy(&w0, &h[0], 16);
                        memcpy(&w1, &h[4], 16);
                        bf16 *dst = (bf16 *)p.out + pix * p.out_cs + p.out_coff + co0;
                        reinterpret_cast<uint4 *>(dst)[0] = w0;
                        reinterpret_cast<uint4 *>(dst)[1] = w1;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (c + j >= ncols) break;
                        int col = c + j, pj = cph, co = col;
                        int yy = oy, xx = ox;
                        if (p.mode == MODE_T3) {
                            pj = (int)p.fdco.div((uint32_t)col);
                            co = col - pj * p.co;
                            yy = 2 * gy + (pj >> 1);
                            xx = 2 * gx + (pj & 1);
                        }
                        epi_elem<SB>(p, sbias, sscale, n, yy, xx, co, __uint_as_float(r[j]));
                    }
                }
            }
            }
            if (ibr) { // this warp is done with the tile's I_blend slot
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->empty[STAGES + 1 + tk % NIB]));
            }
            }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(ptx::smem_u32(&bars->tmem_empty[acc]));
            if (++acc == ACCB) { acc = 0; acc_phase ^= 1; }
        }
        // every TMA store of this warp has finished before shared memory goes away
        if (TS && lane == 0) ptx::bulk_wait<0>();
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// Host side: tensor maps, weight packing, tile shape choice, launch.

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int get_encoder() {
    if (g_encode) return FVV_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        set_error("cuTensorMapEncodeTiled unavailable (%s)", cudaGetErrorString(e));
        return FVV_ECUDA;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return FVV_OK;
}

bool g_encode_u8 = false; // next encode() describes 1-byte (FP8) elements
bool g_encode_l2_64 = false; // next encode() asks for 64-byte L2 fills (instead of 256)

CUtensorMapSwizzle swz_for(int ck_bytes) {
    return ck_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                           : (ck_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

int encode(CUtensorMap *m, int rank, void *base, const cuuint64_t *dims, const cuuint64_t *strides_bytes,
           const cuuint32_t *box, int ck_bytes) {
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = g_encode(m, g_encode_u8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, base,
                          dims, strides_bytes, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz_for(ck_bytes),
                          g_encode_l2_64 ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d), rank %d", (int)r, rank);
        return FVV_ECUDA;
    }
    return FVV_OK;
}

int pad16(int c) { return (c + 15) / 16 * 16; }
int ci_pad_of(int ci) { return ci <= 16 ? 16 : (ci <= 32 ? 32 : (ci + 63) / 64 * 64); }
int ck_of(int ci_pad) { return ci_pad >= 64 ? 64 : ci_pad; }

struct Shape { int th_log, tw_log; };

// Tile rectangle of 2^pix_log pixels with the fewest tiles covering gh x gw (ties: wider).
Shape pick_shape(int gh, int gw, int pix_log) {
    Shape best{pix_log - 4, 4};
    long best_tiles = -1;
    for (int tw_log = pix_log; tw_log >= 3; --tw_log) {
        int th_log = pix_log - tw_log;
        if (tw_log > 8 || th_log > 8) continue; // TMA box dimensions are at most 256
        long tiles = (long)ceil_div(gh, 1 << th_log) * ceil_div(gw, 1 << tw_log);
        if (best_tiles < 0 || tiles < best_tiles) { best_tiles = tiles; best = {th_log, tw_log}; }
    }
    return best;
}

// Row blocks per tile: two for the wide layers (the weight slice then feeds two MMAs).
// (N = 256 keeps one block: two 256-column accumulators would fill TMEM and lose the
// double buffering that hides the epilogue.)
int mt_for(int bn, int ck, int es) { return ck * es == 128 && bn == 128 ? 2 : 1; }

// Resources of one (N tile, channel block, row blocks) configuration.  Small-N
// configs put several CTAs on an SM (their TMEM columns and shared memory allow
// it), so more TMA copies are in flight per SM: those layers are bound by copy latency.
constexpr uint32_t kSmemBudget = 220 * 1024; // per SM, for all resident CTAs
// TS = 1 adds the epilogue's staging buffers (4 warps x 2 x 32 rows).
// (4 warps x NSB buffers x 32 rows; NSB = 1 for two row blocks per tile)
constexpr uint32_t stg_bytes(int bn, int ts, int mt = 1) {
    return ts ? (mt == 2 ? 4u : 8u) * 32u * (bn * 2 < 128 ? bn * 2 : 128) : 0u;
}
template <int BN, int CK, int MT, int F8 = 0, int TS = 0> struct Cfg {
    static constexpr uint32_t ES = F8 ? 1 : 2;
    static constexpr uint32_t A = ((128 * MT * CK * ES) + 1023) & ~1023u, B = ((BN * CK * ES) + 1023) & ~1023u;
    static constexpr uint32_t STG = stg_bytes(BN, TS, MT);
    static constexpr uint32_t TMEM_COLS = AccCfg<BN, MT>::TMEM_COLS;
    static constexpr int stages_for(int ctas) { return (int)((kSmemBudget / ctas - 2048 - STG) / (A + B)); }
    static constexpr int ctas_for(int c) { return c > 1 && stages_for(c) < 3 + !TS ? ctas_for(c - 1) : c; }
    static constexpr int CTAS = ctas_for((512 / TMEM_COLS) < 4 ? (512 / TMEM_COLS) : 4);
    static constexpr int STAGES = stages_for(CTAS) > 8 ? 8 : stages_for(CTAS);
    static constexpr size_t SMEM = (size_t)STAGES * (A + B) + STG + sizeof(Bars) + 8 * BN + 1024;
    static_assert(STAGES >= 2 && CTAS * TMEM_COLS <= 512, "tensor-core config");
};

int g_num_sms = 0;

template <int BN, int CK, int F8, int TS>
int launch_cfg(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const TcParams &p,
               cudaStream_t st) {
    constexpr int MT = (CK * (F8 ? 1 : 2) == 128 && BN == 128) ? 2 : 1; // = mt_for(BN, CK, ES)
    using C = Cfg<BN, CK, MT, F8, TS>;
    auto kern = conv_tc_kernel<BN, CK, MT, C::STAGES, C::CTAS, F8, 0, C::STAGES, TS>;
    static bool attr_set = false;
    if (!attr_set) {
        FVV_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
        attr_set = true;
    }
    if (!g_num_sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    int slots = g_num_sms * C::CTAS;
    int grid = p.num_tiles < slots ? p.num_tiles : slots;
    kern<<<grid, kThreads, C::SMEM, st>>>(ma, mb, mc, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

// Halo configurations (128-byte operand rows, one accumulator block): A boxes of
// 130 rows and B slices in separate rings, sized per N tile by hand so that the
// resident CTAs fill the shared-memory budget.
// MT = 2 (N = 256): tiles of 2 x 128 pixels, each weight slice feeds two MMAs; the
// two accumulators fill TMEM, so the epilogue is not overlapped with the next tile.
template <int BN, int TS, int MT = 1> struct HaloCfg {
    static constexpr uint32_t A = (130 * MT * 128 + 1023) & ~1023u, B = ((BN * 128) + 1023) & ~1023u;
    static constexpr uint32_t STG = stg_bytes(BN, TS, MT);
    static constexpr uint32_t TMEM_COLS = AccCfg<BN, MT>::TMEM_COLS;
    static constexpr int CTAS = BN >= 256 ? 1 : (BN >= 64 || TS ? 2 : 3);
    // N = 256: one A box feeds 3 weight slices (~0.8 us of MMA), so two A stages
    // suffice and the weight ring gets the rest (its slices are 32 KB).
    static constexpr int STAGES = MT == 2 ? 2
                                  : TS ? (BN >= 256 ? 2 : (BN >= 128 ? 2 : (BN >= 64 ? 3 : 4)))
                                       : (BN >= 256 ? 2 : (BN >= 128 ? 3 : (BN >= 64 ? 4 : 3)));
    static constexpr int STAGES_B = TS ? (BN >= 256 ? 4 : (BN >= 128 ? 2 : (BN >= 64 ? 3 : 4)))
                                       : (BN >= 256 ? 5 : (BN >= 128 ? 3 : 4));
    static constexpr size_t SMEM = (size_t)STAGES * A + (size_t)STAGES_B * B + STG + sizeof(Bars) + 8 * BN + 1024;
    static_assert(CTAS * SMEM <= kSmemBudget + 8 * 1024 && CTAS * TMEM_COLS <= 512 && STAGES >= 2 && STAGES_B >= 2,
                  "halo config");
};

// Grouped halo stages (a stage = one A box + its three weight slices) for the small-N
// layers: the narrow 16/32-channel convs, the VIB t1 and RefineNet d3 transposed convs
// (measured 3-18% faster than split A/B rings; the 64-column convs with the
// TMA-store epilogue keep split rings, which fit two CTAs per SM).
// RES = 1: the nine weight slices of a one-block layer resident (BR bytes), stages hold A only.
// N <= 32: up to four CTAs per SM where two stages fit (more epilogue warps: the 16 -> 3
// output conv 388 -> 328 us against three).
template <int BN, int CK, int TS, int F8 = 0, int RES = 0> struct HaloGrpCfg {
    static constexpr uint32_t ES = F8 ? 1 : 2;
    static constexpr uint32_t A = (130 * CK * ES + 1023) & ~1023u;
    static constexpr uint32_t G = RES ? A : A + ((3 * BN * CK * ES + 1023) & ~1023u);
    static constexpr uint32_t BR = RES ? ((9 * BN * CK * ES + 1023) & ~1023u) : 0u;
    // (+ the output conv's I_blend ring: N = 16, resident weights, no TMA-store staging)
    static constexpr uint32_t STG = stg_bytes(BN, TS) + (BN == 16 && !TS && RES ? 4 * 128 * 3 * 4 : 0);
    static constexpr int stages_for(int ctas) { return (int)((kSmemBudget / ctas - 2048 - STG - BR) / G); }
    static constexpr int ctas_for(int c) { return c > 1 && stages_for(c) < 2 ? ctas_for(c - 1) : c; }
    static constexpr int CTAS = ctas_for(BN <= 32 ? 4 : 2);
    static constexpr int STAGES = stages_for(CTAS) > 8 ? 8 : stages_for(CTAS);
    static constexpr size_t SMEM = (size_t)STAGES * G + BR + STG + sizeof(Bars) + 8 * BN + 1024;
    static_assert(STAGES >= 2 && CTAS * AccCfg<BN, 1>::TMEM_COLS <= 512, "grouped halo config");
};

template <int BN, int CK, int TS, int F8 = 0, int RES = 0>
int launch_halo_grp(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const TcParams &p,
                    cudaStream_t st) {
    using C = HaloGrpCfg<BN, CK, TS, F8, RES>;
    auto kern = conv_tc_kernel<BN, CK, 1, C::STAGES, C::CTAS, F8, 1, 2, TS, RES ? 2 : 1>;
    static bool attr_set = false;
    if (!attr_set) {
        FVV_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
        attr_set = true;
    }
    if (!g_num_sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    int slots = g_num_sms * C::CTAS;
    int grid = p.num_tiles < slots ? p.num_tiles : slots;
    kern<<<grid, kThreads, C::SMEM, st>>>(ma, mb, mc, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

// Folded column taps, NCK channel blocks: a stage is the 128 rows of four 32-pixel
// boxes, the 3 x NCK folded weight slices stay resident.  At least 3 stages per CTA.
template <int BN, int CK, int F8, int NCK> struct KxfCfg {
    static constexpr uint32_t ES = F8 ? 1 : 2;
    static constexpr uint32_t A = (128 * CK * ES + 1023) & ~1023u;
    static constexpr uint32_t BR = (3 * NCK * BN * CK * ES + 1023) & ~1023u;
    static constexpr uint32_t KST = 4 * 2 * 300 * 4; // Eq. 2 output staging, 4 epilogue warps
    static constexpr int stages_for(int ctas) { return (int)((kSmemBudget / ctas - 2048 - BR - KST) / A); }
    static constexpr int ctas_for(int c) { return c > 1 && stages_for(c) < 3 ? ctas_for(c - 1) : c; }
    static constexpr int CTAS = ctas_for(3);
    static constexpr int STAGES = stages_for(CTAS) > 8 ? 8 : stages_for(CTAS);
    static constexpr size_t SMEM = (size_t)STAGES * A + BR + KST + sizeof(Bars) + 8 * BN + 1024;
    static_assert(STAGES >= 2 && STAGES < 16 && CTAS * AccCfg<BN, 1>::TMEM_COLS <= 512, "folded-tap config");
};

template <int BN, int CK, int F8, int NCK>
int launch_kxf(const CUtensorMap &ma, const CUtensorMap &mk, const TcParams &p, cudaStream_t st) {
    using C = KxfCfg<BN, CK, F8, NCK>;
    auto kern = conv_tc_kernel<BN, CK, 1, C::STAGES, C::CTAS, F8, 1, 2, 0, 2, 0, NCK>;
    static bool attr_set = false;
    if (!attr_set) {
        FVV_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
        attr_set = true;
    }
    if (!g_num_sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    int slots = g_num_sms * C::CTAS;
    int grid = p.num_tiles < slots ? p.num_tiles : slots;
    kern<<<grid, kThreads, C::SMEM, st>>>(ma, mk, ma, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

template <int BN, int F8, int TS, int MT = 1>
int launch_halo(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const TcParams &p,
                cudaStream_t st) {
    using C = HaloCfg<BN, TS, MT>;
    constexpr int CK = F8 ? 128 : 64;
    auto kern = conv_tc_kernel<BN, CK, MT, C::STAGES, C::CTAS, F8, 1, C::STAGES_B, TS>;
    static bool attr_set = false;
    if (!attr_set) {
        FVV_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
        attr_set = true;
    }
    if (!g_num_sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    int slots = g_num_sms * C::CTAS;
    int grid = p.num_tiles < slots ? p.num_tiles : slots;
    kern<<<grid, kThreads, C::SMEM, st>>>(ma, mb, mc, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

// Row blocks per halo tile of the N = 256 layers.  2 halves the weight traffic per
// FLOP but leaves no TMEM for a second accumulator; measured on the 1080p VIBlock
// convs it is ~20% slower than 1 (the epilogue no longer overlaps the next tile).
constexpr int kHaloMT256 = 1;

bool halo_ok(int bn, int ck, int es, bool f8) {
    if (ck * es == 128) return f8 ? (bn == 256 || bn == 32) : (bn == 32 || bn == 64 || bn == 128 || bn == 256);
    return !f8 && ((bn == 16 && ck == 16) || (bn == 32 && ck == 32));
}

// (mb3: box of 3 taps, for the grouped stages)
template <int TS>
int dispatch_halo_ts(int bn, int ck, bool f8, const CUtensorMap &ma, const CUtensorMap &mb,
                     const CUtensorMap &mb3, const CUtensorMap &mc, const TcParams &p, cudaStream_t st) {
    if (f8) // the 256-channel convs; the all-phase t1 (N = 32) on grouped stages
        return bn == 32 ? launch_halo_grp<32, 128, TS, 1>(ma, mb3, mc, p, st)
                        : launch_halo<256, 1, TS, kHaloMT256>(ma, mb, mc, p, st);
    // the 16 / 32-channel convs (one channel block): weight slices resident
    if (ck == 16) return launch_halo_grp<16, 16, TS, 0, 1>(ma, mb3, mc, p, st);
    if (ck == 32) return launch_halo_grp<32, 32, TS, 0, 1>(ma, mb3, mc, p, st);
    switch (bn) {
    case 32: return launch_halo_grp<32, 64, TS>(ma, mb3, mc, p, st);
    case 64: return p.mode == MODE_T3 && !TS ? launch_halo_grp<64, 64, 0, 0, 1>(ma, mb3, mc, p, st)
                                             : launch_halo<64, 0, TS>(ma, mb, mc, p, st);
    case 128: return launch_halo<128, 0, TS>(ma, mb, mc, p, st);
    default: return launch_halo<256, 0, TS, kHaloMT256>(ma, mb, mc, p, st);
    }
}

int dispatch_halo(int bn, int ck, bool f8, const CUtensorMap &ma, const CUtensorMap &mb,
                  const CUtensorMap &mb3, const CUtensorMap &mc, const TcParams &p, cudaStream_t st) {
    return p.tma_store ? dispatch_halo_ts<1>(bn, ck, f8, ma, mb, mb3, mc, p, st)
                       : dispatch_halo_ts<0>(bn, ck, f8, ma, mb, mb3, mc, p, st);
}

// Stride-2 pair halo: an A ring of 129-pair boxes, the nine weight slices resident.
// As many CTAs per SM as keep at least four A stages.
template <int BN, int CK, int TS> struct S2hCfg {
    static constexpr int A = (129 * 4 * CK + 1023) & ~1023, BR = (9 * BN * CK * 2 + 1023) & ~1023;
    static constexpr int STG = (int)stg_bytes(BN, TS);
    static constexpr int TMEM_COLS = (int)AccCfg<BN, 1>::TMEM_COLS;
    static constexpr int stages_for(int c) { return ((int)kSmemBudget / c - 2048 - STG - BR) / A; }
    static constexpr int ctas_for(int c) { return c > 1 && stages_for(c) < 4 ? ctas_for(c - 1) : c; }
    static constexpr int CTAS = ctas_for(512 / TMEM_COLS < 4 ? 512 / TMEM_COLS : 4);
    static constexpr int STAGES = stages_for(CTAS) > 8 ? 8 : stages_for(CTAS);
    static constexpr size_t SMEM = (size_t)STAGES * A + BR + STG + sizeof(Bars) + 8 * BN + 1024;
    static_assert(STAGES >= 3 && CTAS * TMEM_COLS <= 512, "stride-2 halo config");
};

template <int BN, int CK, int TS>
int launch_s2h(const CUtensorMap &ma, const CUtensorMap &mb3, const CUtensorMap &mc, const TcParams &p,
               cudaStream_t st) {
    using C = S2hCfg<BN, CK, TS>;
    auto kern = conv_tc_kernel<BN, CK, 1, C::STAGES, C::CTAS, 0, 0, C::STAGES, TS, 0, 1>;
    static bool attr_set = false;
    if (!attr_set) {
        FVV_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
        attr_set = true;
    }
    if (!g_num_sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    int slots = g_num_sms * C::CTAS;
    int grid = p.num_tiles < slots ? p.num_tiles : slots;
    kern<<<grid, kThreads, C::SMEM, st>>>(ma, mb3, mc, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

// (N tile, channel block) pairs with a stride-2 pair-halo kernel: VIB0's input conv
// (16 channels -> 128), RefineNet e0a and ContextNet c2 (16 -> 32), c4 (32 -> 64).  The
// 32 -> 128 VIB input convs keep the per-tap tiles: their 72 KB of resident weights
// leave room for one CTA per SM, measured 8% slower at 1080p (VIB2 c0 483 -> 525 us).
bool s2h_ok(int bn, int ck) { return (bn == 128 && ck == 16) || (bn == 32 && ck == 16) || (bn == 64 && ck == 32); }

template <int TS>
int dispatch_s2h_ts(int bn, int ck, const CUtensorMap &ma, const CUtensorMap &mb3, const CUtensorMap &mc,
                    const TcParams &p, cudaStream_t st) {
    if (bn == 128 && ck == 16) return launch_s2h<128, 16, TS>(ma, mb3, mc, p, st);
    if (bn == 32 && ck == 16) return launch_s2h<32, 16, TS>(ma, mb3, mc, p, st);
    if (bn == 64 && ck == 32) return launch_s2h<64, 32, TS>(ma, mb3, mc, p, st);
    set_error("no stride-2 halo kernel for N=%d, CK=%d", bn, ck);
    return FVV_EINVAL;
}

template <int TS>
int dispatch_ts(int bn, int ck, bool f8, const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc,
                const TcParams &p, cudaStream_t st) {
    if (f8) {
        if (bn == 256 && ck == 128) return launch_cfg<256, 128, 1, TS>(ma, mb, mc, p, st);
        if (bn == 128 && ck == 128) return launch_cfg<128, 128, 1, TS>(ma, mb, mc, p, st);
        if (bn == 32 && ck == 128) return launch_cfg<32, 128, 1, TS>(ma, mb, mc, p, st);
        set_error("no FP8 tensor-core kernel for N=%d, CK=%d", bn, ck);
        return FVV_EINVAL;
    }
#define FVV_CASE(BN_, CK_) \
    if (bn == BN_ && ck == CK_) return launch_cfg<BN_, CK_, 0, TS>(ma, mb, mc, p, st);
    FVV_CASE(16, 16) FVV_CASE(16, 64) FVV_CASE(32, 16) FVV_CASE(32, 32) FVV_CASE(32, 64)
    FVV_CASE(64, 32) FVV_CASE(64, 64) FVV_CASE(128, 16) FVV_CASE(128, 32) FVV_CASE(128, 64)
    FVV_CASE(256, 64)
#undef FVV_CASE
    set_error("no tensor-core kernel for N=%d, CK=%d", bn, ck);
    return FVV_EINVAL;
}

int dispatch(int bn, int ck, bool f8, const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc,
             const TcParams &p, cudaStream_t st) {
    return p.tma_store ? dispatch_ts<1>(bn, ck, f8, ma, mb, mc, p, st) : dispatch_ts<0>(bn, ck, f8, ma, mb, mc, p, st);
}

} // namespace

// A bf16 tensor map with the swizzle of ck_bytes-wide rows, for the kernels of other files.
int tc_encode_map(CUtensorMap *m, int rank, void *base, const cuuint64_t *dims, const cuuint64_t *strides_bytes,
                  const cuuint32_t *box, int ck_bytes) {
    return encode(m, rank, base, dims, strides_bytes, box, ck_bytes);
}

// Pack every layer's weights as bf16 [G][Co_pad][Ci_pad] (G = 9 taps, or 4 phases
// x 4 taps for the transposed conv) and build its B tensor map.
int tc_prepare_fp8(fvv_interp *h, const float *blob);

// Layers whose column taps are folded into N: the VIB t1 transposed convs (all four
// phases, 4 x 5 columns per tap: N = 64 instead of 3 MMAs of N = 32 per K step), BF16.
bool tc_kxf_layer(int li) {
    const LayerDef &L = kLayers[li];
    return L.kind == K_CONVT && tc_all_phases(li) && L.co == 5;
}

// Folded weights from the per-tap packing pk ([9][cop][cip], element type T): slice ky
// holds rows kx * G + j = row j of tap (ky, kx), padded to nk rows; uploaded to tw.wk
// with map_k (box: one channel block of the 3 slices).
template <typename T>
int fold_column_taps(fvv_interp *h, TcWeights &tw, const std::vector<T> &pk, int cop, int cip, int G, int ck) {
    const int nk = pad16(3 * G);
    std::vector<T> f((size_t)3 * nk * cip);
    memset(f.data(), 0, f.size() * sizeof(T)); // +0 in bf16 and in E4M3
    for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx)
            for (int j = 0; j < G; ++j)
                memcpy(&f[((size_t)ky * nk + kx * G + j) * cip], &pk[((size_t)(ky * 3 + kx) * cop + j) * cip],
                       cip * sizeof(T));
    FVV_TRY(dalloc(h, &tw.wk, f.size() * sizeof(T)));
    FVV_CHECK_CUDA(cudaMemcpy(tw.wk, f.data(), f.size() * sizeof(T), cudaMemcpyHostToDevice));
    const cuuint64_t es = sizeof(T);
    cuuint64_t dims[3] = {(cuuint64_t)cip, (cuuint64_t)nk, 3};
    cuuint64_t strides[2] = {(cuuint64_t)cip * es, (cuuint64_t)nk * cip * es};
    cuuint32_t box[3] = {(cuuint32_t)ck, (cuuint32_t)nk, 3};
    g_encode_u8 = sizeof(T) == 1;
    int rc = encode((CUtensorMap *)tw.map_k, 3, tw.wk, dims, strides, box, ck * (int)es);
    g_encode_u8 = false;
    FVV_TRY(rc);
    tw.kxf_n = nk;
    return FVV_OK;
}

int tc_prepare(fvv_interp *h, const float *blob) {
    FVV_TRY(get_encoder());
    size_t off = 0;
    struct Fold { int li; std::vector<bf16> pk; int cop, cip, G, ck; };
    std::vector<Fold> folds;
    for (int i = 0; i < kNumLayers; ++i) {
        const LayerDef &L = kLayers[i];
        const bool t3 = tc_all_phases(i);
        int taps = L.kind == K_CONV || t3 ? 9 : 16;  // B slices: conv/all-phase taps, or phase x tap
        int cip = ci_pad_of(L.ci), cop = pad16(t3 ? 4 * L.co : L.co);
        const float *w = blob + off;
        off += (size_t)L.ci * L.co * (L.kind == K_CONV ? 9 : 16) + L.co;
        std::vector<bf16> pk((size_t)taps * cop * cip, __float2bfloat16_rn(0.f));
        if (L.kind == K_CONV) {
            for (int tap = 0; tap < 9; ++tap)
                for (int co = 0; co < L.co; ++co)
                    for (int ci = 0; ci < L.ci; ++ci)
                        pk[((size_t)tap * cop + co) * cip + ci] = __float2bfloat16_rn(w[((size_t)co * L.ci + ci) * 9 + tap]);
        } else if (t3) {
            // tap (dy, dx) in {-1,0,1}^2 of phase (py, px): rows dy in {-1, 0} (py = 0,
            // kernel rows 3, 1) or {0, 1} (py = 1, kernel rows 2, 0); same for columns
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    for (int py = 0; py < 2; ++py)
                        for (int px = 0; px < 2; ++px) {
                            bool oky = py == 0 ? dy <= 0 : dy >= 0, okx = px == 0 ? dx <= 0 : dx >= 0;
                            if (!oky || !okx) continue;
                            int ky = py == 0 ? (dy == 0 ? 1 : 3) : (dy == 1 ? 0 : 2);
                            int kx = px == 0 ? (dx == 0 ? 1 : 3) : (dx == 1 ? 0 : 2);
                            int tap = (dy + 1) * 3 + (dx + 1), ph = py * 2 + px;
                            for (int co = 0; co < L.co; ++co)
                                for (int ci = 0; ci < L.ci; ++ci)
                                    pk[((size_t)tap * cop + ph * L.co + co) * cip + ci] =
                                        __float2bfloat16_rn(w[((size_t)ci * L.co + co) * 16 + ky * 4 + kx]);
                        }
        } else {
            for (int py = 0; py < 2; ++py)
                for (int px = 0; px < 2; ++px)
                    for (int ty = 0; ty < 2; ++ty)
                        for (int tx = 0; tx < 2; ++tx) {
                            int ky = py == 0 ? 1 + 2 * ty : 2 * ty, kx = px == 0 ? 1 + 2 * tx : 2 * tx;
                            int g = (py * 2 + px) * 4 + ty * 2 + tx;
                            for (int co = 0; co < L.co; ++co)
                                for (int ci = 0; ci < L.ci; ++ci)
                                    pk[((size_t)g * cop + co) * cip + ci] =
                                        __float2bfloat16_rn(w[((size_t)ci * L.co + co) * 16 + ky * 4 + kx]);
                        }
        }
        TcWeights &tw = h->tc[i];
        tw.ci_pad = cip;
        tw.co_pad = cop;
        FVV_TRY(dalloc(h, &tw.w, pk.size() * 2));
        FVV_CHECK_CUDA(cudaMemcpy(tw.w, pk.data(), pk.size() * 2, cudaMemcpyHostToDevice));
        int ck = ck_of(cip);
        cuuint64_t dims[3] = {(cuuint64_t)cip, (cuuint64_t)cop, (cuuint64_t)taps};
        cuuint64_t strides[2] = {(cuuint64_t)cip * 2, (cuuint64_t)cip * cop * 2};
        cuuint32_t box[3] = {(cuuint32_t)ck, (cuuint32_t)cop, 1};
        static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
        FVV_TRY(encode((CUtensorMap *)tw.map, 3, tw.w, dims, strides, box, ck * 2));
        if (taps == 9) { // three consecutive taps (one row tap's column taps) per box
            box[2] = 3;
            FVV_TRY(encode((CUtensorMap *)tw.map3, 3, tw.w, dims, strides, box, ck * 2));
            box[2] = 1;
        }
        // (and RefineNet's output conv and d3, whose dedicated kernels read the folded slices)
        if (tc_kxf_layer(i) || i == kRef + 12 || i == kRef + 11)
            folds.push_back({i, std::move(pk), cop, cip, t3 ? 4 * L.co : L.co, ck});
    }
    // folded copies allocated after every layer's own weights: the per-layer weight
    // allocations keep the addresses they have without them (the per-tap convs reload
    // their slices from L2 on every tile, and where those land in L2 was measured to
    // change their speed by up to 40 %)
    for (Fold &f : folds) FVV_TRY(fold_column_taps(h, h->tc[f.li], f.pk, f.cop, f.cip, f.G, f.ck));
    // the VIB1 / VIB2 input convs (18 -> 128, stride 2, per-tap tiles): four weight copies
    for (int i = 0; i < kNumLayers; ++i) {
        const LayerDef &L = kLayers[i];
        if (!(L.kind == K_CONV && L.stride == 2 && L.ci == 18 && L.co == 128)) continue;
        TcWeights &tw = h->tc[i];
        const int copies = 4, cip = tw.ci_pad, cop = tw.co_pad, ck = ck_of(cip);
        const size_t one = (size_t)9 * cop * cip * 2;
        FVV_TRY(dalloc(h, &tw.wrep, copies * one));
        for (int c = 0; c < copies; ++c)
            FVV_CHECK_CUDA(cudaMemcpy((char *)tw.wrep + c * one, tw.w, one, cudaMemcpyDeviceToDevice));
        cuuint64_t dims[3] = {(cuuint64_t)cip, (cuuint64_t)cop, (cuuint64_t)(9 * copies)};
        cuuint64_t strides[2] = {(cuuint64_t)cip * 2, (cuuint64_t)cip * cop * 2};
        cuuint32_t box[3] = {(cuuint32_t)ck, (cuuint32_t)cop, 1};
        FVV_TRY(encode((CUtensorMap *)tw.map_rep, 3, tw.wrep, dims, strides, box, ck * 2));
        tw.wcopies = copies;
    }
    if (h->o.precision == FVV_FP8) FVV_TRY(tc_prepare_fp8(h, blob));
    return FVV_OK;
}

// E4M3 weights of the FP8 layers: per output channel s_w = max |w| / 448 over
// its taps and input channels, codes = RNE-satfinite(w / s_w), layout [slice][C_out][C_in]
// (9 conv taps, or the transposed conv's 16 phase x tap slices in the BF16 order).
int tc_prepare_fp8(fvv_interp *h, const float *blob) {
    size_t off = 0;
    for (int i = 0; i < kNumLayers; ++i) {
        const LayerDef &L = kLayers[i];
        const float *w = blob + off;
        off += (size_t)L.ci * L.co * (L.kind == K_CONV ? 9 : 16) + L.co;
        if (!fp8_layer(i)) continue;
        const bool conv = L.kind == K_CONV, t3 = tc_all_phases(i);
        // conv taps, the all-phase transposed conv's 3x3 taps, or phase x tap slices
        const int taps = conv || t3 ? 9 : 16;
        const int rows = t3 ? pad16(4 * L.co) : L.co; // weight rows = GEMM columns
        // kernel value of (output channel, input channel, kernel position): conv
        // weights are [C_out][C_in][3][3], transposed-conv weights [C_in][C_out][4][4]
        auto wv = [&](int co, int ci, int k) {
            return conv ? w[((size_t)co * L.ci + ci) * 9 + k] : w[((size_t)ci * L.co + co) * 16 + k];
        };
        std::vector<float> sw(L.co);
        std::vector<uint8_t> pk((size_t)taps * rows * L.ci, 0); // 0 = the E4M3 code of +0
        for (int co = 0; co < L.co; ++co) {
            float m = 0.f;
            for (int ci = 0; ci < L.ci; ++ci)
                for (int k = 0; k < (conv ? 9 : 16); ++k) m = fmaxf(m, fabsf(wv(co, ci, k)));
            sw[co] = m > 0.f ? m / 448.f : 1.f;
        }
        auto code = [&](int co, int ci, int k) {
            return (uint8_t)__nv_cvt_float_to_fp8(wv(co, ci, k) / sw[co], __NV_SATFINITE, __NV_E4M3);
        };
        if (t3) {
            // all phases: 3x3 tap (dy, dx) of phase (py, px) in column ph * C_out + co, the
            // same kernel positions as the BF16 packing; the 5 taps a phase skips stay 0
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    for (int py = 0; py < 2; ++py)
                        for (int px = 0; px < 2; ++px) {
                            if (!(py == 0 ? dy <= 0 : dy >= 0) || !(px == 0 ? dx <= 0 : dx >= 0)) continue;
                            const int ky = py == 0 ? (dy == 0 ? 1 : 3) : (dy == 1 ? 0 : 2);
                            const int kx = px == 0 ? (dx == 0 ? 1 : 3) : (dx == 1 ? 0 : 2);
                            const int tap = (dy + 1) * 3 + (dx + 1), ph = py * 2 + px;
                            for (int co = 0; co < L.co; ++co)
                                for (int ci = 0; ci < L.ci; ++ci)
                                    pk[((size_t)tap * rows + ph * L.co + co) * L.ci + ci] = code(co, ci, ky * 4 + kx);
                        }
        } else {
            for (int g = 0; g < taps; ++g) {
                // transposed conv slice g = phase (py, px) x tap (ty, tx): kernel row
                // 1 + 2 ty (py = 0) or 2 ty (py = 1), the same for columns
                const int py = g >> 3, px = (g >> 2) & 1, ty = (g >> 1) & 1, tx = g & 1;
                const int k = conv ? g : (py == 0 ? 1 + 2 * ty : 2 * ty) * 4 + (px == 0 ? 1 + 2 * tx : 2 * tx);
                for (int co = 0; co < L.co; ++co)
                    for (int ci = 0; ci < L.ci; ++ci) pk[((size_t)g * rows + co) * L.ci + ci] = code(co, ci, k);
            }
        }
        TcWeights &tw = h->tc8[i];
        tw.ci_pad = L.ci;
        tw.co_pad = rows;
        FVV_TRY(dalloc(h, &tw.w, pk.size()));
        FVV_CHECK_CUDA(cudaMemcpy(tw.w, pk.data(), pk.size(), cudaMemcpyHostToDevice));
        FVV_TRY(dalloc(h, (void **)&h->q_acc[i], L.co * sizeof(float)));
        h->s_w[i] = sw;
        cuuint64_t dims[3] = {(cuuint64_t)L.ci, (cuuint64_t)rows, (cuuint64_t)taps};
        cuuint64_t strides[2] = {(cuuint64_t)L.ci, (cuuint64_t)L.ci * rows};
        cuuint32_t box[3] = {128, (cuuint32_t)rows, 3}; // three consecutive taps (grouped stages)
        g_encode_u8 = true;
        int rc = taps == 9 ? encode((CUtensorMap *)tw.map3, 3, tw.w, dims, strides, box, 128) : FVV_OK;
        box[2] = 1;
        if (rc == FVV_OK) rc = encode((CUtensorMap *)tw.map, 3, tw.w, dims, strides, box, 128);
        g_encode_u8 = false;
        FVV_TRY(rc);
    }
    FVV_TRY(dalloc(h, (void **)&h->d_amax, kNumLayers * sizeof(float)));
    FVV_CHECK_CUDA(cudaMemset(h->d_amax, 0, kNumLayers * sizeof(float)));
    return FVV_OK;
}

// (C_out <= 32: VIB t1, RefineNet d2 and d3; one A fetch per MMA then serves the four
// phases' columns, which outweighs the zero taps for these narrow layers)
bool tc_all_phases(int li) { return kLayers[li].kind == K_CONVT && 4 * kLayers[li].co <= 128; }

int tc_conv(fvv_interp *h, int li, const void *in, int in_cs, int in_coff, int N, int Hin, int Win, void *out,
            int out_cs, int out_coff, bool out_f32, cudaStream_t st, const TcEpi *epi) {
    const LayerDef &L = kLayers[li];
    // FP8 once calibrated (calibration itself runs every layer in BF16)
    const bool f8_on = h->o.precision == FVV_FP8 && h->fp8_ready && !h->calibrating;
    const bool f8 = f8_on && fp8_layer(li);
    const TcWeights &tw = f8 ? h->tc8[li] : h->tc[li];
    const int es = f8 ? 1 : 2;                       // input element bytes
    const int cip = tw.ci_pad, ck = f8 ? 128 : ck_of(cip), bn = tw.co_pad;
    if (in_cs % (16 / es) || in_coff % (16 / es) || in_coff + cip > in_cs) {
        set_error("layer %s: input slice (cs %d, off %d, %d ch) not TMA-aligned", L.name, in_cs, in_coff, cip);
        return FVV_EINVAL;
    }
    // circular padding: the layer reads a copy of its input window with a wrapped border
    // of kCircPad pixels (TMA fills out-of-range coordinates with zeros only); the maps
    // cover the padded image, the kernel shifts its A coordinates by the pad
    int Hm = Hin, Wm = Win, ipad = 0;
    if (h->o.pad_mode == FVV_PAD_CIRCULAR) {
        const size_t need = (size_t)N * (Hin + 2 * kCircPad) * (Win + 2 * kCircPad) * cip * es;
        if (need > h->cpad_bytes) {
            set_error("layer %s: circular-pad buffer too small (%zu > %zu bytes)", L.name, need, h->cpad_bytes);
            return FVV_ESHAPE;
        }
        FVV_TRY(launch_wrap_pad(in, N, count_word(h, li), Hin, Win, in_cs * es, in_coff * es, cip * es, kCircPad,
                                h->cpad, st));
        in = h->cpad; in_cs = cip; in_coff = 0;
        Hm = Hin + 2 * kCircPad; Wm = Win + 2 * kCircPad; ipad = kCircPad;
    }
    TcParams p{};
    p.mode = L.kind == K_CONVT ? (tc_all_phases(li) ? MODE_T3 : MODE_T) : (L.stride == 2 ? MODE_S2 : MODE_S1);
    p.n_img = N;
    if (L.kind == K_CONV) { p.gh = (Hin - 1) / L.stride + 1; p.gw = (Win - 1) / L.stride + 1; }
    else { p.gh = Hin; p.gw = Win; }
    p.out_h = L.kind == K_CONV ? p.gh : 2 * Hin;
    p.out_w = L.kind == K_CONV ? p.gw : 2 * Win;
    const int mt = mt_for(bn, ck, es), pix_log = mt == 2 ? 8 : 7;
    Shape s = pick_shape(p.gh, p.gw, pix_log);
    const int force = h->tile_force >= 0 ? h->tile_force : h->tile_tw[li]; // autotuned width
    if (force >= 0) {
        int tw = force < pix_log ? force : pix_log;
        if (pix_log - tw <= 8) s = Shape{pix_log - tw, tw};
    }
    // default tile of the 3x3 stride-1 layers (and the all-phase transposed convs): one
    // row of 128 pixels, A loaded once per (ky, channel block) as a 130-pixel halo box
    const bool halo = force < 0 && (p.mode == MODE_S1 || p.mode == MODE_T3) && halo_ok(bn, ck, es, f8) &&
                      p.gw >= 96;
    // stride-2 layers whose input pixel is exactly one 16/32-channel block: one row of 128
    // output pixels, one box of 129 pixel pairs per row tap, resident weights
    const bool s2h = force < 0 && p.mode == MODE_S2 && !f8 && cip == ck && in_cs == cip && in_coff == 0 &&
                     s2h_ok(bn, ck) && p.gw >= 96 && (!epi || epi->mode == EPI_STORE);
    // column taps folded into N (VIB t1): rows of 120 output pixels
    // (the epilogue reads the accumulator in 4-column loads: 4 C_out % 4 == 0)
    // (grids narrower than 256 keep the per-row-tap boxes, measured faster on VIB0's
    // 240-wide grid; so does E4M3, whose K = 32 MMAs already take a third as many steps:
    // VIB2 t1 262 us there against 413 folded)
    const bool kxf = !f8 && halo && tc_kxf_layer(li) && tw.kxf_n == 64 && p.mode == MODE_T3 && cip == 128 && L.co == 5 &&
                     p.gw >= 256 &&
                     (!epi || epi->mode == EPI_STORE || epi->mode == EPI_RESID);
    const int halo_mt = bn == 256 ? kHaloMT256 : 1;
    if (halo) s = Shape{halo_mt - 1, 7};
    if (s2h) s = Shape{0, 7};
    p.th_log = s.th_log; p.tw_log = s.tw_log;
    p.tiles_y = ceil_div(p.gh, 1 << s.th_log);
    p.tiles_x = kxf ? ceil_div(p.gw, kKxfTile) : ceil_div(p.gw, 1 << s.tw_log);
    p.fdx = FastDiv((uint32_t)p.tiles_x);
    p.fdy = FastDiv((uint32_t)p.tiles_y);
    p.kxf = kxf ? 1 : 0;
    long long tiles = (long long)N * p.tiles_y * p.tiles_x * (p.mode == MODE_T ? 4 : 1);
    if (tiles > (1ll << 30)) { set_error("too many tiles"); return FVV_ESHAPE; }
    p.num_tiles = (int)tiles;
    p.nck = cip / ck;
    p.nck_log = 0;
    while ((1 << p.nck_log) < p.nck) ++p.nck_log;
    if ((1 << p.nck_log) != p.nck) { set_error("layer %s: channel blocks per tap not a power of two", L.name); return FVV_ESHAPE; }
    p.taps = p.mode == MODE_T ? 4 : 9;
    p.in_cs = in_cs; p.in_coff = in_coff;
    p.co = L.co; p.relu = L.relu; p.out_f32 = out_f32 ? 1 : 0;
    p.fdco = FastDiv((uint32_t)L.co);
    p.acc_scale = f8 ? h->q_acc[li] : nullptr;
    p.out_fp8 = f8_on && feeds_fp8(li) && !out_f32 ? 1 : 0;
    p.out_q = h->q_out[li];
    p.amax = h->calibrating && feeds_fp8(li) ? h->d_amax + li : nullptr;
    const int ovec = p.out_fp8 ? 16 : 8;             // elements per 16 bytes of output
    p.vec_ok = (out_cs % ovec == 0 && out_coff % ovec == 0 && ((uintptr_t)out % 16) == 0) ? 1 : 0;
    p.out = out; p.out_cs = out_cs; p.out_coff = out_coff;
    p.bias = h->bias + h->b_off[li];
    p.err = h->d_err;
    p.stall_cycles = h->stall_now;
    p.n_dev = count_word(h, li);
    p.ipad = ipad;
    if (epi) {
        p.epi = *epi;
        // the fused epilogues are written for the layers that use them
        bool ok = (epi->mode == EPI_STORE) ||
                  (epi->mode == EPI_RESID && p.mode == MODE_T3 && L.co == 5 && bn == 32 && out_f32 && out_cs == 5 &&
                   out_coff == 0) ||
                  (epi->mode == EPI_OUTPUT && p.mode == MODE_S1 && L.co == 3 && bn == 16 && !f8 && epi->ib &&
                   epi->final_out_ref && epi->crop_h <= p.gh && epi->crop_w <= p.gw);
        if (!ok) { set_error("layer %s: unsupported fused epilogue", L.name); return FVV_EINVAL; }
    }

    CUtensorMap ma;
    const int tw_ = 1 << s.tw_log, th_ = 1 << s.th_log;
    const cuuint64_t e = (cuuint64_t)es;
    g_encode_u8 = f8;
    int rc;
    if (p.mode == MODE_S2) {
        if (Hin % 2 || Win % 2) { g_encode_u8 = false; set_error("stride-2 layer %s needs even input size", L.name); return FVV_ESHAPE; }
        cuuint64_t dims[5] = {(cuuint64_t)2 * in_cs, (cuuint64_t)Wm / 2, 2, (cuuint64_t)Hm / 2, (cuuint64_t)N};
        cuuint64_t strides[4] = {(cuuint64_t)2 * in_cs * e, (cuuint64_t)Wm * in_cs * e,
                                 (cuuint64_t)2 * Wm * in_cs * e, (cuuint64_t)Hm * Wm * in_cs * e};
        if (s2h) { // 129 whole pixel pairs (2 x ck channels) of one input row
            cuuint32_t box[5] = {(cuuint32_t)(2 * ck), 129, 1, 1, 1};
            rc = encode(&ma, 5, (void *)in, dims, strides, box, 2 * ck * es);
        } else {
            cuuint32_t box[5] = {(cuuint32_t)ck, (cuuint32_t)tw_, 1, (cuuint32_t)th_, 1};
            // a channel slice of wider pixels (RefineNet's stride-2 encoders read their
            // level's slots): 64-byte L2 fills, so the unread channels are not fetched
            g_encode_l2_64 = in_cs > cip;
            rc = encode(&ma, 5, (void *)in, dims, strides, box, ck * es);
            g_encode_l2_64 = false;
        }
    } else {
        cuuint64_t dims[4] = {(cuuint64_t)in_cs, (cuuint64_t)Wm, (cuuint64_t)Hm, (cuuint64_t)N};
        cuuint64_t strides[3] = {(cuuint64_t)in_cs * e, (cuuint64_t)Wm * in_cs * e, (cuuint64_t)Hm * Wm * in_cs * e};
        // halo boxes: MT rows x 130 pixels (folded column taps: 32 pixels, four per stage)
        cuuint32_t box[4] = {(cuuint32_t)ck, (cuuint32_t)(kxf ? 32 : (halo ? tw_ + 2 : tw_)), (cuuint32_t)th_, 1};
        rc = encode(&ma, 4, (void *)in, dims, strides, box, ck * es);
    }
    g_encode_u8 = false;
    FVV_TRY(rc);
    // TMA-store epilogue: plain bf16 / E4M3 stores of whole 16-byte channel groups
    // (every output channel of the tile is a real channel: C_out = N tile)
    CUtensorMap mc = ma;
    {
        // (MODE_T3: one chunk per phase, C_out columns wide; only for N = 128 (RefineNet
        // d2): d3 (N = 64) keeps its grouped stages at two CTAs per SM, measured 2x faster
        // than with the staging buffers)
        const int oes = p.out_fp8 ? 1 : 2;
        const int chb = p.mode == MODE_T3 ? L.co * oes : (bn * oes < 128 ? bn * oes : 128);
        p.tma_store = !kxf && (!epi || epi->mode == EPI_STORE) && !out_f32 &&
                      (p.mode == MODE_T3 ? 4 * L.co == bn && bn == 128 && L.co % 32 == 0 : L.co == bn) &&
                      (chb == 32 || chb == 64 || chb == 128) && (out_cs * oes) % 16 == 0 &&
                      (out_coff * oes) % 16 == 0 && ((uintptr_t)out % 16) == 0;
        if (p.tma_store) {
            const cuuint64_t oe = (cuuint64_t)oes;
            const cuuint32_t bw = tw_ < 32 ? tw_ : 32, bh = 32 / bw;
            g_encode_u8 = p.out_fp8 != 0;
            if (p.mode == MODE_T || p.mode == MODE_T3) {
                cuuint64_t dims[5] = {(cuuint64_t)2 * out_cs, (cuuint64_t)p.gw, 2, (cuuint64_t)p.gh, (cuuint64_t)N};
                cuuint64_t strides[4] = {(cuuint64_t)2 * out_cs * oe, (cuuint64_t)p.out_w * out_cs * oe,
                                         (cuuint64_t)2 * p.out_w * out_cs * oe,
                                         (cuuint64_t)p.out_h * p.out_w * out_cs * oe};
                cuuint32_t box[5] = {(cuuint32_t)(chb / oes), bw, 1, bh, 1};
                rc = encode(&mc, 5, out, dims, strides, box, chb);
            } else {
                cuuint64_t dims[4] = {(cuuint64_t)out_cs, (cuuint64_t)p.out_w, (cuuint64_t)p.out_h, (cuuint64_t)N};
                cuuint64_t strides[3] = {(cuuint64_t)out_cs * oe, (cuuint64_t)p.out_w * out_cs * oe,
                                         (cuuint64_t)p.out_h * p.out_w * out_cs * oe};
                cuuint32_t box[4] = {(cuuint32_t)(chb / oes), bw, bh, 1};
                rc = encode(&mc, 4, out, dims, strides, box, chb);
            }
            g_encode_u8 = false;
            FVV_TRY(rc);
        }
    }
    if (kxf)
        return launch_kxf<64, 64, 0, 2>(ma, *(const CUtensorMap *)tw.map_k, p, st);
    if (s2h)
        return p.tma_store ? dispatch_s2h_ts<1>(bn, ck, ma, *(const CUtensorMap *)tw.map3, mc, p, st)
                           : dispatch_s2h_ts<0>(bn, ck, ma, *(const CUtensorMap *)tw.map3, mc, p, st);
    if (halo)
        return dispatch_halo(bn, ck, f8, ma, *(const CUtensorMap *)tw.map,
                             *(const CUtensorMap *)tw.map3, mc, p, st);
    if (p.mode == MODE_S2 && !f8 && tw.wcopies > 1) {
        p.wcopies = tw.wcopies;
        return dispatch(bn, ck, f8, ma, *(const CUtensorMap *)tw.map_rep, mc, p, st);
    }
    return dispatch(bn, ck, f8, ma, *(const CUtensorMap *)tw.map, mc, p, st);
}

} // namespace fvv
