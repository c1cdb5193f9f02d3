// RefineNet's last transposed conv d3 (Table 3: 4x4, stride 2, 64 -> 16, ReLU) as one 3x3
// conv over the input grid whose 4 x 16 output columns are the four output phases, with
// the column taps folded into N (N = 3 x 64 = 192).
//
// With N = 64 per tap the generic all-phase kernel issues 36 MMAs of 128 x 64 x 16 per
// 128-pixel row (9 taps x 4 channel steps), each re-reading its 4 KB A tile: the tensor
// pipe's operand traffic, not its math, sets that pace.  Folded, one MMA per (row tap ky,
// 16-channel step) computes, for every input pixel i of the row, the 192 columns
// (kx, phase, co) = W[ky][kx][phase][co] . in(i); output (phase, co) of pixel i then sums
// column (0, phase, co) of pixel i - 1, (1, ..) of i and (2, ..) of i + 1 (neighbouring
// TMEM lanes: warp shuffles).  12 MMAs per row instead of 36.
//
// Work: one persistent CTA per SM.  A tile is one input row y of a 120-pixel column strip;
// a CTA owns a contiguous range of tiles in (view, strip, row) order, so walking down a
// strip a tile loads only input row y + 1 (rows y - 1, y came with the tiles before it).
// Row slot: 128 rows of 128 bytes (the 64 input channels, SW128): accumulator lane
// 32 q + l is input pixel x0 - 1 + 30 q + l, four 32-pixel TMA boxes per row (zeros
// outside the grid = the zero padding).  Weights: the three folded row-tap slices, 192 x
// 64 channels each, resident.  Two accumulators of 192 columns in TMEM.
//
// Warps: 0 issues the copies, 1 allocates TMEM and issues the MMAs, 2-9 are the epilogue:
// warp 2 + 4 h + q reads TMEM lane quarter q and computes output row 2 y + h (phases
// 2 h, 2 h + 1): tap sums, bias, ReLU, bf16; its 30 input pixels' 60 output pixels x 32
// bytes (1920 contiguous bytes of the output row) are staged in shared memory, two output
// pixels per 64-byte row in the 64-byte swizzle, and one lane stores them with TMA.  Same arithmetic as the generic conv up to the FP32 order of the
// three column taps' sums.
#include <cuda.h>

#include <cstring>

#include "interp.h"
#include "tc_ptx.h"
#include "tc_wait.h"

namespace fvv {

// (csrc/conv_tc.cu) bf16 tensor map, rows of ck_bytes swizzled accordingly
int tc_encode_map(CUtensorMap *m, int rank, void *base, const cuuint64_t *dims, const cuuint64_t *strides_bytes,
                  const cuuint32_t *box, int ck_bytes);

namespace {

constexpr int kTw = 120;                                   // strip width (input pixels)
constexpr int kWp = 30;                                    // input pixels per epilogue warp
constexpr int kCi = 64, kCo = 16, kN = 192;                // N = 3 column taps x 4 phases x 16
constexpr uint32_t kRowBytes = kCi * 2;                    // 128
constexpr uint32_t kSlotBytes = 128 * kRowBytes;           // 16 KB: one input row (4 boxes)
constexpr uint32_t kBoxBytes = 32 * kRowBytes;             // 4 KB: one 32-pixel box
constexpr int kSlots = 6;                                  // the producer runs 4 tiles ahead
constexpr uint32_t kSliceBytes = kN * kRowBytes;           // 24 KB: one folded row-tap slice
constexpr int kThreads = 320;
constexpr uint32_t kIdesc = ptx::make_idesc(128, kN, 1, 1);
constexpr uint32_t kStgBytes = 2048;                       // per epilogue warp: 60 output pixels x 32 B,
                                                           // 512-byte aligned (the 64-byte swizzle's span)
static_assert(kStgBytes >= 2 * kWp * kCo * 2, "d3 staging");

struct __align__(16) CfBars {
    uint64_t wfull;
    uint64_t full[kSlots], empty[kSlots];
    uint64_t tmem_full[2], tmem_empty[2];
    uint64_t drain;
    uint64_t never; // signalled by nothing: the fault-injection wait
    uint32_t tmem_base;
    int abort;
};

constexpr uint32_t kOffSlot = 3 * kSliceBytes;             // 72 KB of weights
constexpr uint32_t kOffStg = kOffSlot + kSlots * kSlotBytes;
constexpr uint32_t kOffBars = kOffStg + 8 * kStgBytes;
constexpr size_t kSmem = kOffBars + sizeof(CfBars) + 1024;
static_assert(kSmem <= 227 * 1024, "folded transposed conv shared memory");
static_assert(kOffSlot % 1024 == 0 && kOffStg % 1024 == 0 && kOffBars % 16 == 0, "folded transposed conv layout");

struct CfParams {
    const float *bias;                // 16 output biases
    bf16 *out;                        // 2 h x 2 w x 16 per view (pixel stride 16)
    const int *n_dev;                 // device view count (size-bucket graphs), or NULL
    int n_img, h, w, strips;
    long long stall_cycles;           // fault injection (tests): > 0 makes the MMA warp wait on `never`
    int *err;
};

// Contiguous walk over (view, strip, row) without divisions after the first tile.
struct CfWalk {
    int n, strip, y, h, strips;
    bool cont;
    __device__ CfWalk(int t, int h_, int strips_) : h(h_), strips(strips_), cont(false) {
        const int per_view = h * strips;
        n = t / per_view;
        const int r = t - n * per_view;
        strip = r / h;
        y = r - strip * h;
    }
    __device__ void next() {
        cont = true;
        if (++y == h) { y = 0; cont = false; if (++strip == strips) { strip = 0; ++n; } }
    }
};
struct CfRing {
    int slot = 0;
    uint32_t par = 0;
    __device__ void step() { if (++slot == kSlots) { slot = 0; par ^= 1; } }
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

__global__ void __launch_bounds__(kThreads, 1)
convt_fold_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ CUtensorMap tmC, const CfParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = smem;
    uint8_t *sSlot = smem + kOffSlot;
    uint8_t *sStg = smem + kOffStg;
    CfBars *bars = (CfBars *)(smem + kOffBars);
    volatile int *abort = &bars->abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        ptx::mbar_init(ptx::smem_u32(&bars->wfull), 1);
        for (int s = 0; s < kSlots; ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_full[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_empty[a]), 8); // one arrive per epilogue warp
        }
        ptx::mbar_init(ptx::smem_u32(&bars->drain), 1);
        ptx::mbar_init(ptx::smem_u32(&bars->never), 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(&bars->tmem_base), 512); // two accumulators of 192 columns
        ptx::tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        ptx::prefetch_tmap(&tmC);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;

    const int n_img = p.n_dev ? min(__ldg(p.n_dev), p.n_img) : p.n_img;
    const int per_view = p.strips * p.h;
    const int num_tiles = n_img * per_view;
    const int per_cta = (num_tiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_begin = min(num_tiles, (int)blockIdx.x * per_cta), t_end = min(num_tiles, t_begin + per_cta);

    if (warp == 0) {
        // ---------------- copy producer ----------------
        if (lane == 0) {
            const uint32_t fw = ptx::smem_u32(&bars->wfull);
            ptx::mbar_arrive_expect_tx(fw, 3 * kSliceBytes);
            ptx::tma_load_3d(ptx::smem_u32(sB), &tmB, fw, 0, 0, 0); // the three folded slices
            CfRing ring;
            long long issued = 0;
            CfWalk tw(t_begin, p.h, p.strips);
            bool stop = false;
            for (int t = t_begin; t < t_end && !stop && !*abort; ++t, tw.next()) {
                const int x0 = tw.strip * kTw;
                // new input rows: y + 1, and y - 1, y where a segment starts
                for (int j = tw.cont ? 2 : 0; j < 3; ++j) {
                    if (!wait_bar(ptx::smem_u32(&bars->empty[ring.slot]), ring.par ^ 1u, abort, p.err, 1)) {
                        stop = true;
                        break;
                    }
                    const uint32_t fs = ptx::smem_u32(&bars->full[ring.slot]);
                    ptx::mbar_arrive_expect_tx(fs, kSlotBytes);
                    const uint32_t dst = ptx::smem_u32(sSlot) + ring.slot * kSlotBytes;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        ptx::tma_load_4d(dst + q * kBoxBytes, &tmA, fs, 0, x0 - 1 + kWp * q, tw.y - 1 + j, tw.n);
                    ++issued;
                    ring.step();
                }
            }
            // every copy issued has landed before the CTA can exit
            for (long long k = 1; k <= issued && k <= kSlots; ++k) {
                const long long q = issued - k;
                drain_wait(ptx::smem_u32(&bars->full[q % kSlots]), (uint32_t)((q / kSlots) & 1));
            }
            drain_wait(fw, 0);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            // fault injection: a wait that runs out records code 6 and raises the abort flag
            // before any MMA is issued; the other roles leave, the copies land, TMEM is freed
            if (p.stall_cycles > 0) wait_bar(ptx::smem_u32(&bars->never), 0, abort, p.err, 6, p.stall_cycles);
            bool ok = wait_bar(ptx::smem_u32(&bars->wfull), 0, abort, p.err, 3);
            ptx::tc_fence_after();
            const uint32_t bw = ptx::smem_u32(sB), sw = ptx::smem_u32(sSlot);
            int acc = 0;
            uint32_t acc_phase = 0;
            CfRing ring;
            int rs[3] = {0, 0, 0};
            uint32_t rp[3] = {0, 0, 0}; // slot and phase parity of input rows y - 1, y, y + 1
            bool issued_any = false;
            CfWalk tw(t_begin, p.h, p.strips);
            for (int t = t_begin; ok && t < t_end && !*abort; ++t, tw.next()) {
                if (tw.cont) { rs[0] = rs[1]; rp[0] = rp[1]; rs[1] = rs[2]; rp[1] = rp[2]; }
                for (int r = tw.cont ? 2 : 0; r < 3; ++r) {
                    rs[r] = ring.slot;
                    rp[r] = ring.par;
                    ring.step();
                }
                if (!wait_bar(ptx::smem_u32(&bars->tmem_empty[acc]), acc_phase ^ 1, abort, p.err, 2)) break;
                ptx::tc_fence_after();
                for (int r = 0; r < 3 && ok; ++r)
                    ok = wait_bar(ptx::smem_u32(&bars->full[rs[r]]), rp[r], abort, p.err, 3);
                if (!ok) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem + acc * 256;
#pragma unroll
                for (int ky = 0; ky < 3; ++ky) {
                    const uint32_t a0 = sw + rs[ky] * kSlotBytes, b0 = bw + ky * kSliceBytes;
#pragma unroll
                    for (int k = 0; k < kCi / 16; ++k) {
                        const uint64_t ad = ptx::smem_desc(a0 + k * 32, kRowBytes);
                        const uint64_t bd = ptx::smem_desc(b0 + k * 32, kRowBytes);
                        ptx::mma_bf16(d, ad, bd, kIdesc, (ky | k) != 0);
                    }
                }
                issued_any = true;
                ptx::mma_commit(ptx::smem_u32(&bars->tmem_full[acc]));
                // row y - 1 is done; y, y + 1 stay when the next tile continues
                ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[0]]));
                if (!(t + 1 < t_end && tw.y + 1 < p.h)) {
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[1]]));
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[2]]));
                }
                if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            }
            if (issued_any) {
                ptx::mma_commit(ptx::smem_u32(&bars->drain));
                drain_wait(ptx::smem_u32(&bars->drain), 0);
            }
        }
    } else {
        // ---------------- epilogue: output row 2 y + hh of 30 input pixels ----------------
        const int q = warp & 3, hh = (warp - 2) >> 2;
        const uint32_t stg = ptx::smem_u32(sStg + (warp - 2) * kStgBytes);
        float bias[kCo];
#pragma unroll
        for (int c = 0; c < kCo; ++c) bias[c] = __ldg(p.bias + c);
        const int wo = 2 * p.w;
        int acc = 0;
        uint32_t acc_phase = 0;
        CfWalk tw(t_begin, p.h, p.strips);
        for (int t = t_begin; t < t_end && !*abort; ++t, tw.next()) {
            const int xw = tw.strip * kTw + kWp * q; // the warp's first input pixel
            const int nw = min(kWp, p.w - xw);       // its input pixels inside the grid
            int ok = 1;
            if (lane == 0) ok = wait_bar(ptx::smem_u32(&bars->tmem_full[acc]), acc_phase, abort, p.err, 4);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            ptx::tc_fence_after();
            // the previous tile's store has read the staging rows
            if (lane == 0) ptx::bulk_wait_read<0>();
            __syncwarp();
            const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + acc * 256;
            const bool mine = lane >= 1 && lane <= nw;
            // phases 2 hh + px: 16 columns per phase in each column tap's block of 64
#pragma unroll
            for (int px = 0; px < 2; ++px) {
                const uint32_t c0 = (uint32_t)((2 * hh + px) * kCo);
                uint32_t ra[16], rb[16], rc[16];
                __syncwarp();
                ptx::tmem_ld16(tb + c0, ra);
                ptx::tmem_ld16(tb + 64 + c0, rb);
                ptx::tmem_ld16(tb + 128 + c0, rc);
                ptx::tmem_ld_wait();
                if (px == 1) {
                    // the accumulator is free once read
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->tmem_empty[acc]));
                }
                float v[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float left = __shfl_up_sync(0xffffffffu, __uint_as_float(ra[c]), 1);
                    const float right = __shfl_down_sync(0xffffffffu, __uint_as_float(rc[c]), 1);
                    v[c] = fmaxf(left + __uint_as_float(rb[c]) + right + bias[c], 0.f); // d3 has ReLU
                }
                // output pixel 2 i + px of this lane: 32 bytes = chunks 2 px, 2 px + 1 of the
                // lane's 64-byte staging row, chunk k stored at k ^ ((lane - 1) >> 1 & 3) (the
                // 64-byte swizzle of a 512-byte-aligned buffer)
                if (mine) {
                    const int r = lane - 1, key = (r >> 1) & 3;
                    const uint32_t row = stg + r * 64;
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        const uint4 u = make_uint4(pack_bf16x2(v[8 * hf], v[8 * hf + 1]), pack_bf16x2(v[8 * hf + 2], v[8 * hf + 3]),
                                                   pack_bf16x2(v[8 * hf + 4], v[8 * hf + 5]),
                                                   pack_bf16x2(v[8 * hf + 6], v[8 * hf + 7]));
                        ptx::st_shared_v4(row + (((2 * px + hf) ^ key) << 4), u);
                    }
                }
            }
            if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            // output row 2 y + hh, pixels 2 xw .. 2 xw + 2 nw - 1 = pixel pairs xw .. xw + nw - 1:
            // one box of 30 pairs x 64 bytes (the map clips the grid's right edge)
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0 && nw > 0) {
                ptx::tma_store_4d(&tmC, stg, 0, xw, 2 * tw.y + hh, tw.n);
                ptx::bulk_commit();
            }
        }
        if (lane == 0) ptx::bulk_wait<0>(); // the stores have completed before the CTA exits
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

} // namespace

bool convt_fold_ok(const fvv_interp *h, int li, int in_cs, int in_coff, int out_cs, int out_coff, bool out_f32) {
    const LayerDef &L = kLayers[li];
    return li == kRef + 11 && L.kind == K_CONVT && L.ci == kCi && L.co == kCo && L.relu && tc_all_phases(li) &&
           h->tc[li].ci_pad == kCi && h->tc[li].kxf_n == kN && h->tc[li].wk && h->o.pad_mode == FVV_PAD_ZERO &&
           in_cs % 8 == 0 && in_cs >= kCi && in_coff == 0 && out_cs == kCo && out_coff == 0 && !out_f32;
}

int tc_convt_fold(fvv_interp *h, int li, const void *in, int in_cs, int N, int hin, int win, void *out, const int *n_dev,
                  cudaStream_t st) {
    if (!convt_fold_ok(h, li, in_cs, 0, kCo, 0, false) || ((uintptr_t)in & 15) || ((uintptr_t)out & 15) || N < 1 ||
        hin < 1 || win < 1) {
        set_error("layer %s: not the folded transposed conv", kLayers[li].name);
        return FVV_EINVAL;
    }
    // the input: N x hin x win pixels of in_cs bf16 channels (the first 64 used); boxes of
    // one row x 32 pixels x 64 channels
    CUtensorMap ma;
    cuuint64_t dims[4] = {(cuuint64_t)in_cs, (cuuint64_t)win, (cuuint64_t)hin, (cuuint64_t)N};
    cuuint64_t strides[3] = {(cuuint64_t)in_cs * 2, (cuuint64_t)win * in_cs * 2, (cuuint64_t)hin * win * in_cs * 2};
    cuuint32_t box[4] = {kCi, 32, 1, 1};
    FVV_TRY(tc_encode_map(&ma, 4, (void *)in, dims, strides, box, 128));
    CfParams p{};
    p.bias = h->bias + h->b_off[li];
    p.out = (bf16 *)out;
    p.n_dev = n_dev;
    p.n_img = N;
    p.h = hin; p.w = win;
    p.strips = (win + kTw - 1) / kTw;
    p.err = h->d_err;
    p.stall_cycles = h->stall_now;
    const long long tiles = (long long)N * p.strips * hin;
    if (tiles > (1ll << 30)) { set_error("too many tiles"); return FVV_ESHAPE; }
    static int sms = 0;
    if (!sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FVV_CHECK_CUDA(cudaFuncSetAttribute(convt_fold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    }
    // the output: N x 2 hin rows of win pixel pairs (2 x 16 bf16 channels = 64 bytes); boxes
    // of one row x 30 pairs
    CUtensorMap mc;
    cuuint64_t odims[4] = {2 * kCo, (cuuint64_t)win, (cuuint64_t)(2 * hin), (cuuint64_t)N};
    cuuint64_t ostrides[3] = {4 * kCo, (cuuint64_t)win * 4 * kCo, (cuuint64_t)2 * hin * win * 4 * kCo};
    cuuint32_t obox[4] = {2 * kCo, kWp, 1, 1};
    FVV_TRY(tc_encode_map(&mc, 4, out, odims, ostrides, obox, 64));
    const int grid = (int)(tiles < sms ? tiles : sms);
    convt_fold_kernel<<<grid, kThreads, kSmem, st>>>(ma, *(const CUtensorMap *)h->tc[li].map_k, mc, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

} // namespace fvv
