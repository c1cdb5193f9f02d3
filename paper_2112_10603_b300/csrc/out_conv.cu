// RefineNet's output conv with the network output fused (Sec. 3.1; Table 3: 3x3, 16 -> 3,
// then the residual output clamp(I_blend + 2 sigmoid(z) - 1, 0, 1) on the cropped grid).
//
// The layer's MMAs are tiny (N = 3 outputs), so the tensor pipe's per-instruction cost,
// not its FLOPs, sets the pace: the column taps are folded into N.  One MMA per row tap
// ky computes, for every input pixel i of the row, the 9 columns (kx, co) = W[ky][kx][co]
// . in(i); output pixel i then sums column (0, co) of pixel i - 1, (1, co) of i and
// (2, co) of i + 1 (neighbouring TMEM lanes: warp shuffles).  3 MMAs per output row
// instead of 9.
//
// Work: persistent CTAs, several per SM.  A tile is two output rows (2 y2, 2 y2 + 1) of a
// 120-pixel column strip; a CTA owns a contiguous range of tiles in (view, strip, row
// pair) order, so walking down a strip a tile loads only the two input rows it adds
// (2 y2 + 1, 2 y2 + 2).  Only rows of the crop are computed.
//
// Row slot: one input row, 128 rows of 32 bytes (16 bf16 channels): accumulator lane
// 32 q + l is input pixel x0 - 1 + 30 q + l, so epilogue warp q owns 32 pixels of which
// lanes 1..30 produce outputs x0 + 30 q .. x0 + 30 q + 29 (lanes 0 and 31 are its halo);
// four 32-pixel TMA boxes per row (32-byte swizzle; zeros outside the grid = the conv's
// zero padding).  Weights: the three folded row-tap slices, 16 rows (9 used) x 16
// channels, resident.  Accumulators: per tile two 128 x 16 (one per output row), two
// tiles in TMEM.  I_blend: the producer bulk-copies each tile's two 120-pixel rows into a
// ring of shared-memory slots, ahead of the epilogue.
//
// Warps: 0 issues the copies (weights once; rows and I_blend per tile), 1 allocates TMEM
// and issues the MMAs, 2-5 are the epilogue (TMEM lane quarters): tap sums, bias,
// sigmoid, residual, clamp; a warp's 30 pixels of a row (360 contiguous bytes of the
// output) are staged in shared memory and stored as 8-byte vectors.
#include <cuda.h>

#include "interp.h"
#include "tc_ptx.h"
#include "tc_wait.h"

namespace fvv {

// (csrc/conv_tc.cu) bf16 tensor map, rows of ck_bytes swizzled accordingly
int tc_encode_map(CUtensorMap *m, int rank, void *base, const cuuint64_t *dims, const cuuint64_t *strides_bytes,
                  const cuuint32_t *box, int ck_bytes);

namespace {

constexpr int kTw = 120;                                   // strip width (output pixels)
constexpr int kWp = 30;                                    // outputs per epilogue warp
constexpr uint32_t kRowBytes = 32;                         // 16 bf16 channels
constexpr uint32_t kSlotBytes = 128 * kRowBytes;           // 4096: one input row (4 boxes)
constexpr uint32_t kBoxBytes = 32 * kRowBytes;             // 1024: one 32-pixel box
constexpr int kSlots = 12;                                 // rows: the producer runs 5 tiles ahead
constexpr int kIbSlots = 4;                                // I_blend ring (tiles)
constexpr uint32_t kIbRow = kTw * 12;                      // 1440 bytes: 120 pixels x 3 floats
constexpr uint32_t kTapBytes = 16 * kRowBytes;             // one folded slice: 16 x 16 bf16
constexpr int kCtas = 3;                                   // CTAs per SM
constexpr int kThreads = 192;
constexpr uint32_t kIdesc = ptx::make_idesc(128, 16, 1, 1);
constexpr uint32_t kStgBytes = 2 * kWp * 12;               // per epilogue warp: 2 rows x 30 px x 3 floats

struct __align__(16) OcBars {
    uint64_t wfull;
    uint64_t full[kSlots], empty[kSlots];
    uint64_t ib_full[kIbSlots], ib_empty[kIbSlots];
    uint64_t tmem_full[2], tmem_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

// weights 1536 (+ 512 to the next 1 KB), row slots, I_blend ring, staging, barriers
constexpr uint32_t kOffSlot = 2048;
constexpr uint32_t kOffIb = kOffSlot + kSlots * kSlotBytes;
constexpr uint32_t kOffStg = kOffIb + kIbSlots * 2 * kIbRow;
constexpr uint32_t kOffBars = kOffStg + 4 * kStgBytes;
constexpr size_t kSmem = kOffBars + sizeof(OcBars) + 1024;
static_assert(kCtas * (kSmem + 1024) <= 227 * 1024, "output conv shared memory");
static_assert(kOffIb % 16 == 0 && kOffStg % 16 == 0 && kOffBars % 16 == 0, "output conv layout");

struct OcParams {
    const float *bias;                // 3 output biases
    const float *ib;                  // I_blend, n x hp x wp x 3 (padded grid)
    float *const *out_ref;            // device slot: the cropped n x crop_h x crop_w x 3 output
    const int *n_dev;                 // device view count (size-bucket graphs), or NULL
    int n_img, hp, wp, crop_h, crop_w;
    int strips, pairs;                // column strips and row pairs per view
    int *err;
};

// Contiguous walk over (view, strip, row pair) without divisions after the first tile.
struct OcWalk {
    int n, strip, y2, pairs, strips;
    bool cont;
    __device__ OcWalk(int t, int pairs_, int strips_) : pairs(pairs_), strips(strips_), cont(false) {
        const int per_view = pairs * strips;
        n = t / per_view;
        const int r = t - n * per_view;
        strip = r / pairs;
        y2 = r - strip * pairs;
    }
    __device__ void next() {
        cont = true;
        if (++y2 == pairs) { y2 = 0; cont = false; if (++strip == strips) { strip = 0; ++n; } }
    }
};
template <int S> struct OcRing {
    int slot = 0;
    uint32_t par = 0;
    __device__ void step() { if (++slot == S) { slot = 0; par ^= 1; } }
};

__global__ void __launch_bounds__(kThreads, kCtas)
out_conv_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const OcParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = smem;
    uint8_t *sSlot = smem + kOffSlot;
    uint8_t *sIb = smem + kOffIb;
    uint8_t *sStg = smem + kOffStg;
    OcBars *bars = (OcBars *)(smem + kOffBars);
    volatile int *abort = &bars->abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        ptx::mbar_init(ptx::smem_u32(&bars->wfull), 1);
        for (int s = 0; s < kSlots; ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->empty[s]), 1);
        }
        for (int s = 0; s < kIbSlots; ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->ib_full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->ib_empty[s]), 4); // one arrive per epilogue warp
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_full[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_empty[a]), 4);
        }
        ptx::mbar_init(ptx::smem_u32(&bars->drain), 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(&bars->tmem_base), 64); // 2 tiles x 2 rows x 16 columns
        ptx::tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;

    const int n_img = p.n_dev ? min(__ldg(p.n_dev), p.n_img) : p.n_img;
    const int per_view = p.strips * p.pairs;
    const int num_tiles = n_img * per_view;
    const int per_cta = (num_tiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_begin = min(num_tiles, (int)blockIdx.x * per_cta), t_end = min(num_tiles, t_begin + per_cta);

    if (warp == 0) {
        // ---------------- copy producer ----------------
        if (lane == 0) {
            const uint32_t fw = ptx::smem_u32(&bars->wfull);
            ptx::mbar_arrive_expect_tx(fw, 3 * kTapBytes);
            ptx::tma_load_3d(ptx::smem_u32(sB), &tmB, fw, 0, 0, 0); // the three folded slices
            OcRing<kSlots> ring;
            OcRing<kIbSlots> ibr;
            long long issued = 0, ib_issued = 0;
            OcWalk tw(t_begin, p.pairs, p.strips);
            bool stop = false;
            for (int t = t_begin; t < t_end && !stop && !*abort; ++t, tw.next()) {
                const int x0 = tw.strip * kTw;
                // this tile's I_blend rows (16-byte aligned: x0 and wp are multiples of 4)
                if (!wait_bar(ptx::smem_u32(&bars->ib_empty[ibr.slot]), ibr.par ^ 1u, abort, p.err, 1)) break;
                {
                    const uint32_t fi = ptx::smem_u32(&bars->ib_full[ibr.slot]);
                    const uint32_t bytes = (uint32_t)min(kTw, p.wp - x0) * 12u;
                    const int y1 = min(2 * tw.y2 + 1, p.hp - 1); // (a second row past the grid: a copy, unused)
                    ptx::mbar_arrive_expect_tx(fi, 2 * bytes);
                    const uint32_t dst = ptx::smem_u32(sIb) + ibr.slot * 2 * kIbRow;
                    ptx::bulk_load(dst, p.ib + (((size_t)tw.n * p.hp + 2 * tw.y2) * p.wp + x0) * 3, bytes, fi);
                    ptx::bulk_load(dst + kIbRow, p.ib + (((size_t)tw.n * p.hp + y1) * p.wp + x0) * 3, bytes, fi);
                    ++ib_issued;
                    ibr.step();
                }
                // new input rows: 2 y2 + 1, 2 y2 + 2, and 2 y2 - 1, 2 y2 where a segment starts
                for (int j = tw.cont ? 2 : 0; j < 4; ++j) {
                    if (!wait_bar(ptx::smem_u32(&bars->empty[ring.slot]), ring.par ^ 1u, abort, p.err, 1)) {
                        stop = true;
                        break;
                    }
                    const uint32_t fs = ptx::smem_u32(&bars->full[ring.slot]);
                    ptx::mbar_arrive_expect_tx(fs, kSlotBytes);
                    const uint32_t dst = ptx::smem_u32(sSlot) + ring.slot * kSlotBytes;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        ptx::tma_load_4d(dst + q * kBoxBytes, &tmA, fs, 0, x0 - 1 + kWp * q, 2 * tw.y2 - 1 + j, tw.n);
                    ++issued;
                    ring.step();
                }
            }
            // every copy issued has landed before the CTA can exit (the other roles may
            // have stopped waiting for them): the last ring positions of both rings
            for (long long k = 1; k <= issued && k <= kSlots; ++k) {
                const long long q = issued - k;
                drain_wait(ptx::smem_u32(&bars->full[q % kSlots]), (uint32_t)((q / kSlots) & 1));
            }
            for (long long k = 1; k <= ib_issued && k <= kIbSlots; ++k) {
                const long long q = ib_issued - k;
                drain_wait(ptx::smem_u32(&bars->ib_full[q % kIbSlots]), (uint32_t)((q / kIbSlots) & 1));
            }
            drain_wait(fw, 0);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            bool ok = wait_bar(ptx::smem_u32(&bars->wfull), 0, abort, p.err, 3);
            ptx::tc_fence_after();
            const uint32_t bw = ptx::smem_u32(sB), sw = ptx::smem_u32(sSlot);
            int acc = 0;
            uint32_t acc_phase = 0;
            OcRing<kSlots> ring;
            int rs[4] = {0, 0, 0, 0};
            uint32_t rp[4] = {0, 0, 0, 0}; // slot and phase parity of input rows 2 y2 - 1 .. 2 y2 + 2
            bool issued_any = false;
            OcWalk tw(t_begin, p.pairs, p.strips);
            for (int t = t_begin; ok && t < t_end && !*abort; ++t, tw.next()) {
                if (tw.cont) { rs[0] = rs[2]; rp[0] = rp[2]; rs[1] = rs[3]; rp[1] = rp[3]; }
                for (int r = tw.cont ? 2 : 0; r < 4; ++r) {
                    rs[r] = ring.slot;
                    rp[r] = ring.par;
                    ring.step();
                }
                if (!wait_bar(ptx::smem_u32(&bars->tmem_empty[acc]), acc_phase ^ 1, abort, p.err, 2)) break;
                ptx::tc_fence_after();
                for (int r = 0; r < 4 && ok; ++r)
                    ok = wait_bar(ptx::smem_u32(&bars->full[rs[r]]), rp[r], abort, p.err, 3);
                if (!ok) break;
                ptx::tc_fence_after();
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const uint32_t d = tmem + acc * 32 + r * 16;
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky) {
                        const uint64_t ad = ptx::smem_desc(sw + rs[r + ky] * kSlotBytes, kRowBytes);
                        const uint64_t bd = ptx::smem_desc(bw + ky * kTapBytes, kRowBytes);
                        ptx::mma_bf16(d, ad, bd, kIdesc, ky != 0);
                    }
                }
                issued_any = true;
                ptx::mma_commit(ptx::smem_u32(&bars->tmem_full[acc]));
                // rows 2 y2 - 1, 2 y2 are done; 2 y2 + 1, 2 y2 + 2 stay when the next tile continues
                ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[0]]));
                ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[1]]));
                if (!(t + 1 < t_end && tw.y2 + 1 < p.pairs)) {
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[2]]));
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[3]]));
                }
                if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            }
            if (issued_any) {
                ptx::mma_commit(ptx::smem_u32(&bars->drain));
                drain_wait(ptx::smem_u32(&bars->drain), 0);
            }
        }
    } else {
        // ---------------- epilogue: the network output of two rows x 30 pixels ----------------
        const int q = warp & 3;
        const uint32_t stg = ptx::smem_u32(sStg + q * kStgBytes);
        float *const out = *p.out_ref;
        const bool vec = (p.crop_w % 2) == 0 && ((uintptr_t)out & 7) == 0; // 8-byte aligned rows
        const float b0 = __ldg(p.bias), b1 = __ldg(p.bias + 1), b2 = __ldg(p.bias + 2);
        int acc = 0;
        uint32_t acc_phase = 0;
        OcRing<kIbSlots> ibr;
        OcWalk tw(t_begin, p.pairs, p.strips);
        for (int t = t_begin; t < t_end && !*abort; ++t, tw.next()) {
            const int xw = tw.strip * kTw + kWp * q; // the warp's first output pixel
            const int nw = min(kWp, p.crop_w - xw);  // its outputs inside the crop
            int ok = 1;
            if (lane == 0) ok = wait_bar(ptx::smem_u32(&bars->tmem_full[acc]), acc_phase, abort, p.err, 4);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            ptx::tc_fence_after();
            uint32_t ra[16], rb[16];
            const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + acc * 32;
            ptx::tmem_ld16(tb, ra);
            ptx::tmem_ld16(tb + 16, rb);
            ptx::tmem_ld_wait();
            // the accumulators are free once read
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->tmem_empty[acc]));
            if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            // tap sums: output of lane l (1..30) = column (0, co) of lane l - 1 + (1, co) of
            // lane l + (2, co) of lane l + 1
            float z[2][3];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const uint32_t *a = r == 0 ? ra : rb;
#pragma unroll
                for (int co = 0; co < 3; ++co) {
                    const float left = __shfl_up_sync(0xffffffffu, __uint_as_float(a[co]), 1);
                    const float right = __shfl_down_sync(0xffffffffu, __uint_as_float(a[6 + co]), 1);
                    z[r][co] = left + __uint_as_float(a[3 + co]) + right;
                }
            }
            if (lane == 0 && !wait_bar(ptx::smem_u32(&bars->ib_full[ibr.slot]), ibr.par, abort, p.err, 4)) ok = 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            const bool mine = lane >= 1 && lane <= nw;
            // (lane 0 never reads: its address is only formed)
            const uint32_t ibs = ptx::smem_u32(sIb) + ibr.slot * 2 * kIbRow + (uint32_t)(kWp * q + (mine ? lane - 1 : 0)) * 12u;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int Y = 2 * tw.y2 + r;
                if (Y >= p.crop_h || nw <= 0) break; // warp-uniform
                float o[3];
#pragma unroll
                for (int co = 0; co < 3; ++co) {
                    const float zz = z[r][co] + (co == 0 ? b0 : (co == 1 ? b1 : b2));
                    // (1 + e^-z >= 1: the fast reciprocal division is within 2 ulp;
                    // the fast exponential adds ~2^-21 relative, far inside BF16)
                    const float res = __fdividef(2.f, 1.f + __expf(-zz)) - 1.f;
                    const float ibv = mine ? ptx::lds_f32(ibs + r * kIbRow + co * 4) : 0.f;
                    o[co] = fminf(fmaxf(ibv + res, 0.f), 1.f);
                }
                float *dst = out + (((size_t)tw.n * p.crop_h + Y) * p.crop_w + xw) * 3;
                if (vec && nw == kWp) {
                    // 30 pixels x 12 bytes: staged, then stored as 45 8-byte vectors
                    const uint32_t srow = stg + r * (kWp * 12);
                    if (mine) {
#pragma unroll
                        for (int co = 0; co < 3; ++co)
                            asm volatile("st.shared.f32 [%0], %1;" ::"r"(srow + (lane - 1) * 12 + co * 4), "f"(o[co])
                                         : "memory");
                    }
                    __syncwarp();
#pragma unroll
                    for (int k = lane; k < kWp * 3 / 2; k += 32) {
                        float2 v;
                        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(srow + k * 8) : "memory");
                        reinterpret_cast<float2 *>(dst)[k] = v;
                    }
                    __syncwarp(); // the staging row is rewritten by the next tile
                } else if (mine) {
#pragma unroll
                    for (int co = 0; co < 3; ++co) dst[(lane - 1) * 3 + co] = o[co];
                }
            }
            // the I_blend slot is free once read
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->ib_empty[ibr.slot]));
            ibr.step();
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 64);
    }
}

} // namespace

bool out_conv_ok(const fvv_interp *h, int li, int in_cs, int N, int hp, int wp, int crop_h, int crop_w) {
    const LayerDef &L = kLayers[li];
    return li == kRef + 12 && L.kind == K_CONV && L.stride == 1 && L.ci == 16 && L.co == 3 && in_cs == 16 &&
           h->tc[li].ci_pad == 16 && h->tc[li].kxf_n == 16 && h->tc[li].wk && h->o.pad_mode == FVV_PAD_ZERO &&
           N >= 1 && hp >= 1 && wp >= 1 && wp % 4 == 0 && crop_h >= 1 && crop_w >= 1 && crop_h <= hp && crop_w <= wp;
}

int tc_out_conv(fvv_interp *h, int li, const void *in, int N, int hp, int wp, const float *ib,
                float *const *out_ref, int crop_h, int crop_w, const int *n_dev, cudaStream_t st) {
    if (!out_conv_ok(h, li, 16, N, hp, wp, crop_h, crop_w) || ((uintptr_t)in & 15) || !ib || ((uintptr_t)ib & 15) ||
        !out_ref) {
        set_error("layer %s: not the fusable output conv", kLayers[li].name);
        return FVV_EINVAL;
    }
    // the input: N x hp x wp pixels of 16 bf16 channels; boxes of one row x 32 pixels
    CUtensorMap ma;
    cuuint64_t dims[4] = {16, (cuuint64_t)wp, (cuuint64_t)hp, (cuuint64_t)N};
    cuuint64_t strides[3] = {32, (cuuint64_t)wp * 32, (cuuint64_t)hp * wp * 32};
    cuuint32_t box[4] = {16, 32, 1, 1};
    FVV_TRY(tc_encode_map(&ma, 4, (void *)in, dims, strides, box, 32));
    OcParams p{};
    p.bias = h->bias + h->b_off[li];
    p.ib = ib;
    p.out_ref = out_ref;
    p.n_dev = n_dev;
    p.n_img = N;
    p.hp = hp; p.wp = wp; p.crop_h = crop_h; p.crop_w = crop_w;
    p.strips = (crop_w + kTw - 1) / kTw;
    p.pairs = (crop_h + 1) / 2;
    p.err = h->d_err;
    const long long tiles = (long long)N * p.strips * p.pairs;
    if (tiles > (1ll << 30)) { set_error("too many tiles"); return FVV_ESHAPE; }
    static int sms = 0;
    if (!sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FVV_CHECK_CUDA(cudaFuncSetAttribute(out_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    }
    const long long slots = (long long)sms * kCtas;
    const int grid = (int)(tiles < slots ? tiles : slots);
    out_conv_kernel<<<grid, kThreads, kSmem, st>>>(ma, *(const CUtensorMap *)h->tc[li].map_k, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

} // namespace fvv
