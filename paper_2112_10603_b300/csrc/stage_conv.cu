// VIBlock s > 0: the stage input (a3) computed inside the loader of the block's first conv.
//
// Sec. 3.1 / Fig. 3: the input of VIBlock s is [I_l, I_r, I_l warped, I_r warped, up(M),
// up(F) x 2, t] on the stage grid, built from the previous stage's flows and mask (the
// same quantities and order as the standalone stage-input kernel); its only consumer is
// the block's first layer c0 (Table 3: 3x3, stride 2, 18 -> 128, ReLU).  Here loader warps
// compute that input pixel by pixel straight into the tensor-core operand tiles of c0, so
// it never exists in HBM.
//
// Work: one persistent CTA per SM owns a contiguous range of row tiles in (view, column
// strip, output row) order: a tile is output row y, pixels x0 .. x0 + 125 of a 126-pixel
// strip.  Output row y reads input rows 2y - 1, 2y, 2y + 1; walking down a strip, row
// 2y - 1 is the previous tile's row 2y + 1, so each input row is computed once (plus one
// row where a CTA's range enters a strip).
//
// Row slot (one input row of one strip, the operand layout of the stride-2 pair view):
// 129 rows of 128 bytes, row r = the input pixels 2 (x0 - 1 + r) and 2 (x0 - 1 + r) + 1,
// 32 bf16 channels each (the 18 stage channels, then zeros), 16-byte chunks swizzled in
// 128-byte mode.  Output pixel j reads pixels 2 (x0 + j) + kx - 1: for kx = 1 / 2 the
// even / odd pixel of slot row j + 1, for kx = 0 the odd pixel of row j, so the three
// column taps of a row tap are three descriptors into one slot (no copy per tap).
//
// Warps: 0 loads the resident weights (TMA), 1 allocates TMEM and issues the MMAs, 2-5 are
// the epilogue (TMEM lane quarters), 6 .. 6 + 8 NG - 1 are NG loader groups of 8 warps;
// group g computes the new input rows of the CTA's tiles g, g + NG, ... (one pixel per
// thread and row) into a ring of row slots.
#include <cuda.h>
#include <cuda_fp8.h>

#include <cstring>

#include "interp.h"
#include "sampling.h"
#include "tc_ptx.h"
#include "tc_wait.h"

namespace fvv {

// (csrc/conv_tc.cu) bf16 tensor map, rows of ck_bytes swizzled accordingly
int tc_encode_map(CUtensorMap *m, int rank, void *base, const cuuint64_t *dims, const cuuint64_t *strides_bytes,
                  const cuuint32_t *box, int ck_bytes);

namespace {

constexpr int kSt = 126;                                       // output pixels per tile
constexpr int kNeed = 2 * kSt + 1;                              // slot pixels 1 .. 253 feed them
constexpr uint32_t kSlotBytes = ((129 * 128 + 1023) / 1024) * 1024;
constexpr int kSlots = 7;
constexpr int kCo = 128;                                        // output channels (the N tile)
constexpr uint32_t kTapBytes = kCo * 64;                        // one tap's weights: 128 x 32 bf16
constexpr uint32_t kStgBytes = 32 * kCo * 2;                    // epilogue staging per warp
constexpr uint32_t kIdesc = ptx::make_idesc(128, kCo, 1, 1);

struct __align__(16) ScBars {
    uint64_t wfull;
    uint64_t full[kSlots], empty[kSlots];
    uint64_t tmem_full[2], tmem_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

template <int NG> struct ScCfg {
    static constexpr int kThreads = 32 * (6 + 8 * NG);
    static constexpr size_t kSmem =
        9 * kTapBytes + kSlots * kSlotBytes + 4 * kStgBytes + sizeof(ScBars) + kCo * 4 + 1024;
    static_assert(kSmem <= 227 * 1024, "stage conv shared memory");
};

struct ScParams {
    // stage input
    const float4 *imgs;    // frame level of the stage grid, one float4 per pixel, per camera
    const float *fm_prev;  // previous stage F, M: (h / 2) x (w / 2) x 5 per view
    const int *cam_l, *cam_r;
    const float *t;
    const int *n_dev;      // device view count (size-bucket graphs), or NULL
    int n_img;
    int h, w, circ;        // stage grid, padding mode
    // c0
    int ho, wo, strips;    // output grid; column strips of kSt pixels
    const float *bias;
    void *out;             // ho x wo x 128 per view: bf16, or E4M3 codes (out_fp8)
    int out_fp8;
    float out_q;           // E4M3: 1 / activation scale of the consumer
    float *amax;           // calibration: running max |output|, or NULL
    int *err;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

// The 18 stage-input channels of pixel (X, Y[r]) of view v, for NR rows at once (their
// gathers in flight together), as three 16-byte chunks of bf16 each (channels 0-7, 8-15,
// 16-23; 18-23 are zero): the standalone stage-input kernel's arithmetic.  The
// coordinates must lie in the grid.
template <bool CIRC, int NR>
__device__ __forceinline__ void stage_pixels(const ScParams &p, int v, int X, const int (&Y)[NR], uint4 (&c)[NR][3]) {
    const int h = p.h, w = p.w;
    const int P = h * w;
    const float *fm = p.fm_prev + (size_t)v * (P / 4) * 5;
    const float4 *L = p.imgs + (size_t)__ldg(p.cam_l + v) * P;
    const float4 *R = p.imgs + (size_t)__ldg(p.cam_r + v) * P;
    const float tv = __ldg(p.t + v);
    float up[NR][5];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        // x2 upsampling of the previous stage's F, M: the four taps' 5 channels each
        const Taps u = up_taps_t<CIRC>(X, Y[r], h / 2, w / 2);
        const float *a = fm + u.o00 * 5, *b = fm + u.o01 * 5, *d = fm + u.o10 * 5, *e = fm + u.o11 * 5;
#pragma unroll
        for (int k = 0; k < 5; ++k)
            up[r][k] = (1.f - u.ly) * ((1.f - u.lx) * __ldg(a + k) + u.lx * __ldg(b + k)) +
                       u.ly * ((1.f - u.lx) * __ldg(d + k) + u.lx * __ldg(e + k));
#pragma unroll
        for (int k = 0; k < 4; ++k) up[r][k] *= 2.f;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int pix = Y[r] * w + X;
        const Taps tl = warp_taps_t<CIRC>(X, Y[r], up[r][0], up[r][1], h, w);
        const Taps tr = warp_taps_t<CIRC>(X, Y[r], up[r][2], up[r][3], h, w);
        const float4 lc = __ldg(L + pix), rc = __ldg(R + pix);
        const float3 wl = bilerp_rgb(L, tl), wr = bilerp_rgb(R, tr);
        c[r][0] = make_uint4(pack_bf16x2(lc.x, lc.y), pack_bf16x2(lc.z, rc.x), pack_bf16x2(rc.y, rc.z),
                             pack_bf16x2(wl.x, wl.y));
        c[r][1] = make_uint4(pack_bf16x2(wl.z, wr.x), pack_bf16x2(wr.y, wr.z), pack_bf16x2(up[r][4], up[r][0]),
                             pack_bf16x2(up[r][1], up[r][2]));
        c[r][2] = make_uint4(pack_bf16x2(up[r][3], tv), 0u, 0u, 0u);
    }
}

// Walk over a CTA's contiguous tile range in (view, strip, row) order, without divisions
// after the first tile.  cont: the tile continues the previous one down its strip (its
// input row 2y - 1 is the previous tile's row 2y + 1).
struct TileWalk {
    int n, strip, y, ho, strips;
    bool cont;
    __device__ TileWalk(int t, int ho_, int strips_) : ho(ho_), strips(strips_), cont(false) {
        const int per_view = ho * strips;
        n = t / per_view;
        const int r = t - n * per_view;
        strip = r / ho;
        y = r - strip * ho;
    }
    __device__ void next() {
        cont = true;
        if (++y == ho) { y = 0; cont = false; if (++strip == strips) { strip = 0; ++n; } }
    }
};
// Position in the ring of row slots: slot and the parity of its current phase.
struct Ring {
    int slot = 0;
    uint32_t par = 0;
    __device__ void step() { if (++slot == kSlots) { slot = 0; par ^= 1; } }
};

// Bounded wait of a whole warp: lane 0 waits, every lane gets the same answer (so that the
// warp leaves its loop together when the CTA aborts).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *err, int code) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = wait_bar(bar, parity, abort, err, code);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

template <int NG, bool CIRC>
__global__ void __launch_bounds__(ScCfg<NG>::kThreads, 1)
stage_conv_kernel(const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmC32,
                  const __grid_constant__ CUtensorMap tmC30, const ScParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = smem;
    uint8_t *sSlot = sB + 9 * kTapBytes;
    uint8_t *sStg = sSlot + kSlots * kSlotBytes;
    ScBars *bars = (ScBars *)(sStg + 4 * kStgBytes);
    float *sBias = (float *)(bars + 1); // c0's 128 biases (16-byte aligned: ScBars is a multiple of 16)
    volatile int *abort = &bars->abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        ptx::mbar_init(ptx::smem_u32(&bars->wfull), 1);
        for (int s = 0; s < kSlots; ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->full[s]), 8); // one arrive per warp of a loader group
            ptx::mbar_init(ptx::smem_u32(&bars->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_full[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_empty[a]), 4); // one arrive per epilogue warp
        }
        ptx::mbar_init(ptx::smem_u32(&bars->drain), 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(&bars->tmem_base), 2 * kCo); // two accumulators
        ptx::tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        ptx::prefetch_tmap(&tmB);
        ptx::prefetch_tmap(&tmC32);
        ptx::prefetch_tmap(&tmC30);
    }
    if (threadIdx.x >= 64 && threadIdx.x < 64 + kCo) sBias[threadIdx.x - 64] = __ldg(p.bias + threadIdx.x - 64);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;

    // this CTA's contiguous range of row tiles, (view, strip, row) order
    const int n_img = p.n_dev ? min(__ldg(p.n_dev), p.n_img) : p.n_img;
    const int per_view = p.strips * p.ho;
    const int num_tiles = n_img * per_view;
    const int per_cta = (num_tiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_begin = min(num_tiles, (int)blockIdx.x * per_cta), t_end = min(num_tiles, t_begin + per_cta);

    if (warp == 0) {
        // ---------------- resident weights ----------------
        if (lane == 0) {
            const uint32_t fw = ptx::smem_u32(&bars->wfull);
            ptx::mbar_arrive_expect_tx(fw, 9 * kTapBytes);
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) // taps 3 ky .. 3 ky + 2 per box
                ptx::tma_load_3d(ptx::smem_u32(sB) + ky * 3 * kTapBytes, &tmB, fw, 0, 0, ky * 3);
            drain_wait(fw, 0); // landed before the CTA can exit
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            bool ok = wait_bar(ptx::smem_u32(&bars->wfull), 0, abort, p.err, 3);
            ptx::tc_fence_after();
            const uint32_t bw = ptx::smem_u32(sB), sw = ptx::smem_u32(sSlot);
            int acc = 0;
            uint32_t acc_phase = 0;
            Ring ring;                  // the next input row's slot
            int rs[3] = {0, 0, 0};
            uint32_t rp[3] = {0, 0, 0}; // slot and phase parity of rows 2y - 1, 2y, 2y + 1
            bool issued_any = false;
            TileWalk tw(t_begin, p.ho, p.strips);
            for (int t = t_begin; ok && t < t_end && !*abort; ++t, tw.next()) {
                const bool c = tw.cont;
                if (c) { rs[0] = rs[2]; rp[0] = rp[2]; }
                for (int r = c ? 1 : 0; r < 3; ++r) {
                    rs[r] = ring.slot;
                    rp[r] = ring.par;
                    ring.step();
                }
                if (!wait_bar(ptx::smem_u32(&bars->tmem_empty[acc]), acc_phase ^ 1, abort, p.err, 2)) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem + acc * kCo;
                for (int ky = 0; ky < 3; ++ky) {
                    if (!wait_bar(ptx::smem_u32(&bars->full[rs[ky]]), rp[ky], abort, p.err, 3)) { ok = false; break; }
                    ptx::tc_fence_after();
                    const uint32_t a0 = sw + rs[ky] * kSlotBytes;
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
                        const uint32_t b0 = bw + (ky * 3 + kx) * kTapBytes;
                        const uint32_t ak = a0 + (kx == 0 ? 0u : 128u) + (kx == 1 ? 0u : 64u);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t bd = ptx::smem_desc(b0 + kk * 32, 64);
                            const uint64_t ad = ptx::smem_desc(ak + kk * 32, 128);
                            ptx::mma_bf16(d, ad, bd, kIdesc, (ky | kx | kk) != 0);
                        }
                    }
                }
                if (!ok) break;
                issued_any = true;
                ptx::mma_commit(ptx::smem_u32(&bars->tmem_full[acc]));
                // free the rows no later tile reads (row 2y + 1 stays when the next tile continues)
                ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[0]]));
                ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[1]]));
                if (!(t + 1 < t_end && tw.y + 1 < p.ho)) ptx::mma_commit(ptx::smem_u32(&bars->empty[rs[2]]));
                if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            }
            // every MMA and barrier arrival issued above has completed before TMEM and the
            // shared memory go away
            if (issued_any) {
                ptx::mma_commit(ptx::smem_u32(&bars->drain));
                drain_wait(ptx::smem_u32(&bars->drain), 0);
            }
        }
    } else if (warp < 6) {
        // ---------------- epilogue: bias, ReLU, bf16 / E4M3, TMA row stores ----------------
        // The warp's 32 pixels are staged as 128-byte rows in the tensor maps' 128-byte
        // swizzle (bf16: two 4 KB boxes, channels 0-63 and 64-127; E4M3: one box) and one
        // lane stores them with TMA: tmC32 stores 32 pixels, tmC30 the last warp's 30 (the
        // tile's pixels 126, 127 are the next strip's); the map clips the grid's right edge.
        const int q = warp & 3; // TMEM lanes 32 q .. 32 q + 31 = tile pixels
        const uint32_t stg_s = ptx::smem_u32(sStg + q * kStgBytes);
        const CUtensorMap *tmC = q == 3 ? &tmC30 : &tmC32;
        int acc = 0;
        uint32_t acc_phase = 0;
        float vmax = 0.f;
        TileWalk tw(t_begin, p.ho, p.strips);
        for (int t = t_begin; t < t_end; ++t, tw.next()) {
            const int n = tw.n, y = tw.y, x0 = tw.strip * kSt;
            const int nvalid = min(kSt, p.wo - x0);
            const bool valid = q * 32 + lane < nvalid;
            if (!warp_wait(ptx::smem_u32(&bars->tmem_full[acc]), acc_phase, abort, p.err, 4)) break;
            ptx::tc_fence_after();
            // the previous tile's store has read the staging buffer
            if (lane == 0) ptx::bulk_wait_read<0>();
            __syncwarp();
            const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + acc * kCo;
#pragma unroll 1
            for (int c = 0; c < kCo; c += 32) {
                // two accumulator loads in flight per wait
                uint32_t rr[2][16];
                __syncwarp();
                ptx::tmem_ld16(tb + c, rr[0]);
                ptx::tmem_ld16(tb + c + 16, rr[1]);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int hb = 0; hb < 2; ++hb) {
                    const int cb = c + 16 * hb;
                    float v[16];
#pragma unroll
                    for (int j4 = 0; j4 < 16; j4 += 4) {
                        const float4 b = *reinterpret_cast<const float4 *>(sBias + cb + j4);
                        v[j4] = fmaxf(__uint_as_float(rr[hb][j4]) + b.x, 0.f); // c0 has ReLU
                        v[j4 + 1] = fmaxf(__uint_as_float(rr[hb][j4 + 1]) + b.y, 0.f);
                        v[j4 + 2] = fmaxf(__uint_as_float(rr[hb][j4 + 2]) + b.z, 0.f);
                        v[j4 + 3] = fmaxf(__uint_as_float(rr[hb][j4 + 3]) + b.w, 0.f);
                    }
                    if (p.amax && valid) { // calibration only
#pragma unroll
                        for (int j = 0; j < 16; ++j) vmax = fmaxf(vmax, v[j]);
                    }
                    if (p.out_fp8) {
                        // E4M3 codes of v x out_q, value j in byte j (paired conversions)
                        uint32_t w[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t lo = __nv_cvt_float2_to_fp8x2(
                                make_float2(v[4 * k] * p.out_q, v[4 * k + 1] * p.out_q), __NV_SATFINITE, __NV_E4M3);
                            const uint32_t hi = __nv_cvt_float2_to_fp8x2(
                                make_float2(v[4 * k + 2] * p.out_q, v[4 * k + 3] * p.out_q), __NV_SATFINITE, __NV_E4M3);
                            w[k] = lo | (hi << 16);
                        }
                        ptx::st_shared_v4(stg_s + lane * 128 + (((cb >> 4) ^ (lane & 7)) << 4),
                                          make_uint4(w[0], w[1], w[2], w[3]));
                    } else {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const uint4 u = make_uint4(
                                pack_bf16x2(v[8 * hh], v[8 * hh + 1]), pack_bf16x2(v[8 * hh + 2], v[8 * hh + 3]),
                                pack_bf16x2(v[8 * hh + 4], v[8 * hh + 5]), pack_bf16x2(v[8 * hh + 6], v[8 * hh + 7]));
                            const int ck = (cb >> 3) + hh; // 16-byte chunk 0..15 of the pixel's 256 bytes
                            ptx::st_shared_v4(stg_s + (ck >> 3) * 4096 + lane * 128 + (((ck & 7) ^ (lane & 7)) << 4), u);
                        }
                    }
                }
            }
            // the accumulator is free once read
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->tmem_empty[acc]));
            if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            // generic-proxy staging writes, read by the TMA store (async proxy)
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0 && q * 32 < nvalid) {
                const int xs = x0 + q * 32;
                ptx::tma_store_4d(tmC, stg_s, 0, xs, y, n);
                if (!p.out_fp8) ptx::tma_store_4d(tmC, stg_s + 4096, 64, xs, y, n);
                ptx::bulk_commit();
            }
        }
        if (lane == 0) ptx::bulk_wait<0>(); // the stores have completed before the CTA exits
        if (p.amax && vmax > 0.f) atomicMax(reinterpret_cast<int *>(p.amax), __float_as_int(vmax));
    } else {
        // ---------------- loaders: the stage input, one pixel per thread and row ----------------
        // group g computes the new input rows of the CTA's tiles g, g + NG, ...: the two rows
        // of a continuing tile together (their gathers in flight at once), plus row 2y - 1
        // where a tile starts a strip segment
        // Warp w of a group covers slot pixels 32 w .. 32 w + 31; lane l takes pair row
        // 16 w + (l & 7) + 8 (l >> 4), pixel (l >> 3) & 1 of the pair, so that the 8 lanes of
        // each quarter-warp store phase write 8 consecutive pair rows: 8 distinct 16-byte
        // chunks of the 128-byte swizzle, no bank conflicts (consecutive pixels per lane
        // put two rows 4 apart on the same chunk).  Pixels 1 .. 253 feed the tile.
        const int g = (warp - 6) / 8, w8 = (warp - 6) % 8;
        const int pr = 16 * w8 + (lane & 7) + 8 * (lane >> 4), half = (lane >> 3) & 1; // slot row, pixel of its pair
        const int i = 2 * pr + half;        // slot pixel of this thread
        const uint32_t slot0 = ptx::smem_u32(sSlot) + pr * 128;
        bool stop = false;
        auto put = [&](int slot, const uint4 (&cv)[3], bool inside) {
            const uint32_t row = slot0 + (uint32_t)slot * kSlotBytes;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
                ptx::st_shared_v4(row + (((half * 4 + cc) ^ (pr & 7)) << 4),
                                  inside && cc < 3 ? cv[cc] : make_uint4(0, 0, 0, 0));
        };
        Ring ring; // the next input row's slot
        TileWalk tw(t_begin, p.ho, p.strips);
        for (int t = t_begin, tl = 0; t < t_end && !stop; ++t, ++tl, tw.next()) {
            const int nr = tw.cont ? 2 : 3;
            Ring rg[3]; // slots of this tile's new rows
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                rg[j] = ring;
                if (j < nr) ring.step();
            }
            if (tl % NG != g) continue;
            const int n = tw.n, y = tw.y, x0 = tw.strip * kSt;
            for (int j = 0; j < nr && !stop; ++j)
                stop = !warp_wait(ptx::smem_u32(&bars->empty[rg[j].slot]), rg[j].par ^ 1u, abort, p.err, 1);
            if (stop) break;
            if (i >= 1 && i <= kNeed) {
                // rows Y = 2y + rr - 1 for rr = 3 - nr .. 2; outside the grid: zeros (zero
                // padding) computed from clamped coordinates, or wrapped (circular)
                const int X0 = 2 * x0 - 2 + i;
                const bool xin = CIRC || (X0 >= 0 && X0 < p.w);
                const int X = fix_index_t<CIRC>(X0, p.w);
                int Y[2];
                bool yin[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int Y0 = 2 * y + (nr == 3 ? j : j + 1) - 1;
                    yin[j] = CIRC || (Y0 >= 0 && Y0 < p.h);
                    Y[j] = fix_index_t<CIRC>(Y0, p.h);
                }
                uint4 cv[2][3];
                stage_pixels<CIRC, 2>(p, n, X, Y, cv);
                put(rg[0].slot, cv[0], xin && yin[0]);
                put(rg[1].slot, cv[1], xin && yin[1]);
                if (nr == 3) {
                    const int Y0 = 2 * y + 1;
                    const int Y1[1] = {fix_index_t<CIRC>(Y0, p.h)};
                    uint4 c1[1][3];
                    stage_pixels<CIRC, 1>(p, n, X, Y1, c1);
                    put(rg[2].slot, c1[0], xin && (CIRC || Y0 < p.h));
                }
            }
            // generic-proxy writes, read by the tensor cores (async proxy)
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0)
                for (int j = 0; j < nr; ++j) ptx::mbar_arrive(ptx::smem_u32(&bars->full[rg[j].slot]));
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 2 * kCo);
    }
}

constexpr int kGroups = 2;

} // namespace

bool stage_conv_layer(const fvv_interp *h, int li) {
    const LayerDef &L = kLayers[li];
    return (li == kVib1 || li == kVib2) && L.kind == K_CONV && L.stride == 2 && L.ci == 18 && L.co == kCo &&
           h->tc[li].ci_pad == 32 && h->tc[li].co_pad == kCo;
}

int tc_stage_conv(fvv_interp *h, int li, const float4 *imgs, const float *fm_prev, const ViewTab &vt, int nv, int hs,
                  int ws, int circ, void *out, int out_cs, cudaStream_t st) {
    const LayerDef &L = kLayers[li];
    if (!stage_conv_layer(h, li) || hs % 2 || ws % 2 || out_cs != kCo || ((uintptr_t)out % 16) != 0) {
        set_error("layer %s: not a fusable stage-input conv", L.name);
        return FVV_EINVAL;
    }
    const bool f8_on = h->o.precision == FVV_FP8 && h->fp8_ready && !h->calibrating;
    ScParams p{};
    p.imgs = imgs;
    p.fm_prev = fm_prev;
    p.cam_l = vt.cam_l;
    p.cam_r = vt.cam_r;
    p.t = vt.t;
    p.n_dev = vt.n;
    p.n_img = nv;
    p.h = hs; p.w = ws; p.circ = circ;
    p.ho = hs / 2; p.wo = ws / 2;
    p.strips = (p.wo + kSt - 1) / kSt;
    p.bias = h->bias + h->b_off[li];
    p.out = out;
    p.out_fp8 = f8_on && feeds_fp8(li) ? 1 : 0;
    p.out_q = h->q_out[li];
    p.amax = h->calibrating && feeds_fp8(li) ? h->d_amax + li : nullptr;
    p.err = h->d_err;
    const long long tiles = (long long)nv * p.strips * p.ho;
    if (tiles <= 0) return FVV_OK;
    if (tiles > (1ll << 30)) { set_error("too many tiles"); return FVV_ESHAPE; }
    using C = ScCfg<kGroups>;
    auto kern = circ ? stage_conv_kernel<kGroups, true> : stage_conv_kernel<kGroups, false>;
    static int sms = 0;
    if (!sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FVV_CHECK_CUDA(cudaFuncSetAttribute(stage_conv_kernel<kGroups, false>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem));
        FVV_CHECK_CUDA(cudaFuncSetAttribute(stage_conv_kernel<kGroups, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem));
    }
    // output maps: n x ho x wo pixels of 128 channels; E4M3 codes are described as 64
    // two-byte elements per pixel (a store moves bytes), so both precisions use 128-byte
    // box rows in the 128-byte swizzle
    const cuuint64_t pxb = p.out_fp8 ? 128 : 256;
    cuuint64_t dims[4] = {pxb / 2, (cuuint64_t)p.wo, (cuuint64_t)p.ho, (cuuint64_t)nv};
    cuuint64_t strides[3] = {pxb, (cuuint64_t)p.wo * pxb, (cuuint64_t)p.ho * p.wo * pxb};
    cuuint32_t box32[4] = {64, 32, 1, 1}, box30[4] = {64, kSt - 96, 1, 1};
    CUtensorMap mc32, mc30;
    FVV_TRY(tc_encode_map(&mc32, 4, out, dims, strides, box32, 128));
    FVV_TRY(tc_encode_map(&mc30, 4, out, dims, strides, box30, 128));
    const int grid = (int)(tiles < sms ? tiles : sms);
    kern<<<grid, C::kThreads, C::kSmem, st>>>(*(const CUtensorMap *)h->tc[li].map3, mc32, mc30, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

} // namespace fvv
