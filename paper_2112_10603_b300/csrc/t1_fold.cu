// The last layer t1 of VIBlock s > 0 (Table 3: transposed conv 4x4, stride 2, 128 -> 5,
// no activation) with the Eq. 2 update fused: F^s, M^s = up(F^{s-1}, M^{s-1}) + Res^s,
// the x2 upsampling of F scaled by 2.
//
// As the generic folded-tap kernel: the transposed conv runs as one 3x3 conv over its
// input grid whose 4 x 5 output columns are the four output phases, with the three column
// taps folded into N (3 x 20 + 4 = 64; one MMA per (row tap ky, channel block, 16-channel
// step), 24 per row) and the taps summed across neighbouring TMEM lanes.  Unlike it,
// tiles walk down 120-pixel column strips, so each input row (and each row of F^{s-1}) is
// loaded once instead of once per row tap, and F^{s-1} reaches the epilogue through
// shared memory (bulk copies issued ahead by the producer) instead of per-lane global
// gathers; eight epilogue warps (two per TMEM lane quarter, one per output row parity)
// instead of four.  The MMAs, the tap sums and the Eq. 2 arithmetic are those of the
// generic kernel, in the same order: the same bits.
//
// Work: one persistent CTA per SM; a tile is input row y of a strip (input pixels x0 ..
// x0 + 119), a CTA owns a contiguous range of tiles in (view, strip, row) order.
// Input row slot: 2 channel blocks x 128 rows of 128 bytes (SW128): accumulator lane
// 32 q + l is input pixel x0 - 1 + 30 q + l, eight 32-pixel x 64-channel TMA boxes per row
// (zeros outside the grid).  F^{s-1} row slot: pixels max(0, x0 - 4) .. min(w, x0 + 124) - 1
// of the row (clamped into the grid, as the upsampling clamps), 20 bytes each, one bulk
// copy.  Weights: the folded slices, [channel block][ky][64 rows][64 channels], resident.
//
// Warps: 0 issues the copies, 1 allocates TMEM and issues the MMAs, 2-9 are the epilogue:
// warp 2 + 4 h + q reads lane quarter q and writes output row 2 y + h (phases (h, 0),
// (h, 1)): lanes 1..30 each produce two output pixels x 5 channels; the warp's 60 pixels
// (1200 contiguous bytes of the output row) are staged in shared memory and written by one
// bulk copy (the warp's 30 pixels and the grid's width even; otherwise per-lane stores).
#include <cuda.h>

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
constexpr int kN = 64;                                     // 3 column taps x 20 + 4
constexpr uint32_t kRowBytes = 128;                        // 64 bf16 channels
constexpr uint32_t kBlkBytes = 128 * kRowBytes;            // 16 KB: one channel block of a row
constexpr uint32_t kSlotBytes = 2 * kBlkBytes;             // 32 KB: one input row
constexpr uint32_t kBoxBytes = 32 * kRowBytes;             // 4 KB: one 32-pixel box
constexpr int kSlots = 4;                                  // input rows: the producer runs 2 tiles ahead
constexpr int kFSlots = 6;                                 // F^{s-1} rows
constexpr uint32_t kFRow = 128 * 20;                       // 2560 bytes: 128 pixels x 5 floats
constexpr uint32_t kSliceBytes = kN * kRowBytes;           // 8 KB: one (channel block, ky) slice
constexpr int kThreads = 320;
constexpr uint32_t kIdesc = ptx::make_idesc(128, kN, 1, 1);
constexpr uint32_t kStgBytes = 2 * kWp * 5 * 4;            // per epilogue warp: 60 output pixels x 20 B

struct __align__(16) T1Bars {
    uint64_t wfull;
    uint64_t full[kSlots], empty[kSlots];
    uint64_t ffull[kFSlots], fempty[kFSlots];
    uint64_t tmem_full[2], tmem_empty[2];
    uint64_t drain;
    uint64_t never; // signalled by nothing: the fault-injection wait
    uint32_t tmem_base;
    int abort;
};

constexpr uint32_t kOffSlot = 6 * kSliceBytes;             // 48 KB of weights
constexpr uint32_t kOffF = kOffSlot + kSlots * kSlotBytes;
constexpr uint32_t kOffStg = kOffF + kFSlots * kFRow;
constexpr uint32_t kOffBars = kOffStg + 8 * kStgBytes;
constexpr size_t kSmem = kOffBars + sizeof(T1Bars) + 1024;
static_assert(kSmem <= 227 * 1024, "t1 shared memory");
static_assert(kOffSlot % 1024 == 0 && kOffF % 16 == 0 && kOffStg % 16 == 0 && kOffBars % 16 == 0, "t1 layout");

struct T1Params {
    const float *bias;                // 5 output biases
    const float *fm_prev;             // F^{s-1}, M^{s-1}: n x h x w x 5 (the input grid)
    float *out;                       // F^s, M^s: n x 2 h x 2 w x 5
    const int *n_dev;                 // device view count (size-bucket graphs), or NULL
    int n_img, h, w, strips;
    long long stall_cycles;           // fault injection (tests): > 0 makes the MMA warp wait on `never`
    int *err;
};

struct T1Walk {
    int n, strip, y, h, strips;
    bool cont;
    __device__ T1Walk(int t, int h_, int strips_) : h(h_), strips(strips_), cont(false) {
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
template <int S> struct T1Ring {
    int slot = 0;
    uint32_t par = 0;
    __device__ void step() { if (++slot == S) { slot = 0; par ^= 1; } }
};

// The slots of rows y - 1, y, y + 1 of the current tile: the same ring walk in every role.
template <int S> struct T1Rows {
    T1Ring<S> ring;
    int rs[3] = {0, 0, 0};
    uint32_t rp[3] = {0, 0, 0};
    __device__ void take(int r) {
        rs[r] = ring.slot;
        rp[r] = ring.par;
        ring.step();
    }
    __device__ void advance(bool cont) { // (static indices: the arrays stay in registers)
        if (cont) {
            rs[0] = rs[1]; rp[0] = rp[1]; rs[1] = rs[2]; rp[1] = rp[2];
        } else {
            take(0);
            take(1);
        }
        take(2);
    }
};

__global__ void __launch_bounds__(kThreads, 1)
vib_t1_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const T1Params p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = smem;
    uint8_t *sSlot = smem + kOffSlot;
    uint8_t *sF = smem + kOffF;
    uint8_t *sStg = smem + kOffStg;
    T1Bars *bars = (T1Bars *)(smem + kOffBars);
    volatile int *abort = &bars->abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        ptx::mbar_init(ptx::smem_u32(&bars->wfull), 1);
        for (int s = 0; s < kSlots; ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->empty[s]), 1);
        }
        for (int s = 0; s < kFSlots; ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->ffull[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->fempty[s]), 8); // one arrive per epilogue warp
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_full[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->tmem_empty[a]), 8);
        }
        ptx::mbar_init(ptx::smem_u32(&bars->drain), 1);
        ptx::mbar_init(ptx::smem_u32(&bars->never), 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(&bars->tmem_base), 128); // two accumulators of 64 columns
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
    const int per_view = p.strips * p.h;
    const int num_tiles = n_img * per_view;
    const int per_cta = (num_tiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t_begin = min(num_tiles, (int)blockIdx.x * per_cta), t_end = min(num_tiles, t_begin + per_cta);

    if (warp == 0) {
        // ---------------- copy producer ----------------
        if (lane == 0) {
            const uint32_t fw = ptx::smem_u32(&bars->wfull);
            ptx::mbar_arrive_expect_tx(fw, 6 * kSliceBytes);
#pragma unroll
            for (int c = 0; c < 2; ++c) // channel block c: its three row-tap slices in one box
                ptx::tma_load_3d(ptx::smem_u32(sB) + c * 3 * kSliceBytes, &tmB, fw, c * 64, 0, 0);
            T1Ring<kSlots> ring;
            T1Ring<kFSlots> fring;
            long long issued = 0, f_issued = 0;
            T1Walk tw(t_begin, p.h, p.strips);
            bool stop = false;
            for (int t = t_begin; t < t_end && !stop && !*abort; ++t, tw.next()) {
                const int x0 = tw.strip * kTw;
                const int f0 = max(0, x0 - 4), f1 = min(p.w, x0 + 124); // F^{s-1} pixels (multiples of 4)
                // new rows: y + 1, and y - 1, y where a segment starts
                for (int j = tw.cont ? 2 : 0; j < 3; ++j) {
                    const int row = tw.y - 1 + j;
                    if (!wait_bar(ptx::smem_u32(&bars->empty[ring.slot]), ring.par ^ 1u, abort, p.err, 1) ||
                        !wait_bar(ptx::smem_u32(&bars->fempty[fring.slot]), fring.par ^ 1u, abort, p.err, 1)) {
                        stop = true;
                        break;
                    }
                    const uint32_t fs = ptx::smem_u32(&bars->full[ring.slot]);
                    ptx::mbar_arrive_expect_tx(fs, kSlotBytes);
                    const uint32_t dst = ptx::smem_u32(sSlot) + ring.slot * kSlotBytes;
#pragma unroll
                    for (int c = 0; c < 2; ++c)
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            ptx::tma_load_4d(dst + c * kBlkBytes + q * kBoxBytes, &tmA, fs, c * 64, x0 - 1 + kWp * q, row,
                                             tw.n);
                    ++issued;
                    ring.step();
                    // the F^{s-1} row, clamped into the grid like the upsampling's taps
                    const int fr = min(max(row, 0), p.h - 1);
                    const uint32_t ff = ptx::smem_u32(&bars->ffull[fring.slot]);
                    const uint32_t bytes = (uint32_t)(f1 - f0) * 20u;
                    ptx::mbar_arrive_expect_tx(ff, bytes);
                    ptx::bulk_load(ptx::smem_u32(sF) + fring.slot * kFRow,
                                   p.fm_prev + (((size_t)tw.n * p.h + fr) * p.w + f0) * 5, bytes, ff);
                    ++f_issued;
                    fring.step();
                }
            }
            // every copy issued has landed before the CTA can exit
            for (long long k = 1; k <= issued && k <= kSlots; ++k) {
                const long long q = issued - k;
                drain_wait(ptx::smem_u32(&bars->full[q % kSlots]), (uint32_t)((q / kSlots) & 1));
            }
            for (long long k = 1; k <= f_issued && k <= kFSlots; ++k) {
                const long long q = f_issued - k;
                drain_wait(ptx::smem_u32(&bars->ffull[q % kFSlots]), (uint32_t)((q / kFSlots) & 1));
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
            T1Rows<kSlots> rows;
            bool issued_any = false;
            T1Walk tw(t_begin, p.h, p.strips);
            for (int t = t_begin; ok && t < t_end && !*abort; ++t, tw.next()) {
                rows.advance(tw.cont);
                if (!wait_bar(ptx::smem_u32(&bars->tmem_empty[acc]), acc_phase ^ 1, abort, p.err, 2)) break;
                ptx::tc_fence_after();
                for (int r = 0; r < 3 && ok; ++r)
                    ok = wait_bar(ptx::smem_u32(&bars->full[rows.rs[r]]), rows.rp[r], abort, p.err, 3);
                if (!ok) break;
                ptx::tc_fence_after();
                const uint32_t d = tmem + acc * kN;
                // K order (row tap, channel block, 16-channel step), as the generic kernel
#pragma unroll
                for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t a0 = sw + rows.rs[ky] * kSlotBytes + c * kBlkBytes;
                        const uint32_t b0 = bw + (c * 3 + ky) * kSliceBytes;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint64_t ad = ptx::smem_desc(a0 + k * 32, kRowBytes);
                            const uint64_t bd = ptx::smem_desc(b0 + k * 32, kRowBytes);
                            ptx::mma_bf16(d, ad, bd, kIdesc, (ky | c | k) != 0);
                        }
                    }
                issued_any = true;
                ptx::mma_commit(ptx::smem_u32(&bars->tmem_full[acc]));
                // input row y - 1 is done; y, y + 1 stay when the next tile continues
                ptx::mma_commit(ptx::smem_u32(&bars->empty[rows.rs[0]]));
                if (!(t + 1 < t_end && tw.y + 1 < p.h)) {
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[rows.rs[1]]));
                    ptx::mma_commit(ptx::smem_u32(&bars->empty[rows.rs[2]]));
                }
                if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            }
            if (issued_any) {
                ptx::mma_commit(ptx::smem_u32(&bars->drain));
                drain_wait(ptx::smem_u32(&bars->drain), 0);
            }
        }
    } else {
        // ---------------- epilogue: Eq. 2 for output row 2 y + hh ----------------
        const int q = warp & 3, hh = (warp - 2) >> 2;
        const uint32_t stg = ptx::smem_u32(sStg + (warp - 2) * kStgBytes);
        float bias[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) bias[k] = __ldg(p.bias + k);
        const int wo = 2 * p.w;
        int acc = 0;
        uint32_t acc_phase = 0;
        T1Rows<kFSlots> frows;
        T1Walk tw(t_begin, p.h, p.strips);
        for (int t = t_begin; t < t_end && !*abort; ++t, tw.next()) {
            frows.advance(tw.cont);
            const int x0 = tw.strip * kTw, xw = x0 + kWp * q;
            const int nw = min(kWp, p.w - xw);          // the warp's input pixels inside the grid
            const int kgx = x0 - 1 + kWp * q + lane;   // this lane's input pixel
            const bool mine = lane >= 1 && lane <= nw;
            int ok = 1;
            if (lane == 0) ok = wait_bar(ptx::smem_u32(&bars->tmem_full[acc]), acc_phase, abort, p.err, 4);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            ptx::tc_fence_after();
            // columns kx * 20 + 10 hh .. + 9 of each column tap (phases (hh, 0), (hh, 1)),
            // read as 4-column loads from the multiple of 4 at or below
            uint32_t r[3][12];
            const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + acc * kN;
            __syncwarp();
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const uint32_t a0 = (uint32_t)(kx * 20 + 10 * hh) & ~3u;
#pragma unroll
                for (int u = 0; u < 3; ++u) ptx::tmem_ld4(tb + a0 + 4 * u, &r[kx][4 * u]);
            }
            ptx::tmem_ld_wait();
            // the accumulator is free once read
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->tmem_empty[acc]));
            if (++acc == 2) { acc = 0; acc_phase ^= 1; }
            // tap sums (the generic kernel's order: tap 0 of the lane before + tap 1 + tap 2 of the next)
            // (column 10 hh sits 2 hh mod 4 into its 4-column-aligned load: 0 or 2, selected
            // with static register indices)
            float v[10];
#pragma unroll
            for (int j = 0; j < 10; ++j) {
                const uint32_t c0 = hh ? r[0][2 + j] : r[0][j], c1 = hh ? r[1][2 + j] : r[1][j],
                               c2 = hh ? r[2][2 + j] : r[2][j];
                const float left = __shfl_up_sync(0xffffffffu, __uint_as_float(c0), 1);
                const float right = __shfl_down_sync(0xffffffffu, __uint_as_float(c2), 1);
                v[j] = left + __uint_as_float(c1) + right;
            }
            // F^{s-1} rows y - 1 + hh, y + hh (the rows the upsampling of output row 2 y + hh
            // reads), clamped columns kgx - 1 .. kgx + 1
            const int fa = hh ? frows.rs[1] : frows.rs[0], fb = hh ? frows.rs[2] : frows.rs[1];
            const uint32_t pa = hh ? frows.rp[1] : frows.rp[0], pb = hh ? frows.rp[2] : frows.rp[1];
            if (lane == 0 && (!wait_bar(ptx::smem_u32(&bars->ffull[fa]), pa, abort, p.err, 4) ||
                              !wait_bar(ptx::smem_u32(&bars->ffull[fb]), pb, abort, p.err, 4)))
                ok = 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            const int f0 = max(0, x0 - 4);
            // every lane computes (its clamped columns lie in the copied row: lanes 0 and 31
            // and lanes past the grid read in-range values), only lanes 1..nw store
            float out10[10];
            {
                float nb[2][3][5];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const uint32_t frow = ptx::smem_u32(sF) + (a ? fb : fa) * kFRow;
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const int xx = min(max(kgx + b - 1, 0), p.w - 1) - f0;
#pragma unroll
                        for (int k = 0; k < 5; ++k) nb[a][b][k] = ptx::lds_f32(frow + (uint32_t)(xx * 20 + k * 4));
                    }
                }
                // F^s, M^s = up(F^{s-1}) x 2, up(M^{s-1}) + Res^s (phase (hh, px), channel k)
                const float ly = hh ? 0.25f : 0.75f;
#pragma unroll
                for (int px = 0; px < 2; ++px) {
                    const float lx = px ? 0.25f : 0.75f;
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        const float up = (1.f - ly) * ((1.f - lx) * nb[0][px][k] + lx * nb[0][px + 1][k]) +
                                         ly * ((1.f - lx) * nb[1][px][k] + lx * nb[1][px + 1][k]);
                        out10[px * 5 + k] = v[px * 5 + k] * 1.f + bias[k] + up * (k < 4 ? 2.f : 1.f);
                    }
                }
            }
            // the F^{s-1} rows this warp read: row y - 1 is done (y, y + 1 stay when the next
            // tile continues); every warp releases every row it walks past
            __syncwarp();
            if (lane == 0) {
                ptx::mbar_arrive(ptx::smem_u32(&bars->fempty[frows.rs[0]]));
                if (!(t + 1 < t_end && tw.y + 1 < p.h)) {
                    ptx::mbar_arrive(ptx::smem_u32(&bars->fempty[frows.rs[1]]));
                    ptx::mbar_arrive(ptx::smem_u32(&bars->fempty[frows.rs[2]]));
                }
            }
            if (nw <= 0) continue;
            // output row 2 y + hh, pixels 2 xw .. 2 xw + 2 nw - 1 (5 floats each)
            float *dst = p.out + (((size_t)tw.n * (2 * p.h) + 2 * tw.y + hh) * wo + 2 * xw) * 5;
            if (nw == kWp && (p.w & 1) == 0) {
                // the previous tile's bulk store has read the staging row
                if (lane == 0) ptx::bulk_wait_read<0>();
                __syncwarp();
                // (lane l - 1's 10 floats at word 10 (l - 1): 2-way bank conflicts)
                if (mine) {
#pragma unroll
                    for (int j = 0; j < 10; ++j)
                        asm volatile("st.shared.f32 [%0], %1;" ::"r"(stg + (uint32_t)((lane - 1) * 40 + j * 4)), "f"(out10[j])
                                     : "memory");
                }
                // 300 floats = 1200 contiguous bytes (the row segment starts 16-byte aligned:
                // 2 xw x 20 bytes with xw a multiple of 30, rows of 2 w x 20 bytes with w even),
                // one bulk copy issued by one lane
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    ptx::bulk_store(dst, stg, 2 * kWp * 5 * 4);
                    ptx::bulk_commit();
                }
            } else if (mine) {
#pragma unroll
                for (int j = 0; j < 10; ++j) dst[(lane - 1) * 10 + j] = out10[j];
            }
        }
        if (lane == 0) ptx::bulk_wait<0>(); // the stores have completed before the CTA exits
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 128);
    }
}

} // namespace

bool vib_t1_ok(const fvv_interp *h, int li, int in_cs, int in_coff, int N, int hin, int win, int out_cs, int out_coff,
               bool out_f32) {
    const LayerDef &L = kLayers[li];
    return li < kCtx && li % 10 == 9 && li != kVib0 + 9 && L.kind == K_CONVT && L.ci == 128 && L.co == 5 &&
           h->o.precision == FVV_BF16 && h->o.pad_mode == FVV_PAD_ZERO && h->tc[li].ci_pad == 128 &&
           h->tc[li].kxf_n == kN && h->tc[li].wk && in_cs == 128 && in_coff == 0 && out_cs == 5 && out_coff == 0 &&
           out_f32 && N >= 1 && hin >= 1 && win >= 4 && win % 4 == 0;
}

int tc_vib_t1(fvv_interp *h, int li, const void *in, int N, int hin, int win, const float *fm_prev, float *out,
              const int *n_dev, cudaStream_t st) {
    if (!vib_t1_ok(h, li, 128, 0, N, hin, win, 5, 0, true) || ((uintptr_t)in & 15) || !fm_prev ||
        ((uintptr_t)fm_prev & 15) || ((uintptr_t)out & 15)) {
        set_error("layer %s: not the fused t1 kernel's call", kLayers[li].name);
        return FVV_EINVAL;
    }
    // the input: N x hin x win pixels of 128 bf16 channels; boxes of 64 channels x 32 pixels
    CUtensorMap ma;
    cuuint64_t dims[4] = {128, (cuuint64_t)win, (cuuint64_t)hin, (cuuint64_t)N};
    cuuint64_t strides[3] = {256, (cuuint64_t)win * 256, (cuuint64_t)hin * win * 256};
    cuuint32_t box[4] = {64, 32, 1, 1};
    FVV_TRY(tc_encode_map(&ma, 4, (void *)in, dims, strides, box, 128));
    T1Params p{};
    p.bias = h->bias + h->b_off[li];
    p.fm_prev = fm_prev;
    p.out = out;
    p.n_dev = n_dev;
    p.n_img = N;
    p.h = hin; p.w = win;
    p.strips = (win + kTw - 1) / kTw;
    p.stall_cycles = h->stall_now;
    p.err = h->d_err;
    const long long tiles = (long long)N * p.strips * hin;
    if (tiles > (1ll << 30)) { set_error("too many tiles"); return FVV_ESHAPE; }
    static int sms = 0;
    if (!sms) {
        int dev;
        FVV_CHECK_CUDA(cudaGetDevice(&dev));
        FVV_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FVV_CHECK_CUDA(cudaFuncSetAttribute(vib_t1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    }
    const int grid = (int)(tiles < sms ? tiles : sms);
    vib_t1_kernel<<<grid, kThreads, kSmem, st>>>(ma, *(const CUtensorMap *)h->tc[li].map_k, p);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

} // namespace fvv
