// Laplacian-pyramid loss (Eq. 3, Sec. 3.1 "Loss functions") of n image pairs:
//   L_Lap = sum_{i=1..5} 2^(i-1) || L^i(pred) - L^i(gt) ||_1
// with the Burt-Adelson pyramid of the binomial kernel k = [1 4 6 4 1] / 16 (edges
// replicated): G^1 = I, G^(i+1) = (k k^T * G^i) at even pixels, up(G) = the
// zero-inserted G filtered by 4 k k^T (coarse indices clamped), L^i = G^i - up(G^(i+1))
// for i < 5 and L^5 = G^5; the L1 norm sums |.| over every pixel and channel.
//
// Every pyramid step is linear, so L^i(pred) - L^i(gt) = L^i(pred - gt): the kernels
// build ONE pyramid, of the difference D = pred - gt, formed as the first level is
// loaded (the two images are read once).  One launch per level i = 1..4: a block
// owns a TY x TX tile of G^(i+1); it stages the G^i rows and columns that tile and its
// one-pixel halo need (edge-replicated) in shared memory, blurs them horizontally at
// the even columns and vertically at the even rows, writes its G^(i+1) tile, and sums
// |G^i - up(G^(i+1))| over its 2TY x 2TX pixels of level i (the halo supplies up()'s
// neighbours); the last level's kernel also sums |G^5| (= L^5) of its tiles.  Block sums
// go to fixed slots; a last kernel adds them per view in a fixed order (deterministic)
// and weights the levels.
#include "common.h"

namespace fvv {
namespace {

constexpr int kLevels = 5;
constexpr int TY = 16, TX = 32;               // coarse tile of G^(i+1)
constexpr int RY = 2 * TY + 7, RX = 2 * TX + 7; // staged rows / columns of G^i
constexpr int GY = TY + 2, GX = TX + 2;        // G^(i+1) tile with its halo
constexpr int kThreadsLap = 256;
constexpr int kThreadsRed = 32 * 5; // final sums: one warp per level
constexpr size_t kLapSmem = (size_t)(RY * RX * 3 + RY * GX * 3 + GY * GX * 3) * sizeof(float);

__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// Level i of the pyramid: src = G^i (n x H x W x 3) or, at the first level, pred and
// gt (D = pred - gt).  Writes G^(i+1) (n x h x w x 3) and one partial L1 sum per block.
template <bool FIRST>
__global__ void __launch_bounds__(kThreadsLap)
lap_level_kernel(const float *__restrict__ a, const float *__restrict__ b, int H, int W, float *__restrict__ g_next,
                 int h, int w, int tiles_x, float *__restrict__ partial, float *__restrict__ partial_next) {
    extern __shared__ float sm[];
    float *sD = sm;                      // RY x RX x 3: G^i around the tile, edge-replicated
    float *sT = sD + RY * RX * 3;        // RY x GX x 3: horizontal blur at even columns
    float *sG = sT + RY * GX * 3;        // GY x GX x 3: G^(i+1), halo indices clamped
    const int view = blockIdx.y;
    const int cy0 = (blockIdx.x / tiles_x) * TY, cx0 = (blockIdx.x % tiles_x) * TX;
    const int fy0 = 2 * cy0 - 4, fx0 = 2 * cx0 - 4; // staged origin in level-i pixels
    const size_t img = (size_t)H * W * 3;
    const float *pa = a + view * img;
    const float *pb = FIRST ? b + view * img : nullptr;

    // 1. stage G^i: rows fy0 .. fy0 + RY - 1, columns fx0 .. fx0 + RX - 1 (clamped), one
    //    pixel (3 channels) per item, a warp per staged row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < RY; r += kThreadsLap / 32) {
        const float *ra = pa + (size_t)clampi(fy0 + r, H) * W * 3;
        const float *rb = FIRST ? pb + (size_t)clampi(fy0 + r, H) * W * 3 : nullptr;
        float *dr = sD + r * RX * 3;
#pragma unroll
        for (int c = lane; c < ((RX + 31) / 32) * 32; c += 32) {
            if (c < RX) {
                const int gx = clampi(fx0 + c, W) * 3;
                float v0 = __ldg(ra + gx), v1 = __ldg(ra + gx + 1), v2 = __ldg(ra + gx + 2);
                if (FIRST) { v0 -= __ldg(rb + gx); v1 -= __ldg(rb + gx + 1); v2 -= __ldg(rb + gx + 2); }
                dr[3 * c] = v0; dr[3 * c + 1] = v1; dr[3 * c + 2] = v2;
            }
        }
    }
    __syncthreads();
    // 2. horizontal blur at the even columns of the coarse tile + halo (coarse column
    //    cx0 - 1 + j, clamped to the image: the halo of a border tile repeats its edge)
    constexpr float k0 = 1.f / 16, k1 = 4.f / 16, k2 = 6.f / 16;
    for (int e = threadIdx.x; e < RY * GX; e += kThreadsLap) {
        const int r = e / GX, j = e - r * GX;
        const int lc = 2 * clampi(cx0 - 1 + j, w) - fx0 - 2; // staged column of tap 0
        const float *d = sD + (r * RX + lc) * 3;
        float *t = sT + e * 3;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            t[ch] = k0 * d[ch] + k1 * d[3 + ch] + k2 * d[6 + ch] + k1 * d[9 + ch] + k0 * d[12 + ch];
    }
    __syncthreads();
    // 3. vertical blur at the even rows -> G^(i+1) on the tile + halo; write the tile
    float *gn = g_next + (size_t)view * h * w * 3;
    float acc_next = 0.f; // last level kernel: ||G^(i+1)||_1 of the tile (L^5 = G^5)
    for (int e = threadIdx.x; e < GY * GX; e += kThreadsLap) {
        const int i = e / GX, j = e - i * GX;
        const int cy = cy0 - 1 + i, cx = cx0 - 1 + j;
        const int lr = 2 * clampi(cy, h) - fy0 - 2;          // staged row of tap 0
        const float *t = sT + (lr * GX + j) * 3;
        const bool store = i >= 1 && i <= TY && j >= 1 && j <= TX && cy < h && cx < w;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float g = k0 * t[ch] + k1 * t[GX * 3 + ch] + k2 * t[2 * GX * 3 + ch] + k1 * t[3 * GX * 3 + ch] +
                            k0 * t[4 * GX * 3 + ch];
            sG[e * 3 + ch] = g;
            if (store) {
                gn[((size_t)cy * w + cx) * 3 + ch] = g;
                acc_next += fabsf(g);
            }
        }
    }
    __syncthreads();
    // 4. |G^i - up(G^(i+1))| over the 2TY x 2TX pixels of level i, a 2 x 2 quad per item:
    //    quad (m, n) = level-i pixels (2m + dy, 2n + dx) of coarse pixel (m, n).  Pixel row
    //    2m takes coarse rows m - 1, m, m + 1 with weights 1/8, 6/8, 1/8 and row 2m + 1 rows
    //    m, m + 1 with 1/2, 1/2; columns alike.  So one 3 x 3 coarse neighbourhood (sG
    //    rows / columns m .. m + 2 of the tile) serves the quad, interpolated separably.
    float acc = 0.f;
    for (int e = threadIdx.x; e < TY * TX; e += kThreadsLap) {
        const int m = e / TX, n = e - m * TX;
        const int y = 2 * (cy0 + m), x = 2 * (cx0 + n);
        if (y >= H || x >= W) continue;
        const bool y1 = y + 1 < H, x1 = x + 1 < W;
        const float *g = sG + (m * GX + n) * 3;
        const float *d = sD + ((2 * m + 4) * RX + 2 * n + 4) * 3;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float ve[3], vo[3]; // vertical interpolation at the even / odd pixel row, per coarse column
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float a0 = g[q * 3 + ch], a1 = g[(GX + q) * 3 + ch], a2 = g[(2 * GX + q) * 3 + ch];
                ve[q] = 0.125f * (a0 + a2) + 0.75f * a1;
                vo[q] = 0.5f * (a1 + a2);
            }
            const float ee = 0.125f * (ve[0] + ve[2]) + 0.75f * ve[1], eo = 0.5f * (ve[1] + ve[2]);
            const float oe = 0.125f * (vo[0] + vo[2]) + 0.75f * vo[1], oo = 0.5f * (vo[1] + vo[2]);
            acc += fabsf(d[ch] - ee);
            if (x1) acc += fabsf(d[3 + ch] - eo);
            if (y1) acc += fabsf(d[RX * 3 + ch] - oe);
            if (x1 && y1) acc += fabsf(d[RX * 3 + 3 + ch] - oo);
        }
    }
    // block sums (fixed order) -> partial[view][block] (and partial_next)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        acc_next += __shfl_xor_sync(0xffffffffu, acc_next, o);
    }
    __shared__ float wsum[2][kThreadsLap / 32];
    if ((threadIdx.x & 31) == 0) {
        wsum[0][threadIdx.x >> 5] = acc;
        wsum[1][threadIdx.x >> 5] = acc_next;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f, s2 = 0.f;
#pragma unroll
        for (int i = 0; i < kThreadsLap / 32; ++i) {
            s += wsum[0][i];
            s2 += wsum[1][i];
        }
        partial[(size_t)view * gridDim.x + blockIdx.x] = s;
        if (partial_next) partial_next[(size_t)view * gridDim.x + blockIdx.x] = s2;
    }
}

struct LapPlan {
    int h[kLevels], w[kLevels];     // size of level i (0-based: G^1 .. G^5)
    int blocks[kLevels - 1];        // blocks per view of the level kernels
    size_t g_off[kLevels], p_off[kLevels], bytes; // p_off[4]: ||G^5||_1 per block of the last level kernel
};

__host__ LapPlan lap_plan(int n, int H, int W) {
    LapPlan P{};
    int h = H, w = W;
    size_t off = 0;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    for (int i = 0; i < kLevels; ++i) {
        P.h[i] = h; P.w[i] = w;
        if (i > 0) { P.g_off[i] = off; off += al((size_t)n * h * w * 3 * sizeof(float)); }
        h = (h + 1) / 2; w = (w + 1) / 2;
    }
    for (int i = 0; i < kLevels - 1; ++i) {
        P.blocks[i] = ceil_div(P.h[i + 1], TY) * ceil_div(P.w[i + 1], TX);
        P.p_off[i] = off;
        off += al((size_t)n * P.blocks[i] * sizeof(float));
    }
    P.p_off[kLevels - 1] = off;
    off += al((size_t)n * P.blocks[kLevels - 2] * sizeof(float));
    P.bytes = off;
    return P;
}

struct LapSums {
    const float *part[kLevels]; // block sums of L^1 .. L^4, and of |G^5| (= L^5)
    int blocks[kLevels];
};

// One block per view, one warp per level: the level's block sums in a fixed order
// (double: lane-strided, then a fixed shuffle tree), then the weighted loss.
__global__ void __launch_bounds__(kThreadsRed) lap_reduce_kernel(const LapSums s, float *loss, float *norms) {
    __shared__ double lvl[kLevels];
    const int view = blockIdx.x, lv = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc = 0.0;
    const float *p = s.part[lv] + (size_t)view * s.blocks[lv];
    for (int i = lane; i < s.blocks[lv]; i += 32) acc += p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        lvl[lv] = acc;
        if (norms) norms[(size_t)view * kLevels + lv] = (float)acc;
    }
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        double tot = 0.0;
#pragma unroll
        for (int i = 0; i < kLevels; ++i) tot += ldexp(lvl[i], i); // weight 2^(i-1), i counted from 1
        loss[view] = (float)tot;
    }
}

} // namespace
} // namespace fvv

using namespace fvv;

extern "C" size_t fvv_lap_loss_workspace(int n, int H, int W) {
    if (n < 1 || H < 2 || W < 2) return 0;
    return lap_plan(n, H, W).bytes;
}

extern "C" int fvv_lap_loss(const float *pred, const float *gt, int n, int H, int W, void *workspace,
                            size_t workspace_bytes, float *loss, float *level_norms, void *stream) {
    clear_error();
    if (!pred || !gt || !workspace || (!loss && !level_norms)) { set_error("lap_loss: NULL argument"); return FVV_EINVAL; }
    if (n < 1 || n > 65535 || H < 2 || W < 2 || (long long)H * W > (1ll << 28)) {
        set_error("lap_loss: need 1 <= n <= 65535 and 2 <= H, W with H x W <= 2^28");
        return FVV_ESHAPE;
    }
    const LapPlan P = lap_plan(n, H, W);
    if (workspace_bytes < P.bytes || ((uintptr_t)workspace & 255)) {
        set_error("lap_loss: workspace of %zu bytes, 256-byte aligned, needed (got %zu)", P.bytes, workspace_bytes);
        return FVV_EINVAL;
    }
    static bool attr_set[2] = {false, false};
    if (!attr_set[0]) {
        FVV_CHECK_CUDA(cudaFuncSetAttribute(lap_level_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kLapSmem));
        attr_set[0] = true;
    }
    if (!attr_set[1]) {
        FVV_CHECK_CUDA(cudaFuncSetAttribute(lap_level_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kLapSmem));
        attr_set[1] = true;
    }
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    LapSums sums{};
    for (int lv = 0; lv < kLevels - 1; ++lv) {
        const float *src = lv == 0 ? pred : (const float *)(ws + P.g_off[lv]);
        float *dst = (float *)(ws + P.g_off[lv + 1]);
        float *part = (float *)(ws + P.p_off[lv]);
        const int tiles_x = ceil_div(P.w[lv + 1], TX);
        dim3 grid(P.blocks[lv], n);
        // the last level kernel also sums |G^5| (= L^5) of its tiles
        float *part_next = lv == kLevels - 2 ? (float *)(ws + P.p_off[kLevels - 1]) : nullptr;
        if (lv == 0)
            lap_level_kernel<true><<<grid, kThreadsLap, kLapSmem, st>>>(src, gt, P.h[lv], P.w[lv], dst, P.h[lv + 1],
                                                                        P.w[lv + 1], tiles_x, part, part_next);
        else
            lap_level_kernel<false><<<grid, kThreadsLap, kLapSmem, st>>>(src, nullptr, P.h[lv], P.w[lv], dst,
                                                                         P.h[lv + 1], P.w[lv + 1], tiles_x, part,
                                                                         part_next);
        FVV_CHECK_CUDA(cudaGetLastError());
        sums.part[lv] = part;
        sums.blocks[lv] = P.blocks[lv];
    }
    sums.part[kLevels - 1] = (const float *)(ws + P.p_off[kLevels - 1]);
    sums.blocks[kLevels - 1] = P.blocks[kLevels - 2];
    lap_reduce_kernel<<<n, kThreadsRed, 0, st>>>(sums, loss, level_norms);
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}
