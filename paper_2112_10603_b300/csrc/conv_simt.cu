// Plain FP32 convolution path: implicit GEMM on the CUDA cores (FFMA, no TF32).
//
// Conv2d 3x3 pad 1 (stride 1 or 2) and ConvTranspose2d 4x4 stride 2 pad 1, the
// two operations of Table 3.  GEMM view: M = output pixels, N = C_out,
// K = taps x C_in.  The transposed conv is split into its 4 output phases
// (oy mod 2, ox mod 2); each phase is a 2x2-tap conv over the input grid:
//   phase p = 0: taps ky in {1, 3} read input rows qy, qy - 1
//   phase p = 1: taps ky in {0, 2} read input rows qy + 1, qy
// (from oy = 2 iy - 1 + ky), and likewise for columns.
//
// Weights are packed on the host into [K][Co] rows (k = tap * Ci + ci), per
// phase for the transposed conv.  Inputs/outputs may be channel slices of wider
// tensors (pixel stride cs, channel offset coff), which is how concatenations
// are formed without copies.
#include <cstring>

#include "common.h"
#include "kernels.h"

namespace fvv {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ float load_in(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_in(const bf16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void store_out(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_out(bf16 *p, float v) { *p = __float2bfloat16_rn(v); }
// 16 consecutive channels of one pixel: 16-byte stores where the address allows
__device__ __forceinline__ void store16(float *p, const float (&v)[16]) {
    if (((uintptr_t)p & 15) == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) reinterpret_cast<float4 *>(p)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) p[k] = v[k];
    }
}
__device__ __forceinline__ void store16(bf16 *p, const float (&v)[16]) {
    if (((uintptr_t)p & 15) == 0) {
        __nv_bfloat162 h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        uint4 u[2];
        memcpy(u, h, 32);
        reinterpret_cast<uint4 *>(p)[0] = u[0];
        reinterpret_cast<uint4 *>(p)[1] = u[1];
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) p[k] = __float2bfloat16_rn(v[k]);
    }
}

__device__ __forceinline__ int wrap_or_mark(int i, int n, int circ) {
    if (circ) { i %= n; return i < 0 ? i + n : i; }
    return (i < 0 || i >= n) ? -1 : i;
}

// Tap geometry of a transposed-conv phase: input offset of tap t (0/1) for phase p.
__device__ __forceinline__ int convt_off(int p, int t) { return p == 0 ? -t : 1 - t; }

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(NT) conv_simt_kernel(ConvArgs a) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN];
    const Tin *in = static_cast<const Tin *>(a.in);
    Tout *out = static_cast<Tout *>(a.out);
    const float *wp = static_cast<const float *>(a.w);

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int phase = blockIdx.z;                 // 0 for conv, 0..3 for convT
    const int py = phase >> 1, px = phase & 1;
    const bool convt = a.kind == K_CONVT;
    // GEMM rows: conv -> output pixels; convT -> input-grid pixels of this phase
    const int GH = convt ? a.H : a.Ho, GW = convt ? a.W : a.Wo;
    const int Mtot = dev_count(a.n_dev, a.N) * GH * GW;
    const int taps = convt ? 4 : 9;
    const int K = taps * a.Ci;
    if (convt) wp += (size_t)phase * K * a.Co;

    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    if (m0 >= Mtot) return; // the whole block lies beyond the images run (size-bucket launch)

    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    // Per-thread A rows: element e = tid + i * NT -> (k = e % BK, m = e / BK)
    int a_n[4], a_y[4], a_x[4];
    bool a_ok[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + (tid + i * NT) / BK;
        a_ok[i] = m < Mtot;
        int mm = a_ok[i] ? m : 0;
        a_x[i] = mm % GW;
        int r = mm / GW;
        a_y[i] = r % GH;
        a_n[i] = r / GH;
    }

    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int e = tid + i * NT;
            int kk = e % BK, m = e / BK;
            int k = k0 + kk;
            float v = 0.f;
            if (a_ok[i] && k < K) {
                int tap = k / a.Ci, ci = k - tap * a.Ci;
                int iy, ix;
                if (convt) {
                    iy = a_y[i] + convt_off(py, tap >> 1);
                    ix = a_x[i] + convt_off(px, tap & 1);
                } else {
                    int ky = tap / 3, kx = tap - ky * 3;
                    iy = a_y[i] * a.stride + ky - 1;
                    ix = a_x[i] * a.stride + kx - 1;
                }
                iy = wrap_or_mark(iy, a.H, a.circ);
                ix = wrap_or_mark(ix, a.W, a.circ);
                if (iy >= 0 && ix >= 0)
                    v = load_in(in + ((size_t)(a_n[i] * a.H + iy) * a.W + ix) * a.in_cs + a.in_coff + ci);
            }
            As[kk][m] = v;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int e = tid + i * NT;
            int n = e % BN, kk = e / BN;
            int k = k0 + kk, co = n0 + n;
            Bs[kk][n] = (k < K && co < a.Co) ? __ldg(wp + (size_t)k * a.Co + co) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 av = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + ty * 4 + i;
        if (m >= Mtot) continue;
        int x = m % GW, r = m / GW, y = r % GH, n = r / GH;
        int oy = convt ? 2 * y + py : y, ox = convt ? 2 * x + px : x;
        Tout *dst = out + ((size_t)(n * a.Ho + oy) * a.Wo + ox) * a.out_cs + a.out_coff;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int co = n0 + tx * 4 + j;
            if (co >= a.Co) continue;
            float v = acc[i][j] + __ldg(a.bias + co);
            if (a.relu) v = fmaxf(v, 0.f);
            store_out(dst + co, v);
        }
    }
}

// Register-blocked form for FP32 layers whose input channels come in blocks of 8 (every
// layer of the FP32 path except the 7- / 18- / 6-channel network inputs): a CTA of 256
// threads computes 128 output pixels x BN2 output channels, each thread 8 pixels (rows
// ty*4 + 0..3 and 64 + ty*4 + 0..3) x BN2/16 channels, with 64 (BN2 = 128) FMAs per 4
// shared-memory vector loads.  A K block is 8 channels of one tap: every thread loads
// one float4 (4 channels of one pixel) of A and one float4 of B per block, through
// registers into the other of two shared-memory buffers while the current block is
// multiplied, so one barrier per block suffices.  Same per-output arithmetic as above
// except for the order of the K sum (blocks of 8 instead of 16).
constexpr int BM2 = 128, BK2 = 8;

template <int BN2>
__global__ void __launch_bounds__(NT) conv_simt_vec_kernel(ConvArgs a) {
    constexpr int TN = BN2 / 16;                        // channels per thread
    __shared__ __align__(16) float As[2][BK2][BM2];
    __shared__ __align__(16) float Bs[2][BK2][BN2];
    const float *in = static_cast<const float *>(a.in);
    float *out = static_cast<float *>(a.out);
    const float *wp = static_cast<const float *>(a.w);
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int phase = blockIdx.z, py = phase >> 1, px = phase & 1;
    const bool convt = a.kind == K_CONVT;
    const int GH = convt ? a.H : a.Ho, GW = convt ? a.W : a.Wo;
    const int Mtot = dev_count(a.n_dev, a.N) * GH * GW;
    const int taps = convt ? 4 : 9;
    const int K = taps * a.Ci, KB = K / BK2;
    if (convt) wp += (size_t)phase * K * a.Co;
    const int m0 = blockIdx.x * BM2, n0 = blockIdx.y * BN2;
    if (m0 >= Mtot) return; // the whole block lies beyond the images run (size-bucket launch)

    // this thread's A element: pixel am of the tile, channels 4 ah .. 4 ah + 3 of the block
    const int am = tid >> 1, ah = tid & 1;
    const int gm = m0 + am;
    const bool a_ok = gm < Mtot;
    int an = 0, ay = 0, ax = 0;
    if (a_ok) { ax = gm % GW; const int r = gm / GW; ay = r % GH; an = r / GH; }
    // this thread's B element: k row bk, channels 4 bc .. 4 bc + 3 of the tile (BN2 / 4
    // float4 per row, BK2 rows: only the first BK2 x BN2 / 4 threads load)
    const int bk = tid / (BN2 / 4), bc = tid % (BN2 / 4);
    const bool b_load = tid < BK2 * BN2 / 4;
    const int bco = n0 + 4 * bc;
    const bool b_vec = (a.Co % 4) == 0 && bco + 3 < a.Co;

    auto load_a = [&](int kb) -> float4 {
        const int k = kb * BK2, tap = k / a.Ci, ci = k - tap * a.Ci + 4 * ah;
        int iy, ix;
        if (convt) {
            iy = ay + convt_off(py, tap >> 1);
            ix = ax + convt_off(px, tap & 1);
        } else {
            const int ky = tap / 3, kx = tap - ky * 3;
            iy = ay * a.stride + ky - 1;
            ix = ax * a.stride + kx - 1;
        }
        iy = wrap_or_mark(iy, a.H, a.circ);
        ix = wrap_or_mark(ix, a.W, a.circ);
        if (!a_ok || iy < 0 || ix < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
        return __ldg(reinterpret_cast<const float4 *>(in + ((size_t)(an * a.H + iy) * a.W + ix) * a.in_cs + a.in_coff + ci));
    };
    auto load_b = [&](int kb) -> float4 {
        if (!b_load) return make_float4(0.f, 0.f, 0.f, 0.f);
        const float *row = wp + (size_t)(kb * BK2 + bk) * a.Co;
        if (b_vec) return __ldg(reinterpret_cast<const float4 *>(row + bco));
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = bco + j < a.Co ? __ldg(row + bco + j) : 0.f;
        return make_float4(v[0], v[1], v[2], v[3]);
    };
    auto store_tiles = [&](int buf, const float4 &va, const float4 &vb) {
        As[buf][4 * ah + 0][am] = va.x;
        As[buf][4 * ah + 1][am] = va.y;
        As[buf][4 * ah + 2][am] = va.z;
        As[buf][4 * ah + 3][am] = va.w;
        if (b_load) *reinterpret_cast<float4 *>(&Bs[buf][bk][4 * bc]) = vb;
    };

    float acc[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    store_tiles(0, load_a(0), load_b(0));
    __syncthreads();
    for (int kb = 0; kb < KB; ++kb) {
        const int buf = kb & 1;
        float4 na, nb;
        const bool more = kb + 1 < KB;
        if (more) { na = load_a(kb + 1); nb = load_b(kb + 1); }
#pragma unroll
        for (int kk = 0; kk < BK2; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float br[TN];
            if (TN == 8) {
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
                br[0] = b0.x; br[1] = b0.y; br[2] = b0.z; br[3] = b0.w;
                br[4 % TN] = b1.x; br[5 % TN] = b1.y; br[6 % TN] = b1.z; br[7 % TN] = b1.w;
            } else if (TN == 4) {
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
                br[0] = b0.x; br[1 % TN] = b0.y; br[2 % TN] = b0.z; br[3 % TN] = b0.w;
            } else {
                const float2 b0 = *reinterpret_cast<const float2 *>(&Bs[buf][kk][tx * 2]);
                br[0] = b0.x; br[1 % TN] = b0.y;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
        if (more) store_tiles(buf ^ 1, na, nb);
        __syncthreads();
    }

    // epilogue: bias, ReLU, stores (4 consecutive channels as one float4 where aligned)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (m >= Mtot) continue;
        const int x = m % GW, r = m / GW, y = r % GH, n = r / GH;
        const int oy = convt ? 2 * y + py : y, ox = convt ? 2 * x + px : x;
        float *dst = out + ((size_t)(n * a.Ho + oy) * a.Wo + ox) * a.out_cs + a.out_coff;
#pragma unroll
        for (int g = 0; g < TN; g += (TN >= 4 ? 4 : TN)) {
            const int cb = n0 + (TN == 8 ? (g == 0 ? tx * 4 : 64 + tx * 4) : tx * TN);
            const int w = TN >= 4 ? 4 : TN;
            float v[4];
#pragma unroll
            for (int j = 0; j < w; ++j) {
                const int co = cb + j;
                v[j] = co < a.Co ? acc[i][g + j] + __ldg(a.bias + co) : 0.f;
                if (a.relu) v[j] = fmaxf(v[j], 0.f);
            }
            if (w == 4 && cb + 3 < a.Co && ((uintptr_t)(dst + cb) & 15) == 0) {
                *reinterpret_cast<float4 *>(dst + cb) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int j = 0; j < w; ++j)
                    if (cb + j < a.Co) dst[cb + j] = v[j];
            }
        }
    }
}

// ContextNet's first layer (Table 3: Conv2d stride 2, 3 -> 16 channels) read
// straight from the FP32 frame: one thread per output pixel keeps all 16
// accumulators; the 27 x 16 weights sit in shared memory.  Same per-output
// summation order as the GEMM kernel (tap, then input channel).
template <typename Tout>
__global__ void __launch_bounds__(256) conv_c3_kernel(ConvArgs a) {
    __shared__ float ws[27 * 16];
    __shared__ float bs[16];
    const float *wp = static_cast<const float *>(a.w);
    for (int i = threadIdx.x; i < 27 * 16; i += blockDim.x) ws[i] = wp[i];
    if (threadIdx.x < 16) bs[threadIdx.x] = a.bias[threadIdx.x];
    __syncthreads();
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)dev_count(a.n_dev, a.N) * a.Ho * a.Wo) return;
    int ox = idx % a.Wo;
    long long r = idx / a.Wo;
    int oy = r % a.Ho, n = r / a.Ho;
    const float *in = static_cast<const float *>(a.in);
    // the frame pyramid's (R, G, B, 0) pixels: one 16-byte load per tap
    const bool vin = a.in_cs == 4 && a.in_coff == 0 && ((uintptr_t)in & 15) == 0;
    float acc[16];
#pragma unroll
    for (int co = 0; co < 16; ++co) acc[co] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        int iy = wrap_or_mark(oy * a.stride + tap / 3 - 1, a.H, a.circ);
        int ix = wrap_or_mark(ox * a.stride + tap % 3 - 1, a.W, a.circ);
        if (iy < 0 || ix < 0) continue;
        const float *src = in + ((size_t)(n * a.H + iy) * a.W + ix) * a.in_cs + a.in_coff;
        float v3[3];
        if (vin) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(src));
            v3[0] = f.x; v3[1] = f.y; v3[2] = f.z;
        } else {
#pragma unroll
            for (int ci = 0; ci < 3; ++ci) v3[ci] = __ldg(src + ci);
        }
#pragma unroll
        for (int ci = 0; ci < 3; ++ci)
#pragma unroll
            for (int co = 0; co < 16; ++co) acc[co] = fmaf(v3[ci], ws[(tap * 3 + ci) * 16 + co], acc[co]);
    }
    Tout *dst = static_cast<Tout *>(a.out) + idx * a.out_cs + a.out_coff;
    float o[16];
#pragma unroll
    for (int co = 0; co < 16; ++co) {
        float v = acc[co] + bs[co];
        o[co] = a.relu ? fmaxf(v, 0.f) : v;
    }
    store16(dst, o);
}

} // namespace

int launch_conv_c3(const ConvArgs &a, bool out_bf16, cudaStream_t st) {
    if (a.Ci != 3 || a.Co != 16 || a.kind != K_CONV) { set_error("conv_c3: 3 -> 16 conv only"); return FVV_EINVAL; }
    long long n = (long long)a.N * a.Ho * a.Wo;
    if (n <= 0) return FVV_OK;
    unsigned blocks = (unsigned)((n + 255) / 256);
    if (out_bf16) conv_c3_kernel<bf16><<<blocks, 256, 0, st>>>(a);
    else conv_c3_kernel<float><<<blocks, 256, 0, st>>>(a);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

int launch_conv_simt(const ConvArgs &a, bool in_bf16, bool out_bf16, cudaStream_t st) {
    const bool convt = a.kind == K_CONVT;
    const int GH = convt ? a.H : a.Ho, GW = convt ? a.W : a.Wo;
    const long long M = (long long)a.N * GH * GW;
    if (M <= 0) return FVV_OK;
    if (M > (1ll << 31) / 2) { set_error("conv: too many pixels"); return FVV_ESHAPE; }
    // FP32 layers with 8-channel input blocks, 16-byte aligned pixels: the register-blocked kernel
    if (!in_bf16 && !out_bf16 && a.Ci % BK2 == 0 && a.in_cs % 4 == 0 && a.in_coff % 4 == 0 &&
        ((uintptr_t)a.in % 16) == 0 && ((uintptr_t)a.w % 16) == 0) {
        const int bn = a.Co > 64 ? 128 : (a.Co > 32 ? 64 : 32);
        dim3 g2(ceil_div((int)M, BM2), ceil_div(a.Co, bn), convt ? 4 : 1);
        if (bn == 128) conv_simt_vec_kernel<128><<<g2, NT, 0, st>>>(a);
        else if (bn == 64) conv_simt_vec_kernel<64><<<g2, NT, 0, st>>>(a);
        else conv_simt_vec_kernel<32><<<g2, NT, 0, st>>>(a);
        count_launch();
        FVV_CHECK_CUDA(cudaGetLastError());
        return FVV_OK;
    }
    dim3 grid(ceil_div((int)M, BM), ceil_div(a.Co, BN), convt ? 4 : 1);
    if (!in_bf16 && !out_bf16) conv_simt_kernel<float, float><<<grid, NT, 0, st>>>(a);
    else if (in_bf16 && out_bf16) conv_simt_kernel<bf16, bf16><<<grid, NT, 0, st>>>(a);
    else if (in_bf16) conv_simt_kernel<bf16, float><<<grid, NT, 0, st>>>(a);
    else conv_simt_kernel<float, bf16><<<grid, NT, 0, st>>>(a);
    count_launch();
    FVV_CHECK_CUDA(cudaGetLastError());
    return FVV_OK;
}

// Host packing of one layer for the SIMT kernel: [phase][K][Co] floats.
void pack_simt(int kind, int Ci, int Co, const float *w, float *dst) {
    if (kind == K_CONV) {
        for (int tap = 0; tap < 9; ++tap)
            for (int ci = 0; ci < Ci; ++ci)
                for (int co = 0; co < Co; ++co)
                    dst[((size_t)tap * Ci + ci) * Co + co] = w[((size_t)co * Ci + ci) * 9 + tap];
        return;
    }
    // convT: phase (py, px), tap (ty, tx) -> kernel index (ky, kx)
    for (int py = 0; py < 2; ++py)
        for (int px = 0; px < 2; ++px)
            for (int ty = 0; ty < 2; ++ty)
                for (int tx = 0; tx < 2; ++tx) {
                    int ky = py == 0 ? 1 + 2 * ty : 2 * ty, kx = px == 0 ? 1 + 2 * tx : 2 * tx;
                    int phase = py * 2 + px, tap = ty * 2 + tx;
                    for (int ci = 0; ci < Ci; ++ci)
                        for (int co = 0; co < Co; ++co)
                            dst[(((size_t)phase * 4 + tap) * Ci + ci) * Co + co] =
                                w[((size_t)ci * Co + co) * 16 + ky * 4 + kx];
                }
}

} // namespace fvv
