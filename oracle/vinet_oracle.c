/*
 * VINet forward, FP64, CPU — the ORACLE.  Test infrastructure only: tests,
 * the smoke check and the bench's CPU-baseline leg call it; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * Plain direct loops, in the order the definitions state them; OpenMP only
 * splits independent output rows across threads.  Every step cites the passage
 * of the paper (arXiv 2112.10603) it follows:
 *
 *   Eq. 1 (Sec. 3.1)   I_mid(u) = M(u) I_l(u + F_m->l(u)) + (1 - M(u)) I_r(u + F_m->r(u))
 *   Eq. 2 (Sec. 3.1)   F^s, M^s = F^{s-1}_up, M^{s-1}_up + Res^s ;
 *                      I^s = M^s . I^s_l->m + (1 - M^s) . I^s_r->m   (s = 1, 2)
 *   Sec. 3.1 "Refinement Network": context extractor on the original views,
 *                      U-Net fed with the two pre-warped views, residual output
 *   Table 3 (supplement S.2): every layer's operation, stride, resolution, channels
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   conv 3x3 pad 1; convT 4x4 stride 2 pad 1; ReLU exactly where Table 3 writes it;
 *   VIB0 input [I_l/4, I_r/4, t] (7 ch), VIB1/2 input [I_l, I_r, W_l, W_r, M_up,
 *   F_up(4), t] (18 ch) at the stage resolution; 5 outputs = F_m->l (x, y),
 *   F_m->r (x, y), mask logit, M = sigmoid(logit); flows in pixels of the stage
 *   grid; upsampling = bilinear x2 with half-pixel centres and edge clamp, flow
 *   values x2; backward warp samples I at (x + F_x, y + F_y) bilinearly, integer
 *   pixel centres, border-clamped indices (zero mode) or wrapped (circular);
 *   stage images = box averages 2x2 / 4x4; inputs zero-padded bottom/right to a
 *   multiple of 16 and the output cropped; context features warped by the box
 *   pyramid of the final flow (values x1/2 per level); RefineNet residual
 *   2 sigmoid(z) - 1 and output clamp(I_blend + residual, 0, 1).
 *
 * Tensors are H x W x C (channels fastest), double.  Weights arrive as the
 * float32 blob in manifest order (per layer W then b; conv W [Co][Ci][3][3],
 * convT W [Ci][Co][4][4]).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Layer table (Table 3), in blob order.                                       */

enum { L_CONV = 0, L_CONVT = 1 };
typedef struct { const char *name; int kind, ci, co, stride, relu; } layer_t;

#define VIB(i, cin)                                                            \
    {"vib" #i ".c0", L_CONV, cin, 128, 2, 1}, {"vib" #i ".c1", L_CONV, 128, 256, 2, 1}, \
    {"vib" #i ".m0", L_CONV, 256, 256, 1, 1}, {"vib" #i ".m1", L_CONV, 256, 256, 1, 1}, \
    {"vib" #i ".m2", L_CONV, 256, 256, 1, 1}, {"vib" #i ".m3", L_CONV, 256, 256, 1, 1}, \
    {"vib" #i ".m4", L_CONV, 256, 256, 1, 1}, {"vib" #i ".m5", L_CONV, 256, 256, 1, 1}, \
    {"vib" #i ".t0", L_CONVT, 256, 128, 2, 1}, {"vib" #i ".t1", L_CONVT, 128, 5, 2, 0}

static const layer_t LAYERS[] = {
    VIB(0, 7), VIB(1, 18), VIB(2, 18),
    {"ctx.c0", L_CONV, 3, 16, 2, 1},   {"ctx.c1", L_CONV, 16, 16, 1, 1},
    {"ctx.c2", L_CONV, 16, 32, 2, 1},  {"ctx.c3", L_CONV, 32, 32, 1, 1},
    {"ctx.c4", L_CONV, 32, 64, 2, 1},  {"ctx.c5", L_CONV, 64, 64, 1, 1},
    {"ctx.c6", L_CONV, 64, 128, 2, 1}, {"ctx.c7", L_CONV, 128, 128, 1, 1},
    {"ref.e0a", L_CONV, 6, 32, 2, 1},    {"ref.e0b", L_CONV, 32, 32, 1, 1},
    {"ref.e1a", L_CONV, 64, 64, 2, 1},   {"ref.e1b", L_CONV, 64, 64, 1, 1},
    {"ref.e2a", L_CONV, 128, 128, 2, 1}, {"ref.e2b", L_CONV, 128, 128, 1, 1},
    {"ref.e3a", L_CONV, 256, 256, 2, 1}, {"ref.e3b", L_CONV, 256, 256, 1, 1},
    {"ref.d0", L_CONVT, 512, 128, 2, 1}, {"ref.d1", L_CONVT, 256, 64, 2, 1},
    {"ref.d2", L_CONVT, 128, 32, 2, 1},  {"ref.d3", L_CONVT, 64, 16, 2, 1},
    {"ref.out", L_CONV, 16, 3, 1, 0},
};
#define N_LAYERS ((int)(sizeof(LAYERS) / sizeof(LAYERS[0])))

static long layer_floats(const layer_t *L) {
    long taps = L->kind == L_CONV ? 9 : 16;
    return (long)L->ci * L->co * taps + L->co;
}

int oracle_n_layers(void) { return N_LAYERS; }

const char *oracle_layer_info(int i, int *kind, int *ci, int *co, int *stride, int *relu) {
    if (i < 0 || i >= N_LAYERS) return 0;
    const layer_t *L = &LAYERS[i];
    *kind = L->kind; *ci = L->ci; *co = L->co; *stride = L->stride; *relu = L->relu;
    return L->name;
}

long oracle_n_floats(void) {
    long n = 0;
    for (int i = 0; i < N_LAYERS; ++i) n += layer_floats(&LAYERS[i]);
    return n;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Index helpers: circular wrap or "outside" test.                              */

static inline int64_t wrapi(int64_t i, int64_t n) { int64_t r = i % n; return r < 0 ? r + n : r; }
static inline int64_t clampi(int64_t i, int64_t n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

/* ------------------------------------------------------------------------- */
/* Conv2d 3x3, pad 1, stride s (Table 3 "Conv2d" rows):
 *   out[oy][ox][co] = b[co] + sum_{ky,kx,ci} in[s*oy+ky-1][s*ox+kx-1][ci] * w[co][ci][ky][kx]
 * Outside taps are zero (zero mode) or wrap around (circular mode).
 * The weight is re-indexed to [ky][kx][ci][co] so that the innermost loop runs
 * over independent output channels; each output keeps the order (ky, kx, ci). */
void oracle_conv3x3(const double *in, int H, int W, int Ci, const float *w, const float *b,
                    int Co, int stride, int circ, int relu, double *out) {
    int Ho = (H + 2 - 3) / stride + 1, Wo = (W + 2 - 3) / stride + 1;
    double *wt = (double *)malloc(sizeof(double) * 9 * Ci * Co);
    for (int co = 0; co < Co; ++co)
        for (int ci = 0; ci < Ci; ++ci)
            for (int k = 0; k < 9; ++k)
                wt[((size_t)k * Ci + ci) * Co + co] = w[((size_t)co * Ci + ci) * 9 + k];
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * Co);
#pragma omp for schedule(static)
        for (int oy = 0; oy < Ho; ++oy)
            for (int ox = 0; ox < Wo; ++ox) {
                for (int co = 0; co < Co; ++co) acc[co] = b[co];
                for (int ky = 0; ky < 3; ++ky) {
                    int64_t iy = (int64_t)stride * oy + ky - 1;
                    if (circ) iy = wrapi(iy, H);
                    else if (iy < 0 || iy >= H) continue;
                    for (int kx = 0; kx < 3; ++kx) {
                        int64_t ix = (int64_t)stride * ox + kx - 1;
                        if (circ) ix = wrapi(ix, W);
                        else if (ix < 0 || ix >= W) continue;
                        const double *src = in + ((size_t)iy * W + ix) * Ci;
                        const double *wk = wt + (size_t)(ky * 3 + kx) * Ci * Co;
                        for (int ci = 0; ci < Ci; ++ci) {
                            const double v = src[ci];
                            const double *restrict wr = wk + (size_t)ci * Co;
                            double *restrict a = acc;
                            for (int co = 0; co < Co; ++co) a[co] += v * wr[co];
                        }
                    }
                }
                double *dst = out + ((size_t)oy * Wo + ox) * Co;
                for (int co = 0; co < Co; ++co) dst[co] = (relu && acc[co] < 0) ? 0.0 : acc[co];
            }
        free(acc);
    }
    free(wt);
}

/* ConvTranspose2d 4x4, stride 2, pad 1 (Table 3 "ConvTranspose2d" rows):
 * every input pixel (iy, ix) adds in[iy][ix][ci] * w[ci][co][ky][kx] to output
 * (2 iy - 1 + ky, 2 ix - 1 + kx).  Written per output pixel: the taps that reach
 * (oy, ox) are those with oy + 1 - ky even, from iy = (oy + 1 - ky) / 2.
 * Circular mode wraps iy, ix (equivalently the output index mod 2H, 2W). */
void oracle_convT(const double *in, int H, int W, int Ci, const float *w, const float *b,
                  int Co, int circ, int relu, double *out) {
    int Ho = 2 * H, Wo = 2 * W;
    double *wt = (double *)malloc(sizeof(double) * 16 * Ci * Co);
    for (int ci = 0; ci < Ci; ++ci)
        for (int co = 0; co < Co; ++co)
            for (int k = 0; k < 16; ++k)
                wt[((size_t)k * Ci + ci) * Co + co] = w[((size_t)ci * Co + co) * 16 + k];
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * Co);
#pragma omp for schedule(static)
        for (int oy = 0; oy < Ho; ++oy)
            for (int ox = 0; ox < Wo; ++ox) {
                for (int co = 0; co < Co; ++co) acc[co] = b[co];
                for (int ky = 0; ky < 4; ++ky) {
                    int ny = oy + 1 - ky;
                    if (ny & 1) continue;
                    int64_t iy = ny / 2;
                    if (circ) iy = wrapi(iy, H);
                    else if (iy < 0 || iy >= H) continue;
                    for (int kx = 0; kx < 4; ++kx) {
                        int nx = ox + 1 - kx;
                        if (nx & 1) continue;
                        int64_t ix = nx / 2;
                        if (circ) ix = wrapi(ix, W);
                        else if (ix < 0 || ix >= W) continue;
                        const double *src = in + ((size_t)iy * W + ix) * Ci;
                        const double *wk = wt + (size_t)(ky * 4 + kx) * Ci * Co;
                        for (int ci = 0; ci < Ci; ++ci) {
                            const double v = src[ci];
                            const double *restrict wr = wk + (size_t)ci * Co;
                            double *restrict a = acc;
                            for (int co = 0; co < Co; ++co) a[co] += v * wr[co];
                        }
                    }
                }
                double *dst = out + ((size_t)oy * Wo + ox) * Co;
                for (int co = 0; co < Co; ++co) dst[co] = (relu && acc[co] < 0) ? 0.0 : acc[co];
            }
        free(acc);
    }
    free(wt);
}

/* Box average over f x f blocks (stage images, "gradually increasing resolution",
 * Sec. 3.1; flow pyramid of the context-aware refinement). */
void oracle_box_down(const double *in, int H, int W, int C, int f, double *out) {
    int Ho = H / f, Wo = W / f;
    double inv = 1.0 / ((double)f * f);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ho; ++y)
        for (int x = 0; x < Wo; ++x)
            for (int c = 0; c < C; ++c) {
                double s = 0.0;
                for (int dy = 0; dy < f; ++dy)
                    for (int dx = 0; dx < f; ++dx)
                        s += in[(((size_t)y * f + dy) * W + (size_t)x * f + dx) * C + c];
                out[((size_t)y * Wo + x) * C + c] = s * inv;
            }
}

/* Bilinear x2 upsampling (F_upscale / M_upscale of Eq. 2), half-pixel centres:
 * output pixel X samples input coordinate X/2 - 1/4; taps clamp to the edge
 * (zero mode) or wrap (circular mode).  The caller scales flow values by 2. */
void oracle_upsample2x(const double *in, int H, int W, int C, int circ, double *out) {
    int Ho = 2 * H, Wo = 2 * W;
#pragma omp parallel for schedule(static)
    for (int Y = 0; Y < Ho; ++Y) {
        double sy = 0.5 * Y - 0.25, fy = floor(sy), ly = sy - fy;
        int64_t y0 = (int64_t)fy, y1 = y0 + 1;
        if (circ) { y0 = wrapi(y0, H); y1 = wrapi(y1, H); }
        else { y0 = clampi(y0, H); y1 = clampi(y1, H); }
        for (int X = 0; X < Wo; ++X) {
            double sx = 0.5 * X - 0.25, fx = floor(sx), lx = sx - fx;
            int64_t x0 = (int64_t)fx, x1 = x0 + 1;
            if (circ) { x0 = wrapi(x0, W); x1 = wrapi(x1, W); }
            else { x0 = clampi(x0, W); x1 = clampi(x1, W); }
            for (int c = 0; c < C; ++c) {
                double a = in[((size_t)y0 * W + x0) * C + c], bb = in[((size_t)y0 * W + x1) * C + c];
                double cc = in[((size_t)y1 * W + x0) * C + c], d = in[((size_t)y1 * W + x1) * C + c];
                out[((size_t)Y * Wo + X) * C + c] =
                    (1.0 - ly) * ((1.0 - lx) * a + lx * bb) + ly * ((1.0 - lx) * cc + lx * d);
            }
        }
    }
}

/* Backward warp (Eq. 1, "differentiably warped"): out(u) = I(u + F(u)), bilinear,
 * pixel centres at integer indices.  flow points at (F_x, F_y) of pixel p at
 * flow[p * fstride]; the sample position x + F_x is split into the integer
 * x + floor(F_x) and the weight F_x - floor(F_x) (the same point; it keeps the
 * weights independent of x).  Taps clamp to the border or wrap. */
void oracle_warp(const double *img, int H, int W, int C, const double *flow, int fstride,
                 int circ, double *out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double *F = flow + ((size_t)y * W + x) * fstride;
            double fx = F[0], fy = F[1];
            if (!circ) { /* beyond the border every tap clamps to the same pixel */
                double lim = (double)(W > H ? W : H) + 4.0;
                fx = fx < -lim ? -lim : (fx > lim ? lim : fx);
                fy = fy < -lim ? -lim : (fy > lim ? lim : fy);
            }
            double flx = floor(fx), fly = floor(fy), lx = fx - flx, ly = fy - fly;
            int64_t x0 = x + (int64_t)flx, y0 = y + (int64_t)fly, x1 = x0 + 1, y1 = y0 + 1;
            if (circ) { x0 = wrapi(x0, W); x1 = wrapi(x1, W); y0 = wrapi(y0, H); y1 = wrapi(y1, H); }
            else { x0 = clampi(x0, W); x1 = clampi(x1, W); y0 = clampi(y0, H); y1 = clampi(y1, H); }
            for (int c = 0; c < C; ++c) {
                double a = img[((size_t)y0 * W + x0) * C + c], bb = img[((size_t)y0 * W + x1) * C + c];
                double cc = img[((size_t)y1 * W + x0) * C + c], d = img[((size_t)y1 * W + x1) * C + c];
                out[((size_t)y * W + x) * C + c] =
                    (1.0 - ly) * ((1.0 - lx) * a + lx * bb) + ly * ((1.0 - lx) * cc + lx * d);
            }
        }
}

static inline double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Mask blend (Eq. 1 / Eq. 2): out = M a + (1 - M) b with M given directly. */
void oracle_blend(const double *a, const double *b, const double *M, long npix, int C, double *out) {
    for (long p = 0; p < npix; ++p)
        for (int c = 0; c < C; ++c)
            out[p * C + c] = M[p] * a[p * C + c] + (1.0 - M[p]) * b[p * C + c];
}

/* ------------------------------------------------------------------------- */
/* Forward.                                                                    */

typedef struct { const float *w, *b; const layer_t *L; } lw_t;

static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

/* Run one layer; returns a new tensor of size (Ho, Wo, Co). */
static double *run_layer(const lw_t *lw, const double *in, int H, int W, int circ, int *Ho, int *Wo) {
    const layer_t *L = lw->L;
    double *out;
    if (L->kind == L_CONV) {
        *Ho = (H + 2 - 3) / L->stride + 1; *Wo = (W + 2 - 3) / L->stride + 1;
        out = dalloc((size_t)*Ho * *Wo * L->co);
        oracle_conv3x3(in, H, W, L->ci, lw->w, lw->b, L->co, L->stride, circ, L->relu, out);
    } else {
        *Ho = 2 * H; *Wo = 2 * W;
        out = dalloc((size_t)*Ho * *Wo * L->co);
        oracle_convT(in, H, W, L->ci, lw->w, lw->b, L->co, circ, L->relu, out);
    }
    return out;
}

/* Channel concatenation of up to 3 tensors of the same H x W. */
static double *concat3(const double *a, int ca, const double *b, int cb, const double *c, int cc, size_t npix) {
    int C = ca + cb + cc;
    double *o = dalloc(npix * C);
    for (size_t p = 0; p < npix; ++p) {
        memcpy(o + p * C, a + p * ca, sizeof(double) * ca);
        if (cb) memcpy(o + p * C + ca, b + p * cb, sizeof(double) * cb);
        if (cc) memcpy(o + p * C + ca + cb, c + p * cc, sizeof(double) * cc);
    }
    return o;
}

/* VIBlock (Table 3 rows 1-5): c0, c1 (stride 2), 6 x conv, 2 x convT. */
static double *vib(const lw_t *lw, const double *x, int H, int W, int circ) {
    int h = H, w = W, ho, wo;
    double *cur = run_layer(&lw[0], x, h, w, circ, &ho, &wo);
    h = ho; w = wo;
    for (int k = 1; k < 10; ++k) {
        double *nx = run_layer(&lw[k], cur, h, w, circ, &ho, &wo);
        free(cur); cur = nx; h = ho; w = wo;
    }
    return cur; /* H x W x 5 */
}

/* Optional intermediate outputs (any may be NULL):
 *   vib_out[s] : Hs x Ws x 5, (F^s, logit M^s) after stage s (Hs = Hp / 2^(2-s))
 *   blend      : Hp x Wp x 3, I_blend (Eq. 1 with the final flow and mask)
 *   z          : Hp x Wp x 3, RefineNet output before the sigmoid            */
typedef struct { double *vib_out[3]; double *blend; double *z; } oracle_dumps;

int oracle_vinet_forward(const float *blob, long n_floats, const float *left, const float *right,
                         int H, int W, double t, int circ, double *out, oracle_dumps *dumps) {
    if (n_floats != oracle_n_floats()) return -1;
    if (H <= 0 || W <= 0) return -2;
    if (circ && (H % 16 || W % 16)) return -2;
    lw_t lw[N_LAYERS];
    long off = 0;
    for (int i = 0; i < N_LAYERS; ++i) {
        const layer_t *L = &LAYERS[i];
        long nw = (long)L->ci * L->co * (L->kind == L_CONV ? 9 : 16);
        lw[i].L = L; lw[i].w = blob + off; lw[i].b = blob + off + nw;
        off += nw + L->co;
    }
    const lw_t *VIBW[3] = {lw, lw + 10, lw + 20}, *CTX = lw + 30, *REF = lw + 38;

    /* Zero-pad to a multiple of 16 (Table 3's deepest level is 1/16). */
    int Hp = (H + 15) / 16 * 16, Wp = (W + 15) / 16 * 16;
    size_t np0 = (size_t)Hp * Wp;
    double *I[2] = {dalloc(np0 * 3), dalloc(np0 * 3)};
    const float *src[2] = {left, right};
    for (int s = 0; s < 2; ++s)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int c = 0; c < 3; ++c)
                    I[s][((size_t)y * Wp + x) * 3 + c] = src[s][((size_t)y * W + x) * 3 + c];

    /* Stage images: full, 1/2, 1/4 (box averages). */
    double *P[2][3];
    for (int s = 0; s < 2; ++s) {
        P[s][2] = I[s];
        P[s][1] = dalloc(np0 / 4 * 3);
        oracle_box_down(I[s], Hp, Wp, 3, 2, P[s][1]);
        P[s][0] = dalloc(np0 / 16 * 3);
        oracle_box_down(I[s], Hp, Wp, 3, 4, P[s][0]);
    }

    /* Stage 0 (VIB0 at 1/4): input [I_l, I_r, t]. */
    int h = Hp / 4, w = Wp / 4;
    size_t np = (size_t)h * w;
    double *x = dalloc(np * 7);
    for (size_t p = 0; p < np; ++p) {
        for (int c = 0; c < 3; ++c) { x[p * 7 + c] = P[0][0][p * 3 + c]; x[p * 7 + 3 + c] = P[1][0][p * 3 + c]; }
        x[p * 7 + 6] = t;
    }
    double *FM = vib(VIBW[0], x, h, w, circ); /* F^0 (4), logit M^0 */
    free(x);
    if (dumps && dumps->vib_out[0]) memcpy(dumps->vib_out[0], FM, sizeof(double) * np * 5);

    /* Stages 1, 2 (Eq. 2): upsample previous flow/mask, warp, residual. */
    for (int s = 1; s <= 2; ++s) {
        double *up = dalloc(np * 4 * 5);
        oracle_upsample2x(FM, h, w, 5, circ, up);
        free(FM);
        h *= 2; w *= 2; np = (size_t)h * w;
        for (size_t p = 0; p < np; ++p)
            for (int c = 0; c < 4; ++c) up[p * 5 + c] *= 2.0; /* flow in pixels of the finer grid */
        double *Wl = dalloc(np * 3), *Wr = dalloc(np * 3);
        oracle_warp(P[0][s], h, w, 3, up + 0, 5, circ, Wl);
        oracle_warp(P[1][s], h, w, 3, up + 2, 5, circ, Wr);
        x = dalloc(np * 18);
        for (size_t p = 0; p < np; ++p) {
            double *d = x + p * 18;
            for (int c = 0; c < 3; ++c) {
                d[c] = P[0][s][p * 3 + c]; d[3 + c] = P[1][s][p * 3 + c];
                d[6 + c] = Wl[p * 3 + c];  d[9 + c] = Wr[p * 3 + c];
            }
            d[12] = up[p * 5 + 4];
            for (int c = 0; c < 4; ++c) d[13 + c] = up[p * 5 + c];
            d[17] = t;
        }
        free(Wl); free(Wr);
        double *res = vib(VIBW[s], x, h, w, circ);
        free(x);
        FM = dalloc(np * 5);
        for (size_t p = 0; p < np * 5; ++p) FM[p] = up[p] + res[p];
        free(up); free(res);
        if (dumps && dumps->vib_out[s]) memcpy(dumps->vib_out[s], FM, sizeof(double) * np * 5);
    }

    /* Final warp + blend (Eq. 1). */
    double *Ilm = dalloc(np0 * 3), *Irm = dalloc(np0 * 3), *Ib = dalloc(np0 * 3), *M = dalloc(np0);
    oracle_warp(I[0], Hp, Wp, 3, FM + 0, 5, circ, Ilm);
    oracle_warp(I[1], Hp, Wp, 3, FM + 2, 5, circ, Irm);
    for (size_t p = 0; p < np0; ++p) M[p] = sigmoid(FM[p * 5 + 4]);
    oracle_blend(Ilm, Irm, M, (long)np0, 3, Ib);
    free(M);
    if (dumps && dumps->blend) memcpy(dumps->blend, Ib, sizeof(double) * np0 * 3);

    /* ContextNet on both original views: keep the output of every stride-1 conv. */
    double *ctx[2][4];
    const int ctxC[4] = {16, 32, 64, 128};
    for (int s = 0; s < 2; ++s) {
        double *cur = I[s];
        int hh = Hp, ww = Wp, ho, wo;
        for (int k = 0; k < 8; ++k) {
            double *nx = run_layer(&CTX[k], cur, hh, ww, circ, &ho, &wo);
            if (k % 2 == 1) { free(cur); ctx[s][k / 2] = nx; } /* free the stride-2 output */
            cur = nx; hh = ho; ww = wo;
        }
    }

    /* Flow pyramid F_k = box2(F_{k-1}) / 2 and warped context cL_k, cR_k. */
    double *warped[2][4];
    {
        double *Fk = dalloc(np0 * 5);
        memcpy(Fk, FM, sizeof(double) * np0 * 5);
        int hh = Hp, ww = Wp;
        for (int k = 0; k < 4; ++k) {
            double *nf = dalloc((size_t)hh / 2 * (ww / 2) * 5);
            oracle_box_down(Fk, hh, ww, 5, 2, nf);
            free(Fk); Fk = nf; hh /= 2; ww /= 2;
            size_t n = (size_t)hh * ww;
            for (size_t p = 0; p < n; ++p)
                for (int c = 0; c < 4; ++c) Fk[p * 5 + c] *= 0.5;
            for (int s = 0; s < 2; ++s) {
                warped[s][k] = dalloc(n * ctxC[k]);
                oracle_warp(ctx[s][k], hh, ww, ctxC[k], Fk + 2 * s, 5, circ, warped[s][k]);
            }
        }
        free(Fk);
    }

    /* RefineNet (context-aware U-Net): encoder e0..e3, decoder d0..d3, out. */
    double *e[4], *cur;
    int eh[4], ew[4], ho, wo;
    cur = concat3(Ilm, 3, Irm, 3, NULL, 0, np0);
    free(Ilm); free(Irm);
    int hh = Hp, ww = Wp;
    for (int k = 0; k < 4; ++k) {
        double *a = run_layer(&REF[2 * k], cur, hh, ww, circ, &ho, &wo);
        free(cur);
        e[k] = run_layer(&REF[2 * k + 1], a, ho, wo, circ, &ho, &wo);
        free(a);
        eh[k] = hh = ho; ew[k] = ww = wo;
        if (k < 3) {
            size_t n = (size_t)hh * ww;
            cur = concat3(e[k], REF[2 * k + 1].L->co, warped[0][k], ctxC[k], warped[1][k], ctxC[k], n);
        }
    }
    /* d0 input = [e3, cL_4, cR_4] at 1/16. */
    cur = concat3(e[3], 256, warped[0][3], 128, warped[1][3], 128, (size_t)eh[3] * ew[3]);
    double *d = run_layer(&REF[8], cur, eh[3], ew[3], circ, &ho, &wo);
    free(cur);
    int dc = REF[8].L->co;
    for (int k = 1; k < 4; ++k) { /* d_k input = [d_{k-1}, e_{3-k}] */
        int skip = 3 - k;
        size_t n = (size_t)ho * wo;
        cur = concat3(d, dc, e[skip], REF[2 * skip + 1].L->co, NULL, 0, n);
        free(d);
        d = run_layer(&REF[8 + k], cur, ho, wo, circ, &ho, &wo);
        free(cur);
        dc = REF[8 + k].L->co;
    }
    double *z = run_layer(&REF[12], d, ho, wo, circ, &ho, &wo);
    free(d);
    if (dumps && dumps->z) memcpy(dumps->z, z, sizeof(double) * np0 * 3);

    /* Residual output and crop: clamp(I_blend + 2 sigmoid(z) - 1, 0, 1). */
    for (int y = 0; y < H; ++y)
        for (int xx = 0; xx < W; ++xx)
            for (int c = 0; c < 3; ++c) {
                size_t p = ((size_t)y * Wp + xx) * 3 + c;
                double v = Ib[p] + (2.0 * sigmoid(z[p]) - 1.0);
                out[((size_t)y * W + xx) * 3 + c] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
            }

    free(z); free(Ib); free(FM);
    for (int k = 0; k < 4; ++k) {
        free(e[k]);
        for (int s = 0; s < 2; ++s) { free(ctx[s][k]); free(warped[s][k]); }
    }
    for (int s = 0; s < 2; ++s) { free(P[s][0]); free(P[s][1]); free(I[s]); }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Laplacian-pyramid loss, Eq. 3 (Sec. 3.1 "Loss functions"):                 */
/*   L_Lap = sum_{i=1..5} 2^(i-1) || L^i(I_hat) - L^i(I_gt) ||_1              */
/* The paper names a five-level Laplace pyramid and no filter; the reading:   */
/* the Burt-Adelson pyramid with the binomial kernel k = [1 4 6 4 1] / 16 and */
/* replicated edges,                                                          */
/*   G^1 = I,  G^(i+1)(y, x) = sum_{a,b} k[a] k[b] G^i(cl(2y+a-2), cl(2x+b-2)) */
/*             of size ceil(H/2) x ceil(W/2);                                 */
/*   up(G)(y, x) = sum_{a,b} 4 k[a] k[b] [y+a-2 even][x+b-2 even]             */
/*                 G(cl((y+a-2)/2), cl((x+b-2)/2)) at the finer size;          */
/*   L^i = G^i - up(G^(i+1)) for i < 5, L^5 = G^5;                            */
/*   ||.||_1 = sum of |.| over every pixel and channel of the level.          */
/* Both pyramids are built in full, then compared level by level.             */

static const double LAPK[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};

static double *lap_down(const double *g, int H, int W, int C, int *Ho, int *Wo) {
    int h = (H + 1) / 2, w = (W + 1) / 2;
    double *out = dalloc((size_t)h * w * C);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            for (int c = 0; c < C; ++c) {
                double s = 0.0;
                for (int a = 0; a < 5; ++a)
                    for (int b = 0; b < 5; ++b) {
                        int64_t yy = clampi(2 * y + a - 2, H), xx = clampi(2 * x + b - 2, W);
                        s += LAPK[a] * LAPK[b] * g[(yy * W + xx) * C + c];
                    }
                out[((size_t)y * w + x) * C + c] = s;
            }
    *Ho = h; *Wo = w;
    return out;
}

/* up(G) at the finer size H x W, G of size h x w */
static double *lap_up(const double *g, int h, int w, int C, int H, int W) {
    double *out = dalloc((size_t)H * W * C);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int c = 0; c < C; ++c) {
                double s = 0.0;
                for (int a = 0; a < 5; ++a) {
                    int yy = y + a - 2;
                    if (yy & 1) continue;               /* odd rows of the zero-inserted image */
                    for (int b = 0; b < 5; ++b) {
                        int xx = x + b - 2;
                        if (xx & 1) continue;
                        int64_t gy = clampi(yy / 2, h), gx = clampi(xx / 2, w);
                        s += 4.0 * LAPK[a] * LAPK[b] * g[(gy * w + gx) * C + c];
                    }
                }
                out[((size_t)y * W + x) * C + c] = s;
            }
    return out;
}

/* pyr[0..levels-1] = L^1 .. L^levels of img (H x W x C); sizes in hs, ws */
static void lap_pyramid(const double *img, int H, int W, int C, int levels, double **pyr, int *hs, int *ws) {
    double *g = dalloc((size_t)H * W * C);
    memcpy(g, img, sizeof(double) * H * W * C);
    int h = H, w = W;
    for (int i = 0; i < levels; ++i) {
        hs[i] = h; ws[i] = w;
        if (i == levels - 1) { pyr[i] = g; break; }        /* L^5 = G^5 */
        int h2, w2;
        double *g2 = lap_down(g, h, w, C, &h2, &w2);
        double *u = lap_up(g2, h2, w2, C, h, w);
        for (size_t k = 0; k < (size_t)h * w * C; ++k) g[k] -= u[k];   /* L^i = G^i - up(G^(i+1)) */
        free(u);
        pyr[i] = g;
        g = g2; h = h2; w = w2;
    }
}

/* Eq. 3 for one image pair; norms[i] = || L^(i+1)(a) - L^(i+1)(b) ||_1 */
double oracle_lap_loss(const double *a, const double *b, int H, int W, int C, int levels, double *norms) {
    double *pa[16], *pb[16];
    int hs[16], ws[16];
    if (levels < 1 || levels > 16) return -1.0;
    lap_pyramid(a, H, W, C, levels, pa, hs, ws);
    lap_pyramid(b, H, W, C, levels, pb, hs, ws);
    double loss = 0.0;
    for (int i = 0; i < levels; ++i) {
        double s = 0.0;
        for (size_t k = 0; k < (size_t)hs[i] * ws[i] * C; ++k) s += fabs(pa[i][k] - pb[i][k]);
        if (norms) norms[i] = s;
        loss += ldexp(s, i);                              /* 2^(i-1), i counted from 1 */
        free(pa[i]); free(pb[i]);
    }
    return loss;
}

/* The pyramid's steps, exposed for their own checks: one reduction step
 * (G^i -> G^(i+1), out ceil(H/2) x ceil(W/2)) and one expansion step (up). */
void oracle_lap_down(const double *g, int H, int W, int C, double *out) {
    int h, w;
    double *d = lap_down(g, H, W, C, &h, &w);
    memcpy(out, d, sizeof(double) * h * w * C);
    free(d);
}

void oracle_lap_up(const double *g, int h, int w, int C, int H, int W, double *out) {
    double *u = lap_up(g, h, w, C, H, W);
    memcpy(out, u, sizeof(double) * H * W * C);
    free(u);
}

/* L^1 .. L^levels of one image, concatenated level by level */
void oracle_lap_levels(const double *img, int H, int W, int C, int levels, double *out) {
    double *p[16];
    int hs[16], ws[16];
    if (levels < 1 || levels > 16) return;
    lap_pyramid(img, H, W, C, levels, p, hs, ws);
    size_t off = 0;
    for (int i = 0; i < levels; ++i) {
        size_t n = (size_t)hs[i] * ws[i] * C;
        memcpy(out + off, p[i], sizeof(double) * n);
        off += n;
        free(p[i]);
    }
}
