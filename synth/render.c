/* Layered-plane scene renderer used by synth/scene.py (input generation only).
 *
 * Renders one pinhole view of up to 8 axis-aligned rectangles lying in planes
 * Z = const, each carrying three channels of summed 2-D gradient noise.  All
 * random parameters (depths, extents, permutations, offsets) are drawn on the
 * Python side and passed in; this file only evaluates them per ray.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

static inline float fade(float t) { return t * t * t * (t * (t * 6.0f - 15.0f) + 10.0f); }

static const float GX[8] = {1, 1, 0, -1, -1, -1, 0, 1};
static const float GY[8] = {0, 1, 1, 1, 0, -1, -1, -1};

static float gnoise(double px, double py, const int32_t *perm) {
    double xf = floor(px), yf = floor(py);
    float fx = (float)(px - xf), fy = (float)(py - yf);
    int xi = ((int64_t)xf) & 255, yi = ((int64_t)yf) & 255;
    float u = fade(fx), v = fade(fy);
    int p0 = perm[xi], p1 = perm[xi + 1];
    int h00 = perm[p0 + yi] & 7, h10 = perm[p1 + yi] & 7;
    int h01 = perm[p0 + yi + 1] & 7, h11 = perm[p1 + yi + 1] & 7;
    float n00 = GX[h00] * fx + GY[h00] * fy;
    float n10 = GX[h10] * (fx - 1) + GY[h10] * fy;
    float n01 = GX[h01] * fx + GY[h01] * (fy - 1);
    float n11 = GX[h11] * (fx - 1) + GY[h11] * (fy - 1);
    float a = n00 + u * (n10 - n00);
    float b = n01 + u * (n11 - n01);
    return a + v * (b - a);
}

static float fbm(double px, double py, const int32_t *perm, int octaves, float persistence) {
    float tot = 0.f, amp = 1.f, norm = 0.f;
    double freq = 1.0;
    for (int o = 0; o < octaves; ++o) {
        tot += amp * gnoise(px * freq, py * freq, perm);
        norm += amp;
        amp *= persistence;
        freq *= 2.0;
    }
    return tot / norm;
}

/* planes: n_planes x 5 doubles (z, x0, x1, y0, y1); perms: n_planes*3 x 512 ints;
 * offsets: n_planes*3 x 2 doubles; out: H x W x 3 floats. */
void synth_render(int H, int W, double f, const double *pos, double yaw,
                  int n_planes, const double *planes, const int32_t *perms,
                  const double *offsets, double contrast, int octaves,
                  float persistence, float *out) {
    double c = cos(yaw), s = sin(yaw);
    double cxp = W / 2.0, cyp = H / 2.0;
    const double sub[2] = {0.25, 0.75};
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            float acc[3] = {0, 0, 0};
            for (int sy = 0; sy < 2; ++sy)
                for (int sx = 0; sx < 2; ++sx) {
                    double dx = (x + sub[sx] - cxp) / f, dy = (y + sub[sy] - cyp) / f;
                    double wx = c * dx + s, wy = dy, wz = -s * dx + c;
                    double best = INFINITY, hx = 0, hy = 0;
                    int idx = -1;
                    for (int j = 0; j < n_planes; ++j) {
                        const double *P = planes + 5 * j;
                        double t = (P[0] - pos[2]) / wz;
                        double X = pos[0] + t * wx, Y = pos[1] + t * wy;
                        if (t > 0 && X >= P[1] && X <= P[2] && Y >= P[3] && Y <= P[4] && t < best) {
                            best = t; idx = j; hx = X; hy = Y;
                        }
                    }
                    if (idx < 0) continue;
                    double freq = 10.0 / planes[5 * idx];
                    for (int ch = 0; ch < 3; ++ch) {
                        const double *o = offsets + 2 * (idx * 3 + ch);
                        float n = fbm(hx * freq + o[0], hy * freq + o[1], perms + 512 * (idx * 3 + ch),
                                      octaves, persistence);
                        float v = 0.5f + (float)contrast * n;
                        acc[ch] += v < 0.f ? 0.f : (v > 1.f ? 1.f : v);
                    }
                }
            float *dst = out + 3 * ((size_t)y * W + x);
            for (int ch = 0; ch < 3; ++ch) dst[ch] = acc[ch] * 0.25f;
        }
    }
}
