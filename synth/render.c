/*
 * Seeded synthetic input generator: a ray-cast box room with value-noise
 * textured walls, Lambertian shading from a point light, a per-frame exposure
 * affine, Gaussian pixel noise and uint8 rounding.  It also returns exact
 * camera-z depth per pixel and at arbitrary sub-pixel positions, and picks
 * sparse map points (max-gradient pixel per grid cell).
 *
 * This module only manufactures inputs.  It holds none of the tracker's
 * arithmetic: no pyramid, no projection Jacobian, no residual, no solver.
 * Both the FP64 oracle and the CUDA path consume what it writes.
 *
 * Conventions: a camera pose T_wc is a row-major 3x4 [R|t] mapping camera
 * coordinates to world coordinates (X_w = R X_c + t).  Pinhole camera with
 * +z forward, +x right, +y down; pixel (u, v) is the ray through
 * ((u - cx)/fx, (v - cy)/fy, 1).  Pixel centres sit at integer coordinates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double lo[3], hi[3];     /* room extent, metres */
    double light[3];         /* point light position */
    double ambient;          /* ambient term of the shading, in [0,1] */
    double base_freq;        /* cycles per metre of octave 0 */
    double lacunarity;       /* frequency ratio between octaves */
    double gain;             /* amplitude ratio between octaves */
    double contrast;         /* stretch of the noise around 0.5 before clamping */
    int octaves;
    int pad_;
    uint64_t tex_seed;
} synth_scene;

static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

/* uniform in [0, 1) with 53 random bits */
static double u01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

static double lattice(uint64_t seed, int plane, int octave, int64_t i, int64_t j)
{
    uint64_t h = splitmix64(seed ^ 0x5851F42D4C957F2DULL);
    h = splitmix64(h ^ (uint64_t)(plane * 16 + octave));
    h = splitmix64(h ^ (uint64_t)i);
    h = splitmix64(h ^ ((uint64_t)j * 0x9E3779B97F4A7C15ULL));
    return u01(h);
}

static double smooth(double t) { return t * t * (3.0 - 2.0 * t); }

/* value noise in [0,1) on plane coordinates (s, t) in metres */
static double value_noise(const synth_scene* sc, int plane, double s, double t)
{
    double f = sc->base_freq, amp = 1.0, sum = 0.0, norm = 0.0;
    for (int o = 0; o < sc->octaves; ++o) {
        double x = s * f, y = t * f;
        double fx = floor(x), fy = floor(y);
        int64_t ix = (int64_t)fx, iy = (int64_t)fy;
        double ax = smooth(x - fx), ay = smooth(y - fy);
        double v00 = lattice(sc->tex_seed, plane, o, ix, iy);
        double v10 = lattice(sc->tex_seed, plane, o, ix + 1, iy);
        double v01 = lattice(sc->tex_seed, plane, o, ix, iy + 1);
        double v11 = lattice(sc->tex_seed, plane, o, ix + 1, iy + 1);
        double v0 = v00 + ax * (v10 - v00), v1 = v01 + ax * (v11 - v01);
        sum += amp * (v0 + ay * (v1 - v0));
        norm += amp;
        amp *= sc->gain;
        f *= sc->lacunarity;
    }
    return sum / norm;
}

/* Cast the camera ray of pixel (u, v); returns camera-z depth (> 0) and the
 * hit point / wall id, or -1 if the camera is outside the room. */
static double cast(const synth_scene* sc, const double T[12], double fx, double fy, double cx,
                   double cy, double u, double v, double p[3], int* wall)
{
    double dc[3] = {(u - cx) / fx, (v - cy) / fy, 1.0};
    double o[3] = {T[3], T[7], T[11]};
    double d[3];
    for (int r = 0; r < 3; ++r) d[r] = T[4 * r] * dc[0] + T[4 * r + 1] * dc[1] + T[4 * r + 2] * dc[2];
    double best = INFINITY;
    int bw = -1;
    for (int ax = 0; ax < 3; ++ax) {
        if (d[ax] > 0) {
            double s = (sc->hi[ax] - o[ax]) / d[ax];
            if (s < best) { best = s; bw = 2 * ax + 1; }
        } else if (d[ax] < 0) {
            double s = (sc->lo[ax] - o[ax]) / d[ax];
            if (s < best) { best = s; bw = 2 * ax; }
        }
    }
    if (bw < 0 || !(best > 0)) return -1.0;
    for (int r = 0; r < 3; ++r) p[r] = o[r] + best * d[r];
    *wall = bw;
    return best; /* dc has unit z, so the ray parameter is the camera z */
}

static double radiance(const synth_scene* sc, const double p[3], int wall)
{
    int ax = wall / 2;
    int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    double n = value_noise(sc, wall, p[a1], p[a2]);
    n = 0.5 + sc->contrast * (n - 0.5);
    if (n < 0) n = 0;
    if (n > 1) n = 1;
    double albedo = 0.15 + 0.7 * n;
    double nrm[3] = {0, 0, 0};
    nrm[ax] = (wall % 2 == 0) ? 1.0 : -1.0; /* inward normal */
    double l[3] = {sc->light[0] - p[0], sc->light[1] - p[1], sc->light[2] - p[2]};
    double ln = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    double c = (nrm[0] * l[0] + nrm[1] * l[1] + nrm[2] * l[2]) / ln;
    if (c < 0) c = 0;
    double shade = sc->ambient + (1.0 - sc->ambient) * c;
    /* albedo*shade lies in [0.045, 0.85]; map 0.85 -> 220 and 0 -> 30 */
    return 30.0 + 190.0 * albedo * shade / 0.85;
}

static double gauss(uint64_t seed, uint64_t idx)
{
    uint64_t h1 = splitmix64(seed ^ splitmix64(2 * idx + 1));
    uint64_t h2 = splitmix64(h1 ^ 0xD1B54A32D192ED03ULL);
    double u1 = 1.0 - u01(h1); /* (0, 1] */
    double u2 = u01(h2);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/*
 * Render one frame.  img: W*H uint8 (row-major, pitch W).  depth / rad /
 * wall_id may be NULL; when given they receive camera-z depth, the noise-free
 * exposed intensity e^a*L + b (before noise and rounding) and the id (0-5) of
 * the wall each pixel sees.
 * Returns 0, or -1 if some pixel ray leaves the room (camera outside).
 */
int synth_render(const synth_scene* sc, const double T_wc[12], double fx, double fy, double cx,
                 double cy, int W, int H, double a_t, double b_t, double sigma,
                 uint64_t noise_seed, uint8_t* img, float* depth, float* rad, uint8_t* wall_id)
{
    int bad = 0;
    double ea = exp(a_t);
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double p[3];
            int wall = 0;
            double z = cast(sc, T_wc, fx, fy, cx, cy, (double)x, (double)y, p, &wall);
            size_t i = (size_t)y * W + x;
            if (z <= 0) {
                bad = 1;
                img[i] = 0;
                if (depth) depth[i] = 0.f;
                if (rad) rad[i] = 0.f;
                if (wall_id) wall_id[i] = 255;
                continue;
            }
            double L = ea * radiance(sc, p, wall) + b_t;
            double val = L;
            if (sigma > 0) val += sigma * gauss(noise_seed, (uint64_t)i);
            double q = floor(val + 0.5);
            if (q < 0) q = 0;
            if (q > 255) q = 255;
            img[i] = (uint8_t)q;
            if (depth) depth[i] = (float)z;
            if (rad) rad[i] = (float)L;
            if (wall_id) wall_id[i] = (uint8_t)wall;
        }
    }
    return bad ? -1 : 0;
}

/* Exact camera-z depth along the ray of sub-pixel (u, v); -1 if none. */
double synth_depth_at(const synth_scene* sc, const double T_wc[12], double fx, double fy,
                      double cx, double cy, double u, double v)
{
    double p[3];
    int wall;
    return cast(sc, T_wc, fx, fy, cx, cy, u, v, p, &wall);
}

/*
 * Sparse map-point selection on a rendered frame.  The image is split into a
 * gx x gy grid; in every cell the pixel with the largest squared central
 * difference gradient (ties: lower linear index) whose depth lies in
 * [dmin, dmax], that is at least `margin` pixels from the border and whose
 * (2*plane_margin+1)^2 neighbourhood sees a single wall (so the patch does not
 * straddle a depth crease) is a candidate.  Candidates are ranked by gradient (ties: lower index) and the
 * best N kept; if fewer exist, the rest are drawn uniformly (seeded) from the
 * remaining admissible pixels.  Each chosen pixel is jittered by a seeded
 * sub-pixel offset in [-0.5, 0.5)^2 and its exact depth re-cast there.
 * Writes uvd[N*3] = (u, v, depth).  Returns the number of points written.
 */
/* 1 where the box of radius m around the pixel holds a single wall id */
static uint8_t* single_wall_mask(const uint8_t* wall, int W, int H, int m)
{
    size_t n = (size_t)W * H;
    uint8_t* mn = (uint8_t*)malloc(n);
    uint8_t* mx = (uint8_t*)malloc(n);
    uint8_t* mask = (uint8_t*)malloc(n);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint8_t a = 255, b = 0;
            for (int i = x - m; i <= x + m; ++i) {
                uint8_t v = (i < 0 || i >= W) ? 254 : wall[(size_t)y * W + i];
                if (v < a) a = v;
                if (v > b) b = v;
            }
            mn[(size_t)y * W + x] = a;
            mx[(size_t)y * W + x] = b;
        }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint8_t a = 255, b = 0;
            for (int j = y - m; j <= y + m; ++j) {
                if (j < 0 || j >= H) { a = 0; b = 255; break; }
                if (mn[(size_t)j * W + x] < a) a = mn[(size_t)j * W + x];
                if (mx[(size_t)j * W + x] > b) b = mx[(size_t)j * W + x];
            }
            mask[(size_t)y * W + x] = (uint8_t)(a == b);
        }
    free(mn);
    free(mx);
    return mask;
}

int synth_select_points(const synth_scene* sc, const double T_wc[12], double fx, double fy,
                        double cx, double cy, const uint8_t* img, const float* depth,
                        const uint8_t* wall, int W, int H, int N, double dmin, double dmax,
                        int margin, int plane_margin, uint64_t seed, float* uvd)
{
    if (N <= 0) return 0;
    uint8_t* flat = single_wall_mask(wall, W, H, plane_margin);
    int gx = (int)ceil(sqrt((double)N * W / H));
    if (gx < 1) gx = 1;
    int gy = (N + gx - 1) / gx;
    int ncell = gx * gy;
    int* cand = (int*)malloc(sizeof(int) * (size_t)ncell);
    int* gval = (int*)malloc(sizeof(int) * (size_t)ncell);
    uint8_t* taken = (uint8_t*)calloc((size_t)W * H, 1);
    int nc = 0;
    for (int cyi = 0; cyi < gy; ++cyi) {
        for (int cxi = 0; cxi < gx; ++cxi) {
            int x0 = (int)((long)cxi * W / gx), x1 = (int)((long)(cxi + 1) * W / gx);
            int y0 = (int)((long)cyi * H / gy), y1 = (int)((long)(cyi + 1) * H / gy);
            int best = -1, bg = -1;
            for (int y = y0; y < y1; ++y) {
                if (y < margin || y >= H - margin) continue;
                for (int x = x0; x < x1; ++x) {
                    if (x < margin || x >= W - margin) continue;
                    size_t i = (size_t)y * W + x;
                    if (!(depth[i] >= dmin && depth[i] <= dmax) || !flat[i]) continue;
                    int ddx = (int)img[i + 1] - (int)img[i - 1];
                    int ddy = (int)img[i + W] - (int)img[i - W];
                    int g2 = ddx * ddx + ddy * ddy;
                    if (g2 > bg) { bg = g2; best = (int)i; }
                }
            }
            if (best >= 0) { cand[nc] = best; gval[nc] = bg; ++nc; }
        }
    }
    /* rank candidates: gradient descending, index ascending (insertion sort on
     * index-sorted input keeps it simple and deterministic) */
    for (int i = 1; i < nc; ++i) {
        int c = cand[i], g = gval[i], j = i - 1;
        while (j >= 0 && (gval[j] < g || (gval[j] == g && cand[j] > c))) {
            cand[j + 1] = cand[j];
            gval[j + 1] = gval[j];
            --j;
        }
        cand[j + 1] = c;
        gval[j + 1] = g;
    }
    int n = nc < N ? nc : N;
    int* pick = (int*)malloc(sizeof(int) * (size_t)N);
    for (int i = 0; i < n; ++i) { pick[i] = cand[i]; taken[cand[i]] = 1; }
    /* fill the rest uniformly from admissible untaken pixels */
    uint64_t ctr = 0;
    long tries = 0, max_tries = 64L * W * H;
    while (n < N && tries < max_tries) {
        uint64_t h = splitmix64(seed ^ splitmix64(0xABCDEFULL + ctr++));
        int i = (int)(h % (uint64_t)((long)W * H));
        int x = i % W, y = i / W;
        ++tries;
        if (taken[i] || x < margin || x >= W - margin || y < margin || y >= H - margin) continue;
        if (!(depth[i] >= dmin && depth[i] <= dmax) || !flat[i]) continue;
        taken[i] = 1;
        pick[n++] = i;
    }
    int out = 0;
    for (int k = 0; k < n; ++k) {
        int i = pick[k];
        uint64_t h = splitmix64(seed ^ splitmix64(0x1234567ULL + (uint64_t)k));
        double ju = u01(h) - 0.5, jv = u01(splitmix64(h)) - 0.5;
        double u = (i % W) + ju, v = (i / W) + jv;
        double z = synth_depth_at(sc, T_wc, fx, fy, cx, cy, u, v);
        if (!(z >= dmin && z <= dmax)) { u = i % W; v = i / W; z = depth[i]; }
        uvd[3 * out + 0] = (float)u;
        uvd[3 * out + 1] = (float)v;
        uvd[3 * out + 2] = (float)z;
        ++out;
    }
    free(flat);
    free(pick);
    free(cand);
    free(gval);
    free(taken);
    return out;
}
