/*
 * diffsoup_oracle.c -- plain, slow CPU oracle for the stochastic-opacity-masked
 * rasteriser of DiffSoup (arXiv 2603.27151) and its gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header or
 * constant table with the CUDA library; both are written from the paper and
 * from the readings recorded with the project's design notes.
 *
 * Every function names the passage it restates.  Decisions that pick an
 * integer (coverage, the depth order, alpha > tau) are taken in FP32 with a
 * fixed operation order, because the GPU path takes them in FP32; gradients
 * are accumulated in FP64.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -o liboracle.so diffsoup_oracle.c -lm
 * (-ffp-contract=off: no fused multiply-add unless written as fmaf()).
 *
 * Parity status per function:
 *   or_expf / or_sigmoidf ... pinned (error bound against libm exp in double)
 *   or_philox4x32 ........... pinned (independent Philox4x32-10 implementation)
 *   or_lookup ............... pinned (linear reproduction, constant grid, texel count)
 *   or_fragment ............. pinned (watertight tiling, ray-plane depth/barycentrics)
 *   or_forward .............. pinned (z-buffer special case, background special case,
 *                             order independence, Monte Carlo selection frequencies)
 *   or_backward (tex, score)  pinned (expectation == finite differences of Eq. 7)
 *   or_backward (interior) .. pinned (finite differences at fixed visibility)
 *   or_backward (edge) ...... pinned against derivatives, not against the paper
 *                             (which prints no formula): silhouette term = finite
 *                             differences of the area-coverage loss over sub-pixel
 *                             placements (about 1%); implicit term unbiased for
 *                             the closed-form expected loss of a moving opacity
 *                             field.
 *   or_expected ............. pinned (finite differences; Monte Carlo of or_forward)
 *   or_compose .............. pinned (affine reproduction, closed-form hat function,
 *                             level-0 barycentrics, identity, constants, the FP64 sum
 *                             of the levels' hat-function expansions)
 *   or_restrict ............. pinned (adjoint identity with or_compose, hat mass)
 *   or_resample ............. pinned (up then down is the identity, affine data)
 *   or_coverage ............. pinned (brute-force count)
 *   or_edge_ratios .......... pinned (pinhole closed form, view selection)
 *   or_soup_rebuild ......... pinned (copy plan = identity; children carry the
 *                             parent's affine field, area and winding)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MODE_STOCHASTIC 0
#define OR_MODE_THRESHOLD_HALF 1

#define OR_G_TEX 1u
#define OR_G_SCORE 2u
#define OR_G_INTERIOR 4u
#define OR_G_EDGE 8u

/* ------------------------------------------------------------------------ */
/* Pinned scalar math                                                        */
/* ------------------------------------------------------------------------ */

static float o_pow2i(int k) /* 2^k for -126 <= k <= 127, built from exponent bits */
{
    uint32_t bits = (uint32_t)(k + 127) << 23;
    float f;
    memcpy(&f, &bits, 4);
    return f;
}

/* exp(x) in FP32 by Cody and Waite's argument reduction (Cody & Waite,
 * "Software Manual for the Elementary Functions", 1980): x = k ln2 + r with
 * ln2 split into a 16-bit head and a float tail, |r| <= ln2/2; e^r from its
 * degree-7 Taylor polynomial (coefficients 1/n! rounded to float) by Horner's
 * rule with fused multiply-adds; then scaled by 2^k in two exact steps so that
 * subnormal results round once. */
float or_expf(float x)
{
    if (x != x) return x;
    if (x >= 0x1.62e430p+6f) return INFINITY;     /* above ln(FLT_MAX)         */
    if (x < -0x1.9fe368p+6f) return 0.0f;         /* below ln(2^-150)          */
    const float log2e = 0x1.715476p+0f;           /* 1/ln2 rounded to float    */
    const float ln2_hi = 0x1.62e400p-1f;          /* ln2 cut to 16 bits        */
    const float ln2_lo = 0x1.7f7d1cp-20f;         /* ln2 - ln2_hi, rounded     */
    float kf = rintf(x * log2e);
    float r = fmaf(-kf, ln2_hi, x);
    r = fmaf(-kf, ln2_lo, r);
    float p = 0x1.a01a02p-13f;                    /* 1/7! */
    p = fmaf(p, r, 0x1.6c16c2p-10f);              /* 1/6! */
    p = fmaf(p, r, 0x1.111112p-7f);               /* 1/5! */
    p = fmaf(p, r, 0x1.555556p-5f);               /* 1/4! */
    p = fmaf(p, r, 0x1.555556p-3f);               /* 1/3! */
    p = fmaf(p, r, 0.5f);                         /* 1/2! */
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int k = (int)kf;
    int k1 = k / 2, k2 = k - k1;
    return (p * o_pow2i(k1)) * o_pow2i(k2);
}

/* Sigmoid activation applied to the accumulated feature grid before
 * rasterisation (Sec. 3.3, "Learnable multi-resolution triangle texture"). */
float or_sigmoidf(float th) { return 1.0f / (1.0f + or_expf(-th)); }

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications by
 * 0xD2511F53 and 0xCD9E8D57, with the Weyl key schedule 0x9E3779B9,
 * 0xBB67AE85. */
void or_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The per-fragment threshold tau_f of Eq. 5: uniform on the 2^-24 grid of
 * [0, 1), one Philox block per (pixel, triangle, group of four samples). */
static float o_tau(uint64_t seed, int px, int py, int t, int s)
{
    uint32_t ctr[4] = {(uint32_t)px, (uint32_t)py, (uint32_t)t, (uint32_t)(s >> 2)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32(ctr, key, out);
    return (float)(out[s & 3] >> 8) * 0x1p-24f;
}

float or_tau(uint64_t seed, int px, int py, int t, int s) { return o_tau(seed, px, py, t, s); }

/* ------------------------------------------------------------------------ */
/* Mesh-colour texture decode (Sec. 3.3; supplementary Fig. "texture_vis")   */
/* ------------------------------------------------------------------------ */

/* Index of grid vertex (i, j), i + j <= N: rows of constant j, i along a row. */
static int o_texel(int N, int i, int j) { return j * (N + 1) - j * (j - 1) / 2 + i; }

/* Micro-triangle containing (b1, b2) and its interpolation weights.  Grid
 * vertex (i, j) sits at barycentrics (1 - (i+j)/N, i/N, j/N).  The value is
 * a0 + wa (a1 - a0) + wb (a2 - a0), i.e. linear interpolation over the three
 * corners with weights (1 - wa - wb, wa, wb). */
static void o_cell(int N, float b1, float b2, int idx[3], float* wa, float* wb, int* lower_out)
{
    float Nf = (float)N;
    float u = Nf * b1, v = Nf * b2;
    float fi = floorf(u), fj = floorf(v);
    int i = fi < 0.0f ? 0 : (fi > (float)(N - 1) ? N - 1 : (int)fi);
    int jmax = N - 1 - i;
    int j = fj < 0.0f ? 0 : (fj > (float)jmax ? jmax : (int)fj);
    float fu = u - (float)i, fv = v - (float)j;
    int lower = (fu + fv <= 1.0f) || (i + j == N - 1);
    if (lower) {
        idx[0] = o_texel(N, i, j); idx[1] = o_texel(N, i + 1, j); idx[2] = o_texel(N, i, j + 1);
        *wa = fu; *wb = fv;
    } else {
        idx[0] = o_texel(N, i + 1, j + 1); idx[1] = o_texel(N, i, j + 1); idx[2] = o_texel(N, i + 1, j);
        *wa = 1.0f - fu; *wb = 1.0f - fv;
    }
    if (lower_out) *lower_out = lower;
}

static float o_interp(float a0, float a1, float a2, float wa, float wb)
{
    return fmaf(wb, a2 - a0, fmaf(wa, a1 - a0, a0));
}

/* Value of one channel plane (stride C between texels) at (b1, b2). */
float or_lookup(const float* grid, int N, int C, float b1, float b2)
{
    int idx[3]; float wa, wb;
    o_cell(N, b1, b2, idx, &wa, &wb, NULL);
    return o_interp(grid[(size_t)idx[0] * C], grid[(size_t)idx[1] * C], grid[(size_t)idx[2] * C], wa, wb);
}

void or_cell(int N, float b1, float b2, int32_t* idx3, float* wab)
{
    int idx[3]; float wa, wb;
    o_cell(N, b1, b2, idx, &wa, &wb, NULL);
    idx3[0] = idx[0]; idx3[1] = idx[1]; idx3[2] = idx[2];
    wab[0] = wa; wab[1] = wb;
}

/* ------------------------------------------------------------------------ */
/* Triangle set-up and fragments (Eq. 1)                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int live;                 /* 0: culled in this view                     */
    int32_t X[3], Y[3];       /* snapped screen position, 1/256 pixel units */
    int sgn;                  /* +1 / -1: orientation of the snapped points */
    float k[3];               /* (1 / w_i) / doubled area, FP32             */
    int px0, px1, py0, py1;   /* pixel rectangle that may be covered        */
} OTri;

/* Camera cam[17] = fx, fy, cx, cy, R (row-major 3x3), t, near. */
static void o_setup(const float* v9, const float* cam, int W, int H, OTri* o)
{
    const float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    const float* R = cam + 4;
    const float* tt = cam + 13;
    const float near_z = cam[16];
    float w[3];
    o->live = 1;
    for (int i = 0; i < 3; ++i) {
        const float* p = v9 + 3 * i;
        float xc = fmaf(R[0], p[0], fmaf(R[1], p[1], fmaf(R[2], p[2], tt[0])));
        float yc = fmaf(R[3], p[0], fmaf(R[4], p[1], fmaf(R[5], p[2], tt[1])));
        float zc = fmaf(R[6], p[0], fmaf(R[7], p[1], fmaf(R[8], p[2], tt[2])));
        if (!(zc > near_z)) { o->live = 0; return; }
        float sx = fmaf(fx, xc / zc, cx);
        float sy = fmaf(fy, yc / zc, cy);
        if (!(fabsf(sx) <= 16384.0f && fabsf(sy) <= 16384.0f)) { o->live = 0; return; }
        o->X[i] = (int32_t)rintf(sx * 256.0f);
        o->Y[i] = (int32_t)rintf(sy * 256.0f);
        w[i] = zc;
    }
    int64_t area = (int64_t)(o->X[1] - o->X[0]) * (o->Y[2] - o->Y[0])
                 - (int64_t)(o->X[2] - o->X[0]) * (o->Y[1] - o->Y[0]);
    if (area == 0) { o->live = 0; return; }
    o->sgn = area > 0 ? 1 : -1;
    float fa = (float)(area > 0 ? area : -area);
    for (int i = 0; i < 3; ++i) o->k[i] = (1.0f / w[i]) / fa;
    int32_t xmin = o->X[0], xmax = o->X[0], ymin = o->Y[0], ymax = o->Y[0];
    for (int i = 1; i < 3; ++i) {
        if (o->X[i] < xmin) xmin = o->X[i];
        if (o->X[i] > xmax) xmax = o->X[i];
        if (o->Y[i] < ymin) ymin = o->Y[i];
        if (o->Y[i] > ymax) ymax = o->Y[i];
    }
    /* pixel px has its centre at 256 px + 128 */
    o->px0 = (int)floor((xmin - 128) / 256.0) ; o->px1 = (int)floor((xmax - 128) / 256.0) + 1;
    o->py0 = (int)floor((ymin - 128) / 256.0) ; o->py1 = (int)floor((ymax - 128) / 256.0) + 1;
    if (o->px0 < 0) o->px0 = 0;
    if (o->py0 < 0) o->py0 = 0;
    if (o->px1 > W - 1) o->px1 = W - 1;
    if (o->py1 > H - 1) o->py1 = H - 1;
}

/* Coverage of the pixel centre by integer edge functions with the top-left
 * fill rule (interior to the right of an edge, or below a horizontal edge,
 * owns the edge).  E[] receives the oriented edge values. */
static int o_cover(const OTri* o, int px, int py, int64_t E[3])
{
    const int64_t Xp = 256 * (int64_t)px + 128, Yp = 256 * (int64_t)py + 128;
    int cov = 1;
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        int64_t e = (o->X[j] - Xp) * (o->Y[k] - Yp) - (o->X[k] - Xp) * (o->Y[j] - Yp);
        e *= o->sgn;
        int64_t gx = (int64_t)o->sgn * (o->Y[j] - o->Y[k]);   /* dE/dx */
        int64_t gy = (int64_t)o->sgn * (o->X[k] - o->X[j]);   /* dE/dy */
        int owns = gx > 0 || (gx == 0 && gy > 0);
        E[i] = e;
        if (!(e > 0 || (e == 0 && owns))) cov = 0;
    }
    return cov;
}

/* Perspective-correct inverse depth rho, depth D = 1/rho and barycentrics
 * (b1, b2) of a covered fragment, FP32 in a fixed order. */
static void o_frag(const OTri* o, const int64_t E[3], float* rho, float* D, float* b1, float* b2)
{
    float q0 = (float)E[0] * o->k[0];
    float q1 = (float)E[1] * o->k[1];
    float q2 = (float)E[2] * o->k[2];
    float r = (q0 + q1) + q2;
    float inv = 1.0f / r;
    *rho = r;
    *D = inv;
    *b1 = q1 * inv;
    *b2 = q2 * inv;
}

/* Fragment of one triangle at one pixel; returns coverage. out = rho, D, b1, b2. */
int or_fragment(const float* v9, const float* cam, int W, int H, int px, int py, float* out4)
{
    OTri o;
    o_setup(v9, cam, W, H, &o);
    if (!o.live) return 0;
    int64_t E[3];
    if (!o_cover(&o, px, py, E)) return 0;
    o_frag(&o, E, out4 + 0, out4 + 1, out4 + 2, out4 + 3);
    return 1;
}

/* (rho, t) is in front of (rho2, t2): larger inverse depth, ties to the lower index. */
static int o_front(float rho, int t, float rho2, int t2)
{
    return rho > rho2 || (rho == rho2 && t < t2);
}

static int V_of(int N) { return (N + 1) * (N + 2) / 2; }

static void o_activate(const float* tex, size_t n, float* act)
{
    for (size_t i = 0; i < n; ++i) act[i] = or_sigmoidf(tex[i]);
}

void or_activate(const float* tex, int64_t n, float* act) { o_activate(tex, (size_t)n, act); }

/* ------------------------------------------------------------------------ */
/* Object-order candidate lists (the bbox-scan mode, used to time the        */
/* oracle; results identical to the brute-force loops)                      */
/* ------------------------------------------------------------------------ */

/* Every live triangle scans the pixel rectangle of its bounding box within
 * rows [r0, r1) and appends its index to the list of each pixel there, in
 * ascending triangle order.  A pixel's list then holds exactly the
 * triangles that pass the brute-force loop's rectangle test, in the order
 * that loop visits them, so every result (and every FP64 summation order)
 * is the same.  off has (r1 - r0) W + 1 entries; returns 0, or -2 when out
 * of memory. */
typedef struct { int32_t* off; int32_t* idx; } OCand;

static int o_candidates(const OTri* tri, int T, int W, int r0, int r1, OCand* c)
{
    const size_t npix = (size_t)(r1 > r0 ? r1 - r0 : 0) * W;
    c->off = (int32_t*)calloc(npix + 1, sizeof(int32_t));
    c->idx = NULL;
    if (!c->off) return -2;
    for (int t = 0; t < T; ++t) {
        const OTri* o = &tri[t];
        if (!o->live) continue;
        const int y0 = o->py0 > r0 ? o->py0 : r0, y1 = o->py1 < r1 - 1 ? o->py1 : r1 - 1;
        for (int y = y0; y <= y1; ++y)
            for (int x = o->px0; x <= o->px1; ++x) c->off[(size_t)(y - r0) * W + x + 1]++;
    }
    for (size_t i = 0; i < npix; ++i) c->off[i + 1] += c->off[i];
    c->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(c->off[npix] > 0 ? c->off[npix] : 1));
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (npix > 0 ? npix : 1));
    if (!c->idx || !fill) {
        free(c->idx); free(fill); free(c->off);
        c->off = NULL; c->idx = NULL;
        return -2;
    }
    memcpy(fill, c->off, sizeof(int32_t) * npix);
    for (int t = 0; t < T; ++t) {
        const OTri* o = &tri[t];
        if (!o->live) continue;
        const int y0 = o->py0 > r0 ? o->py0 : r0, y1 = o->py1 < r1 - 1 ? o->py1 : r1 - 1;
        for (int y = y0; y <= y1; ++y)
            for (int x = o->px0; x <= o->px1; ++x) c->idx[fill[(size_t)(y - r0) * W + x]++] = t;
    }
    free(fill);
    return 0;
}

static void o_candidates_free(OCand* c) { free(c->off); free(c->idx); c->off = NULL; c->idx = NULL; }

/* Sigmoid of the texels of every triangle on a candidate list that has not
 * been activated yet (done[t] marks the activated ones). */
static void o_activate_candidates(const OCand* c, size_t n_entries, const float* tex, size_t VC, float* act,
                                  unsigned char* done)
{
    for (size_t i = 0; i < n_entries; ++i) {
        const int t = c->idx[i];
        if (done[t]) continue;
        o_activate(tex + (size_t)t * VC, VC, act + (size_t)t * VC);
        done[t] = 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Forward: Eq. 5 by brute force (Algorithm A1, step 1)                      */
/* ------------------------------------------------------------------------ */

/* For every view, pixel row in [row0, row1) (all rows if row1 < 0), pixel and
 * mask sample: the foremost covered fragment whose opacity exceeds its
 * threshold.  scan != 0: the per-pixel loops visit the pixel's object-order
 * candidate list (o_candidates) instead of all T triangles, and only those
 * triangles are activated; the results are identical (timing mode).  Outputs per view are concatenated: [S][H][W] for tri_id, depth,
 * n_front, n_cover; [S][H][W][2] for bary; [S][C-1][H][W] for color.
 * order (may be NULL) is the order in which triangles are visited. */
int or_forward(const float* verts, const float* tex, int32_t T, int32_t N, int32_t C,
               const float* cams, const int32_t* wh, const uint64_t* seeds, int32_t n_views,
               int32_t S, int32_t mode, const float* bg, const int32_t* order,
               int32_t row0, int32_t row1,
               int32_t* tri_id, float* bary, float* depth, int32_t* n_front, int32_t* n_cover,
               float* color, int32_t scan)
{
    const int V = V_of(N), Co = C - 1;
    float* act = (float*)malloc(sizeof(float) * (size_t)T * V * C);
    OTri* tri = (OTri*)malloc(sizeof(OTri) * (size_t)(T > 0 ? T : 1));
    unsigned char* done = scan ? (unsigned char*)calloc((size_t)(T > 0 ? T : 1), 1) : NULL;
    if (!act || !tri || (scan && !done)) { free(act); free(tri); free(done); return -2; }
    if (!scan) o_activate(tex, (size_t)T * V * C, act);
    size_t off = 0, coff = 0;
    for (int v = 0; v < n_views; ++v) {
        const int W = wh[2 * v], H = wh[2 * v + 1];
        const float* cam = cams + 17 * v;
        for (int t = 0; t < T; ++t) o_setup(verts + 9 * (size_t)t, cam, W, H, &tri[t]);
        int r0 = row1 < 0 ? 0 : row0, r1 = row1 < 0 ? H : (row1 < H ? row1 : H);
        if (r1 < r0) r1 = r0;   /* a band below this view: no rows */
        OCand cand = {NULL, NULL};
        if (scan) {
            if (o_candidates(tri, T, W, r0, r1, &cand)) { free(act); free(tri); free(done); return -2; }
            o_activate_candidates(&cand, (size_t)cand.off[(size_t)(r1 - r0) * W], tex, (size_t)V * C, act, done);
        }
        for (int s = 0; s < S; ++s)
        for (int py = r0; py < r1; ++py)
        for (int px = 0; px < W; ++px) {
            int bt = -1;
            float brho = 0.0f, bD = INFINITY, bb1 = 0.0f, bb2 = 0.0f;
            const int32_t* cl = scan ? cand.idx + cand.off[(size_t)(py - r0) * W + px] : NULL;
            const int ncand = scan ? cand.off[(size_t)(py - r0) * W + px + 1] - cand.off[(size_t)(py - r0) * W + px] : T;
            for (int n = 0; n < ncand; ++n) {
                int t = cl ? cl[n] : (order ? order[n] : n);
                const OTri* o = &tri[t];
                if (!o->live || px < o->px0 || px > o->px1 || py < o->py0 || py > o->py1) continue;
                int64_t E[3];
                if (!o_cover(o, px, py, E)) continue;
                float rho, D, b1, b2;
                o_frag(o, E, &rho, &D, &b1, &b2);
                const float* at = act + (size_t)t * V * C;
                float alpha = or_lookup(at + (C - 1), N, C, b1, b2);
                float tau = mode == OR_MODE_THRESHOLD_HALF ? 0.5f : o_tau(seeds[v], px, py, t, s);
                if (alpha > tau && (bt < 0 || o_front(rho, t, brho, bt))) {
                    bt = t; brho = rho; bD = D; bb1 = b1; bb2 = b2;
                }
            }
            int nf = 0, nc = 0;
            for (int n = 0; n < ncand; ++n) {
                const int t = cl ? cl[n] : n;
                const OTri* o = &tri[t];
                if (!o->live || px < o->px0 || px > o->px1 || py < o->py0 || py > o->py1) continue;
                int64_t E[3];
                if (!o_cover(o, px, py, E)) continue;
                float rho, D, b1, b2;
                o_frag(o, E, &rho, &D, &b1, &b2);
                ++nc;
                if (bt < 0 || o_front(rho, t, brho, bt)) ++nf;
            }
            size_t pix = off + ((size_t)s * H + py) * W + px;
            if (tri_id) tri_id[pix] = bt;
            if (depth) depth[pix] = bD;
            if (bary) { bary[2 * pix] = bb1; bary[2 * pix + 1] = bb2; }
            if (n_front) n_front[pix] = nf;
            if (n_cover) n_cover[pix] = nc;
            if (color) {
                for (int c = 0; c < Co; ++c) {
                    float val = bt < 0 ? bg[c]
                              : or_lookup(act + (size_t)bt * V * C + c, N, C, bb1, bb2);
                    color[coff + (((size_t)s * Co + c) * H + py) * W + px] = val;
                }
            }
        }
        o_candidates_free(&cand);
        off += (size_t)S * H * W;
        coff += (size_t)S * Co * H * W;
    }
    free(act);
    free(tri);
    free(done);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Continuous geometry (FP64) for the vertex gradients                       */
/* ------------------------------------------------------------------------ */

typedef struct { double x, y, z; } d3;
static d3 d3_cross(d3 a, d3 b) { d3 r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; return r; }
static double d3_dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

/* Camera-space position of a world point. */
static d3 o_to_cam(const float* cam, const float* p)
{
    const float* R = cam + 4;
    const float* tt = cam + 13;
    d3 r;
    r.x = (double)R[0] * p[0] + (double)R[1] * p[1] + (double)R[2] * p[2] + tt[0];
    r.y = (double)R[3] * p[0] + (double)R[4] * p[1] + (double)R[5] * p[2] + tt[1];
    r.z = (double)R[6] * p[0] + (double)R[7] * p[1] + (double)R[8] * p[2] + tt[2];
    return r;
}

/* Add R^T g (a camera-space gradient) to a world-space vertex gradient. */
static void o_add_world(const float* cam, d3 g, double* dst)
{
    const float* R = cam + 4;
    dst[0] += R[0] * g.x + R[3] * g.y + R[6] * g.z;
    dst[1] += R[1] * g.x + R[4] * g.y + R[7] * g.z;
    dst[2] += R[2] * g.x + R[5] * g.y + R[8] * g.z;
}

/* Direction (z = 1) of the camera ray through screen point (sx, sy), a pixel
 * centre or the midpoint of two (both exact in FP32).  The direction is
 * defined by FP32 arithmetic, ((float)sx - cx) / fx rounded once per step, so
 * that the GPU path holds the identical ray: at grazing incidence the
 * barycentrics of the hit point react strongly to the last bit of the ray. */
static d3 o_ray(const float* cam, double sx, double sy)
{
    float dx = ((float)sx - cam[2]) / cam[0];
    float dy = ((float)sy - cam[3]) / cam[1];
    d3 d = {dx, dy, 1.0};
    return d;
}

/* Barycentrics of the point where ray d meets the plane of V[0..2]:
 * beta_l = d.(V_{l+1} x V_{l+2}) / sum (Cramer's rule). nl receives the
 * numerators, the return value is their sum. */
static double o_ray_bary(const d3 V[3], d3 d, double nl[3])
{
    for (int l = 0; l < 3; ++l) nl[l] = d3_dot(d, d3_cross(V[(l + 1) % 3], V[(l + 2) % 3]));
    return nl[0] + nl[1] + nl[2];
}

/* Jacobian rows of the projection (fx X/Z + cx, fy Y/Z + cy) at camera point P. */
static void o_proj_jac(const float* cam, d3 P, d3* jx, d3* jy)
{
    jx->x = cam[0] / P.z; jx->y = 0.0; jx->z = -cam[0] * P.x / (P.z * P.z);
    jy->x = 0.0; jy->y = cam[1] / P.z; jy->z = -cam[1] * P.y / (P.z * P.z);
}

static void o_proj(const float* cam, d3 P, double* sx, double* sy)
{
    *sx = cam[0] * (P.x / P.z) + cam[2];
    *sy = cam[1] * (P.y / P.z) + cam[3];
}

/* ------------------------------------------------------------------------ */
/* Backward: Algorithm A1 step 2, Eq. 8-9, plus vertex gradients             */
/* ------------------------------------------------------------------------ */

/* Chain d(loss)/d(value) at (b1, b2) of one channel to the logits of the
 * three corner texels: value = sum_m w_m sigmoid(theta_m). */
static void o_chain_tex(double g, const float* act_t, double* gtex_t, int N, int C, int c,
                        float b1, float b2)
{
    int idx[3]; float wa, wb;
    o_cell(N, b1, b2, idx, &wa, &wb, NULL);
    double w[3] = {1.0 - (double)wa - (double)wb, (double)wa, (double)wb};
    for (int m = 0; m < 3; ++m) {
        double a = act_t[(size_t)idx[m] * C + c];
        gtex_t[(size_t)idx[m] * C + c] += g * w[m] * a * (1.0 - a);
    }
}

/* Inverse depth and triangle index of the stored winner, recomputed. */
static int o_winner_key(const OTri* tri, int t, int px, int py, float* rho)
{
    int64_t E[3];
    float D, b1, b2;
    if (t < 0 || !tri[t].live || !o_cover(&tri[t], px, py, E)) return 0;
    o_frag(&tri[t], E, rho, &D, &b1, &b2);
    return 1;
}

/* dL/d(b1, b2) of the winner's colour: sum_c g_c d value_c / d b. */
static void o_dcolor_db(const float* act_t, int N, int C, float b1, float b2, const double* g, double G[2])
{
    int idx[3]; float wa, wb; int lower;
    o_cell(N, b1, b2, idx, &wa, &wb, &lower);
    double sgn = lower ? 1.0 : -1.0;   /* wa = N b1 - i (lower) or 1 - (N b1 - i) (upper) */
    G[0] = G[1] = 0.0;
    for (int c = 0; c < C - 1; ++c) {
        double a0 = act_t[(size_t)idx[0] * C + c], a1 = act_t[(size_t)idx[1] * C + c], a2 = act_t[(size_t)idx[2] * C + c];
        G[0] += g[c] * sgn * N * (a1 - a0);
        G[1] += g[c] * sgn * N * (a2 - a0);
    }
}

int or_backward(const float* verts, const float* tex, int32_t T, int32_t N, int32_t C,
                const float* cams, const int32_t* wh, int32_t n_views, int32_t S,
                const int32_t* tri_id, const float* bary, const float* color,
                const float* grad_color, const float* score_w, uint32_t flags,
                int32_t row0, int32_t row1, double* grad_tex, double* grad_verts, int32_t scan)
{
    const int V = V_of(N), Co = C - 1;
    float* act = (float*)malloc(sizeof(float) * (size_t)T * V * C);
    OTri* tri = (OTri*)malloc(sizeof(OTri) * (size_t)(T > 0 ? T : 1));
    double* g = (double*)malloc(sizeof(double) * (size_t)(Co > 0 ? Co : 1));
    unsigned char* done = scan ? (unsigned char*)calloc((size_t)(T > 0 ? T : 1), 1) : NULL;
    if (!act || !tri || !g || (scan && !done)) { free(act); free(tri); free(g); free(done); return -2; }
    if (!scan) o_activate(tex, (size_t)T * V * C, act);
    size_t off = 0, coff = 0;
    for (int v = 0; v < n_views; ++v) {
        const int W = wh[2 * v], H = wh[2 * v + 1];
        const float* cam = cams + 17 * v;
        for (int t = 0; t < T; ++t) o_setup(verts + 9 * (size_t)t, cam, W, H, &tri[t]);
        int r0 = row1 < 0 ? 0 : row0, r1 = row1 < 0 ? H : (row1 < H ? row1 : H);
        if (r1 < r0) r1 = r0;   /* a band below this view: no rows */
        OCand cand = {NULL, NULL};
        if (scan) {
            if (o_candidates(tri, T, W, r0, r1, &cand)) { free(act); free(tri); free(g); free(done); return -2; }
            o_activate_candidates(&cand, (size_t)cand.off[(size_t)(r1 - r0) * W], tex, (size_t)V * C, act, done);
        }
        const size_t HW = (size_t)H * W;
        for (int s = 0; s < S; ++s)
        for (int py = r0; py < r1; ++py)
        for (int px = 0; px < W; ++px) {
            size_t pix = off + (size_t)s * HW + (size_t)py * W + px;
            int ts = tri_id[pix];
            float b1 = bary[2 * pix], b2 = bary[2 * pix + 1];
            for (int c = 0; c < Co; ++c)
                g[c] = grad_color[coff + ((size_t)s * Co + c) * HW + (size_t)py * W + px];

            /* Alg. A1 2(a): colour gradient of the selected fragment. */
            if ((flags & OR_G_TEX) && ts >= 0)
                for (int c = 0; c < Co; ++c)
                    o_chain_tex(g[c], act + (size_t)ts * V * C, grad_tex + (size_t)ts * V * C, N, C, c, b1, b2);

            /* Alg. A1 2(b) with Eq. 9: +l/alpha for the selected fragment,
             * -l/(1 - alpha) for every covered fragment in front of it. */
            if ((flags & OR_G_SCORE) && score_w[pix] != 0.0f) {
                double w = score_w[pix];
                float rs = 0.0f;
                int has = o_winner_key(tri, ts, px, py, &rs);
                const int32_t* cl = scan ? cand.idx + cand.off[(size_t)(py - r0) * W + px] : NULL;
                const int ncand = scan ? cand.off[(size_t)(py - r0) * W + px + 1] - cand.off[(size_t)(py - r0) * W + px] : T;
                for (int n = 0; n < ncand; ++n) {
                    const int t = cl ? cl[n] : n;
                    const OTri* o = &tri[t];
                    if (t == ts || !o->live || px < o->px0 || px > o->px1 || py < o->py0 || py > o->py1) continue;
                    int64_t E[3];
                    if (!o_cover(o, px, py, E)) continue;
                    float rho, D, fb1, fb2;
                    o_frag(o, E, &rho, &D, &fb1, &fb2);
                    if (has && !o_front(rho, t, rs, ts)) continue;
                    const float* at = act + (size_t)t * V * C;
                    double alpha = or_lookup(at + (C - 1), N, C, fb1, fb2);
                    o_chain_tex(-w / (1.0 - alpha), at, grad_tex + (size_t)t * V * C, N, C, C - 1, fb1, fb2);
                }
                if (ts >= 0) {
                    const float* at = act + (size_t)ts * V * C;
                    double alpha = or_lookup(at + (C - 1), N, C, b1, b2);
                    o_chain_tex(w / alpha, at, grad_tex + (size_t)ts * V * C, N, C, C - 1, b1, b2);
                }
            }

            /* First term of Eq. 8 for the vertices: the winner's colour moves
             * with its perspective-correct barycentrics (interior gradient). */
            if ((flags & OR_G_INTERIOR) && ts >= 0) {
                double G[3];
                double Gb[2];
                o_dcolor_db(act + (size_t)ts * V * C, N, C, b1, b2, g, Gb);
                G[0] = 0.0; G[1] = Gb[0]; G[2] = Gb[1];
                d3 Vc[3];
                for (int m = 0; m < 3; ++m) Vc[m] = o_to_cam(cam, verts + 9 * (size_t)ts + 3 * m);
                d3 d = o_ray(cam, px + 0.5, py + 0.5);
                double nl[3];
                double Ssum = o_ray_bary(Vc, d, nl);
                double gb = (G[1] * nl[1] + G[2] * nl[2]) / Ssum;
                double h[3] = {G[0] - gb, G[1] - gb, G[2] - gb};
                for (int m = 0; m < 3; ++m) {
                    int mp = (m + 1) % 3, mm = (m + 2) % 3;
                    d3 c1 = d3_cross(Vc[mp], d);      /* d N_{m-1} / d V_m */
                    d3 c2 = d3_cross(d, Vc[mm]);      /* d N_{m+1} / d V_m */
                    d3 gv = {(h[mm] * c1.x + h[mp] * c2.x) / Ssum,
                             (h[mm] * c1.y + h[mp] * c2.y) / Ssum,
                             (h[mm] * c1.z + h[mp] * c2.z) / Ssum};
                    o_add_world(cam, gv, grad_verts + 9 * (size_t)ts + 3 * m);
                }
            }

            /* Edge gradients on every horizontal and vertical pixel pair of the
             * sampled image (Sec. 3.2, "Handling visibility discontinuities"). */
            if (flags & OR_G_EDGE) {
                for (int dir = 0; dir < 2; ++dir) {
                    int qx = px + (dir == 0), qy = py + (dir == 1);
                    if (qx >= W || qy >= H) continue;
                    size_t qix = off + (size_t)s * HW + (size_t)qy * W + qx;
                    int tq = tri_id[qix];
                    if (tq == ts) continue;
                    double phi = 0.0;   /* d loss / d s for the side at p */
                    for (int c = 0; c < Co; ++c) {
                        size_t pc = coff + ((size_t)s * Co + c) * HW;
                        double gp = grad_color[pc + (size_t)py * W + px], gq = grad_color[pc + (size_t)qy * W + qx];
                        double cp = color[pc + (size_t)py * W + px], cq = color[pc + (size_t)qy * W + qx];
                        phi += 0.5 * (gp + gq) * (cp - cq);
                    }
                    for (int side = 0; side < 2; ++side) {
                        int tx = side == 0 ? ts : tq, ty = side == 0 ? tq : ts;
                        int Xx = side == 0 ? px : qx, Xy = side == 0 ? py : qy;
                        int Yx = side == 0 ? qx : px, Yy = side == 0 ? qy : py;
                        double PhiX = side == 0 ? phi : -phi;
                        double ex = (double)(Yx - Xx), ey = (double)(Yy - Xy);
                        if (tx < 0) continue;
                        const OTri* o = &tri[tx];
                        if (!o->live) continue;
                        int64_t E[3];
                        int covers = o_cover(o, Yx, Yy, E);
                        d3 Vc[3];
                        for (int m = 0; m < 3; ++m) Vc[m] = o_to_cam(cam, verts + 9 * (size_t)tx + 3 * m);
                        if (covers) {
                            float rho, D, fb1, fb2;
                            o_frag(o, E, &rho, &D, &fb1, &fb2);
                            float ry = 0.0f;
                            int hy = o_winner_key(tri, ty, Yx, Yy, &ry);
                            if (hy && !o_front(rho, tx, ry, ty)) continue;   /* occluded at Y */
                            /* implicit (mask) boundary: material point at the midpoint */
                            d3 d = o_ray(cam, 0.5 * (Xx + Yx) + 0.5, 0.5 * (Xy + Yy) + 0.5);
                            double nl[3];
                            double Ssum = o_ray_bary(Vc, d, nl);
                            d3 P = {0, 0, 0};
                            for (int m = 0; m < 3; ++m) {
                                double bm = nl[m] / Ssum;
                                P.x += bm * Vc[m].x; P.y += bm * Vc[m].y; P.z += bm * Vc[m].z;
                            }
                            d3 jx, jy;
                            o_proj_jac(cam, P, &jx, &jy);
                            d3 je = {ex * jx.x + ey * jy.x, ex * jx.y + ey * jy.y, ex * jx.z + ey * jy.z};
                            /* weight 1 per axis: the material displacement is
                             * projected on the pair axis, so the two axes
                             * see orthogonal components (no double counting) */
                            for (int m = 0; m < 3; ++m) {
                                double f = PhiX * nl[m] / Ssum;
                                d3 gv = {f * je.x, f * je.y, f * je.z};
                                o_add_world(cam, gv, grad_verts + 9 * (size_t)tx + 3 * m);
                            }
                        } else {
                            /* silhouette: the first edge the segment X->Y crosses */
                            double sx[3], sy[3];
                            for (int m = 0; m < 3; ++m) o_proj(cam, Vc[m], &sx[m], &sy[m]);
                            double area = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sx[2] - sx[0]) * (sy[1] - sy[0]);
                            double sg = area > 0 ? 1.0 : -1.0;
                            double xX = Xx + 0.5, yX = Xy + 0.5, xY = Yx + 0.5, yY = Yy + 0.5;
                            int best = -1;
                            double bs = 0.0, bfX = 0.0, bfY = 0.0;
                            for (int i = 0; i < 3; ++i) {
                                int a = (i + 1) % 3, b = (i + 2) % 3;
                                double fX = sg * ((sx[a] - xX) * (sy[b] - yX) - (sx[b] - xX) * (sy[a] - yX));
                                double fY = sg * ((sx[a] - xY) * (sy[b] - yY) - (sx[b] - xY) * (sy[a] - yY));
                                if (!(fY < 0.0 && fX > fY)) continue;
                                double si = fX / (fX - fY);
                                if (best < 0 || si < bs) { best = i; bs = si; bfX = fX; bfY = fY; }
                            }
                            if (best < 0) continue;
                            int a = (best + 1) % 3, b = (best + 2) % 3;
                            double fX = bfX * sg, fY = bfY * sg;      /* unoriented values */
                            double den = (fX - fY) * (fX - fY);
                            /* d f(x)/d a = (b_y - x_y, -(b_x - x_x)); d f(x)/d b = (-(a_y - x_y), a_x - x_x) */
                            double dfXa[2] = {sy[b] - yX, -(sx[b] - xX)}, dfYa[2] = {sy[b] - yY, -(sx[b] - xY)};
                            double dfXb[2] = {-(sy[a] - yX), sx[a] - xX}, dfYb[2] = {-(sy[a] - yY), sx[a] - xY};
                            double ux = sx[b] - sx[a], uy = sy[b] - sy[a];
                            double len2 = ux * ux + uy * uy;
                            double omega = (ex != 0.0 ? uy * uy : ux * ux) / len2;   /* squared normal component along the pair axis */
                            double k = omega * PhiX / den;
                            double gs[2][2];
                            for (int r = 0; r < 2; ++r) {
                                gs[0][r] = k * (fX * dfYa[r] - fY * dfXa[r]);
                                gs[1][r] = k * (fX * dfYb[r] - fY * dfXb[r]);
                            }
                            int vid[2] = {a, b};
                            for (int e = 0; e < 2; ++e) {
                                d3 jx, jy;
                                o_proj_jac(cam, Vc[vid[e]], &jx, &jy);
                                d3 gv = {gs[e][0] * jx.x + gs[e][1] * jy.x,
                                         gs[e][0] * jx.y + gs[e][1] * jy.y,
                                         gs[e][0] * jx.z + gs[e][1] * jy.z};
                                o_add_world(cam, gv, grad_verts + 9 * (size_t)tx + 3 * vid[e]);
                            }
                        }
                    }
                }
            }
        }
        o_candidates_free(&cand);
        off += (size_t)S * HW;
        coff += (size_t)S * Co * HW;
    }
    free(act);
    free(tri);
    free(g);
    free(done);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Closed forms: Eq. 6 / A1 selection probabilities, Eq. 7 expected loss and */
/* its exact gradient (the expectation of the Eq. 8 estimator), FP64.        */
/* ------------------------------------------------------------------------ */

typedef struct { float rho; int t; float b1, b2; } OFrag;

/* Per view: E[l] with l = sum_c (C_c - target_c)^2 over every pixel, and its
 * gradient with respect to all texture logits (colour and opacity), where the
 * selected fragment follows p(f) = alpha_f prod_{front} (1 - alpha).  The
 * visibility geometry (coverage, depth order, barycentrics) is the FP32 one of
 * or_forward; logits are FP64 and activations use libm's exp in FP64, so that
 * the result is a smooth function of the logits for finite differences. */
int or_expected(const float* verts, const double* tex, int32_t T, int32_t N, int32_t C,
                const float* cams, const int32_t* wh, int32_t n_views,
                const float* target, const float* bg, double* e_loss, double* e_grad_tex)
{
    const int V = V_of(N), Co = C - 1;
    const size_t n = (size_t)T * V * C;
    double* act = (double*)malloc(sizeof(double) * (n ? n : 1));
    OTri* tri = (OTri*)malloc(sizeof(OTri) * (size_t)(T > 0 ? T : 1));
    OFrag* fr = (OFrag*)malloc(sizeof(OFrag) * (size_t)(T > 0 ? T : 1));
    double* col = (double*)malloc(sizeof(double) * (size_t)(T + 1) * (Co > 0 ? Co : 1));
    double* al = (double*)malloc(sizeof(double) * (size_t)(T + 1));
    double* pf = (double*)malloc(sizeof(double) * (size_t)(T + 1));
    double* lf = (double*)malloc(sizeof(double) * (size_t)(T + 1));
    if (!act || !tri || !fr || !col || !al || !pf || !lf) {
        free(act); free(tri); free(fr); free(col); free(al); free(pf); free(lf); return -2;
    }
    for (size_t i = 0; i < n; ++i) act[i] = 1.0 / (1.0 + exp(-tex[i]));
    size_t toff = 0;
    for (int v = 0; v < n_views; ++v) {
        const int W = wh[2 * v], H = wh[2 * v + 1];
        const float* cam = cams + 17 * v;
        double L = 0.0;
        for (int t = 0; t < T; ++t) o_setup(verts + 9 * (size_t)t, cam, W, H, &tri[t]);
        for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int nf = 0;
            for (int t = 0; t < T; ++t) {
                const OTri* o = &tri[t];
                if (!o->live || px < o->px0 || px > o->px1 || py < o->py0 || py > o->py1) continue;
                int64_t E[3];
                if (!o_cover(o, px, py, E)) continue;
                float D;
                o_frag(o, E, &fr[nf].rho, &D, &fr[nf].b1, &fr[nf].b2);
                fr[nf].t = t;
                ++nf;
            }
            /* depth order, front first (insertion sort) */
            for (int i = 1; i < nf; ++i) {
                OFrag x = fr[i];
                int j = i - 1;
                while (j >= 0 && o_front(x.rho, x.t, fr[j].rho, fr[j].t)) { fr[j + 1] = fr[j]; --j; }
                fr[j + 1] = x;
            }
            double trans = 1.0;
            for (int i = 0; i <= nf; ++i) {
                double li = 0.0;
                for (int c = 0; c < Co; ++c) {
                    double cc;
                    if (i < nf) {
                        int idx[3]; float wa, wb;
                        o_cell(N, fr[i].b1, fr[i].b2, idx, &wa, &wb, NULL);
                        const double* at = act + (size_t)fr[i].t * V * C;
                        double a0 = at[(size_t)idx[0] * C + c], a1 = at[(size_t)idx[1] * C + c], a2 = at[(size_t)idx[2] * C + c];
                        cc = a0 + (double)wa * (a1 - a0) + (double)wb * (a2 - a0);
                    } else {
                        cc = bg[c];
                    }
                    col[(size_t)i * Co + c] = cc;
                    double d = cc - target[toff + (size_t)c * H * W + (size_t)py * W + px];
                    li += d * d;
                }
                double a = 1.0;
                if (i < nf) {
                    int idx[3]; float wa, wb;
                    o_cell(N, fr[i].b1, fr[i].b2, idx, &wa, &wb, NULL);
                    const double* at = act + (size_t)fr[i].t * V * C;
                    double a0 = at[(size_t)idx[0] * C + C - 1], a1 = at[(size_t)idx[1] * C + C - 1], a2 = at[(size_t)idx[2] * C + C - 1];
                    a = a0 + (double)wa * (a1 - a0) + (double)wb * (a2 - a0);
                }
                al[i] = a;
                pf[i] = trans * a;
                lf[i] = li;
                trans *= (1.0 - a);
                L += pf[i] * li;
            }
            if (!e_grad_tex) continue;
            /* exact gradient: sum over outcomes of p(f) [d l(C_f) + l(C_f) d log p(f)] */
            for (int i = 0; i <= nf; ++i) {
                double p = pf[i];
                if (p == 0.0) continue;
                if (i < nf) {
                    int idx[3]; float wa, wb;
                    o_cell(N, fr[i].b1, fr[i].b2, idx, &wa, &wb, NULL);
                    double w[3] = {1.0 - (double)wa - (double)wb, (double)wa, (double)wb};
                    const double* at = act + (size_t)fr[i].t * V * C;
                    double* gt = e_grad_tex + (size_t)fr[i].t * V * C;
                    for (int c = 0; c < Co; ++c) {
                        double dl = 2.0 * (col[(size_t)i * Co + c] - target[toff + (size_t)c * H * W + (size_t)py * W + px]);
                        for (int m = 0; m < 3; ++m) {
                            double a = at[(size_t)idx[m] * C + c];
                            gt[(size_t)idx[m] * C + c] += p * dl * w[m] * a * (1.0 - a);
                        }
                    }
                    for (int m = 0; m < 3; ++m) {
                        double a = at[(size_t)idx[m] * C + C - 1];
                        gt[(size_t)idx[m] * C + C - 1] += p * lf[i] / al[i] * w[m] * a * (1.0 - a);
                    }
                }
                for (int j = 0; j < i; ++j) {
                    int idx[3]; float wa, wb;
                    o_cell(N, fr[j].b1, fr[j].b2, idx, &wa, &wb, NULL);
                    double w[3] = {1.0 - (double)wa - (double)wb, (double)wa, (double)wb};
                    const double* at = act + (size_t)fr[j].t * V * C;
                    double* gt = e_grad_tex + (size_t)fr[j].t * V * C;
                    for (int m = 0; m < 3; ++m) {
                        double a = at[(size_t)idx[m] * C + C - 1];
                        gt[(size_t)idx[m] * C + C - 1] += -p * lf[i] / (1.0 - al[j]) * w[m] * a * (1.0 - a);
                    }
                }
            }
        }
        e_loss[v] = L;
        toff += (size_t)Co * H * W;
    }
    free(act); free(tri); free(fr); free(col); free(al); free(pf); free(lf);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Multi-resolution feature grids (Sec. 3.3, multi-resolution mesh colours;  */
/* supplementary "Coarse-to-Fine Optimization")                              */
/* ------------------------------------------------------------------------ */

/* Level R carries a mesh-colour grid with N_R = 2^R subdivisions per edge,
 * (2^(R-1)+1)(2^R+1) = (N_R+1)(N_R+2)/2 feature vertices; level 0 is the
 * triangle's own three vertices.  Levels r_min..r_max are stored one after
 * the other, level R as [T][V_R][C]. */
static size_t o_level_V(int R) { size_t n = (size_t)1 << R; return (n + 1) * (n + 2) / 2; }

/* Value of a level-R grid at vertex (i, j) of a grid with N = 2^k
 * subdivisions (barycentrics (1-(i+j)/N, i/N, j/N)): a vertex that coincides
 * with a vertex of the level-R grid takes its value; any other point is
 * interpolated in the micro-triangle containing it (the decode of Sec. 3.3),
 * in FP32 in the decode's order. */
static float o_level_value(const float* g, int R, int C, int c, int i, int j, int N)
{
    const int NR = 1 << R;
    if (N <= NR) return g[(size_t)o_texel(NR, i * (NR / N), j * (NR / N)) * C + c];
    const int s = N / NR;
    if (i % s == 0 && j % s == 0) return g[(size_t)o_texel(NR, i / s, j / s) * C + c];
    int idx[3]; float wa, wb;
    o_cell(NR, (float)i / (float)N, (float)j / (float)N, idx, &wa, &wb, NULL);
    return o_interp(g[(size_t)idx[0] * C + c], g[(size_t)idx[1] * C + c], g[(size_t)idx[2] * C + c], wa, wb);
}

/* Composed logits of the finest grid (Sec. 3.3: every lower-resolution grid
 * is queried and accumulated on the finest grid before rendering, then the
 * sigmoid is applied).  fine[t][v][c] is the sum over R = r_min..r_max, in
 * that order, in FP32, of level R read at vertex v = (i, j) of the finest
 * grid (barycentrics (1-(i+j)/N, i/N, j/N), N = 2^r_max) as o_level_value
 * reads it: the coinciding level vertex, else the decode's interpolation in
 * the level's micro-triangle.  The finest level contributes its own value. */
void or_compose(const float* levels, int32_t T, int32_t r_min, int32_t r_max, int32_t C, float* fine)
{
    const int Nf = 1 << r_max;
    const size_t Vf = o_level_V(r_max);
    for (int t = 0; t < T; ++t)
        for (int j = 0; j <= Nf; ++j)
            for (int i = 0; i + j <= Nf; ++i) {
                const int v = o_texel(Nf, i, j);
                for (int c = 0; c < C; ++c) {
                    float z = 0.0f;
                    size_t off = 0;
                    for (int R = r_min; R <= r_max; ++R) {
                        const float* g = levels + off + (size_t)t * o_level_V(R) * C;
                        const float val = o_level_value(g, R, C, c, i, j, Nf);
                        z = R == r_min ? val : z + val;
                        off += (size_t)T * o_level_V(R) * C;
                    }
                    fine[((size_t)t * Vf + v) * C + c] = z;
                }
            }
}

/* Adjoint of or_compose in FP64: the gradient of each level's values given
 * the gradient of the composed logits gfine [T][V_f][C].  Written as the
 * transpose of the composition: every finest vertex hands its gradient to the
 * three corners of its micro-triangle in each level with the interpolation
 * weights (1 - wa - wb, wa, wb), or to the level vertex it coincides with. */
void or_restrict(const double* gfine, int32_t T, int32_t r_min, int32_t r_max, int32_t C, double* glevels)
{
    const int Nf = 1 << r_max;
    const size_t Vf = o_level_V(r_max);
    size_t total = 0;
    for (int R = r_min; R <= r_max; ++R) total += (size_t)T * o_level_V(R) * C;
    memset(glevels, 0, sizeof(double) * total);
    for (int t = 0; t < T; ++t)
        for (int j = 0; j <= Nf; ++j)
            for (int i = 0; i + j <= Nf; ++i) {
                const int v = o_texel(Nf, i, j);
                const float b1 = (float)i / (float)Nf, b2 = (float)j / (float)Nf;
                size_t off = 0;
                for (int R = r_min; R <= r_max; ++R) {
                    double* g = glevels + off + (size_t)t * o_level_V(R) * C;
                    const double* gf = gfine + ((size_t)t * Vf + v) * C;
                    const int s = Nf >> R;
                    if (i % s == 0 && j % s == 0) {
                        const int u = o_texel(1 << R, i / s, j / s);
                        for (int c = 0; c < C; ++c) g[(size_t)u * C + c] += gf[c];
                    } else {
                        int idx[3]; float wa, wb;
                        o_cell(1 << R, b1, b2, idx, &wa, &wb, NULL);
                        const double w[3] = {1.0 - (double)wa - (double)wb, (double)wa, (double)wb};
                        for (int k = 0; k < 3; ++k)
                            for (int c = 0; c < C; ++c) g[(size_t)idx[k] * C + c] += w[k] * gf[c];
                    }
                    off += (size_t)T * o_level_V(R) * C;
                }
            }
}

/* Resampling of one level's grid onto another level (supplementary
 * "Coarse-to-Fine Optimization": the coarse feature is sampled at every grid
 * coordinate of the new level): dst vertex (i, j) of N_dst = 2^r_dst takes
 * the src grid's value at barycentrics (i/N_dst, j/N_dst), read as in
 * o_level_value; the same grid (r_src == r_dst) is copied. */
void or_resample(const float* src, int32_t T, int32_t r_src, int32_t C, float* dst, int32_t r_dst)
{
    const int Nd = 1 << r_dst;
    const size_t Vs = o_level_V(r_src), Vd = o_level_V(r_dst);
    for (int t = 0; t < T; ++t)
        for (int j = 0; j <= Nd; ++j)
            for (int i = 0; i + j <= Nd; ++i) {
                const int v = o_texel(Nd, i, j);
                const float* g = src + (size_t)t * Vs * C;
                for (int c = 0; c < C; ++c)
                    dst[((size_t)t * Vd + v) * C + c] =
                        r_src == r_dst ? g[(size_t)v * C + c]
                                       : o_level_value(g, r_src, C, c, i, j, Nd);
            }
}

/* ------------------------------------------------------------------------ */
/* Adaptive control of primitives (Sec. 3.4 "Adaptive control of            */
/* primitives"; supplementary random-initialisation procedure)               */
/* ------------------------------------------------------------------------ */

/* Pixel coverage per triangle: the number of pixel-samples of the given
 * G-buffers (tri_id planes) whose selected fragment is the triangle; counts
 * are added to `counts` [T]. */
void or_coverage(const int32_t* tri_ids, int64_t n, int32_t T, int64_t* counts)
{
    for (int64_t k = 0; k < n; ++k)
        if (tri_ids[k] >= 0 && tri_ids[k] < T) counts[tri_ids[k]] += 1;
}

/* View-space edge lengths relative to the image height: for every triangle
 * and edge e = (v_e, v_(e+1)%3), the largest over the views of the projected
 * length |pi(v_b) - pi(v_a)| / H, over the views where all three vertices lie
 * in front of the near plane and the projected triangle's bounding box meets
 * the image [0, W] x [0, H]; 0 if there is none.  FP32, projection as in the
 * set-up (Eq. 1), length sqrt(dx^2 + dy^2). */
void or_edge_ratios(const float* verts, int32_t T, const float* cams, const int32_t* wh, int32_t n_views,
                    float* out)
{
    for (int t = 0; t < T; ++t) {
        float best[3] = {0.0f, 0.0f, 0.0f};
        for (int v = 0; v < n_views; ++v) {
            const float* cam = cams + 17 * v;
            const float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
            const float* R = cam + 4;
            const float* tt = cam + 13;
            const int W = wh[2 * v], H = wh[2 * v + 1];
            float sx[3], sy[3];
            int ok = 1;
            for (int i = 0; i < 3 && ok; ++i) {
                const float* p = verts + 9 * (size_t)t + 3 * i;
                float xc = fmaf(R[0], p[0], fmaf(R[1], p[1], fmaf(R[2], p[2], tt[0])));
                float yc = fmaf(R[3], p[0], fmaf(R[4], p[1], fmaf(R[5], p[2], tt[1])));
                float zc = fmaf(R[6], p[0], fmaf(R[7], p[1], fmaf(R[8], p[2], tt[2])));
                if (!(zc > cam[16])) ok = 0;
                sx[i] = fmaf(fx, xc / zc, cx);
                sy[i] = fmaf(fy, yc / zc, cy);
            }
            if (!ok) continue;
            float x0 = fminf(sx[0], fminf(sx[1], sx[2])), x1 = fmaxf(sx[0], fmaxf(sx[1], sx[2]));
            float y0 = fminf(sy[0], fminf(sy[1], sy[2])), y1 = fmaxf(sy[0], fmaxf(sy[1], sy[2]));
            if (x1 < 0.0f || x0 > (float)W || y1 < 0.0f || y0 > (float)H) continue;
            for (int e = 0; e < 3; ++e) {
                const int a = e, b = (e + 1) % 3;
                const float dx = sx[b] - sx[a], dy = sy[b] - sy[a];
                const float r = sqrtf(fmaf(dx, dx, dy * dy)) / (float)H;
                if (r > best[e]) best[e] = r;
            }
        }
        for (int e = 0; e < 3; ++e) out[3 * (size_t)t + e] = best[e];
    }
}

/* The soup after a round of splitting and pruning.  plan[k] describes output
 * triangle k: parent << 3 | op; op 0 copies the parent; op 1 + 2e + c is
 * child c of splitting edge e = (v_e, v_(e+1)%3) at its midpoint m (child 0
 * = (v_e, m, v_(e+2)%3), child 1 = (m, v_(e+1)%3, v_(e+2)%3), the parent's
 * winding).  Each level of a child's texture is the parent's level sampled at
 * the child's grid vertices (mapped into the parent's barycentrics; a point
 * that coincides with a parent grid vertex takes its value, any other is
 * interpolated in the parent's micro-triangle, as the decode).  m = (v_a +
 * v_b) * 0.5 in FP32. */
void or_soup_rebuild(const float* verts, const float* levels, int32_t T, int32_t r_min, int32_t r_max, int32_t C,
                     const int32_t* plan, int32_t n_out, float* verts_out, float* levels_out)
{
    size_t off_in = 0, off_out = 0;
    for (int R = r_min; R <= r_max; ++R) {
        const int N = 1 << R;
        const size_t V = o_level_V(R);
        for (int k = 0; k < n_out; ++k) {
            const int p = plan[k] >> 3, op = plan[k] & 7;
            const float* g = levels + off_in + (size_t)p * V * C;
            float* d = levels_out + off_out + (size_t)k * V * C;
            /* the child's corners in the parent's barycentrics, times 2 */
            int P[3][3];
            for (int i = 0; i < 3; ++i)
                for (int q = 0; q < 3; ++q) P[i][q] = 2 * (i == q);
            if (op) {
                const int e = (op - 1) >> 1, c = (op - 1) & 1;
                const int a = e, b = (e + 1) % 3, o = (e + 2) % 3;
                int Pm[3] = {0, 0, 0};
                Pm[a] = 1; Pm[b] = 1;
                const int* c0 = c == 0 ? P[a] : Pm;
                const int* c1 = c == 0 ? Pm : P[b];
                int Q[3][3];
                for (int q = 0; q < 3; ++q) { Q[0][q] = c0[q]; Q[1][q] = c1[q]; Q[2][q] = P[o][q]; }
                memcpy(P, Q, sizeof(P));
            }
            for (int j = 0; j <= N; ++j)
                for (int i = 0; i + j <= N; ++i) {
                    /* parent position in units of 1/(2N): components 1 and 2 */
                    const int X = (N - i - j) * P[0][1] + i * P[1][1] + j * P[2][1];
                    const int Y = (N - i - j) * P[0][2] + i * P[1][2] + j * P[2][2];
                    const int v = o_texel(N, i, j);
                    for (int ch = 0; ch < C; ++ch) {
                        float val;
                        if (X % 2 == 0 && Y % 2 == 0) {
                            val = g[(size_t)o_texel(N, X / 2, Y / 2) * C + ch];
                        } else {
                            int idx[3]; float wa, wb;
                            o_cell(N, (float)X / (float)(2 * N), (float)Y / (float)(2 * N), idx, &wa, &wb, NULL);
                            val = o_interp(g[(size_t)idx[0] * C + ch], g[(size_t)idx[1] * C + ch],
                                           g[(size_t)idx[2] * C + ch], wa, wb);
                        }
                        d[(size_t)v * C + ch] = val;
                    }
                }
        }
        off_in += (size_t)T * V * C;
        off_out += (size_t)n_out * V * C;
    }
    for (int k = 0; k < n_out; ++k) {
        const int p = plan[k] >> 3, op = plan[k] & 7;
        const float* s = verts + 9 * (size_t)p;
        float* d = verts_out + 9 * (size_t)k;
        if (!op) { memcpy(d, s, 9 * sizeof(float)); continue; }
        const int e = (op - 1) >> 1, c = (op - 1) & 1;
        const int a = e, b = (e + 1) % 3, o = (e + 2) % 3;
        float m[3];
        for (int q = 0; q < 3; ++q) m[q] = (s[3 * a + q] + s[3 * b + q]) * 0.5f;
        const float* c0 = c == 0 ? s + 3 * a : m;
        const float* c1 = c == 0 ? m : s + 3 * b;
        memcpy(d, c0, 3 * sizeof(float));
        memcpy(d + 3, c1, 3 * sizeof(float));
        memcpy(d + 6, s + 3 * o, 3 * sizeof(float));
    }
}
