/*
 * Plain FP64 CPU oracle of DeGraF detection and RLOF tracking (arXiv 1901.09971).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct statement of
 * what the CUDA library computes. Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load it. The product path never calls
 * it, shares no code, header, table or helper with it, and fails loudly instead of
 * falling back to it.
 *
 * Every loop follows the definition in the paper's order and notation:
 *   - DeGraF: one key-point per window of a sliding grid with step delta
 *     (Section 2, "Point detection"); positive centroid Eq. 1, negative centroid
 *     Eq. 2 with weights 1 + m - I where m is the window maximum; the key-point is
 *     the centroid with the larger weight sum (text after Eq. 2).
 *   - RLOF: robust local optical flow (Section 2, "Sparse point tracking", and the
 *     parameter paragraph of Section 3). The paper gives no formulas for it, so
 *     this file states the reading used (pyramid, gradients, Hampel norm,
 *     illumination model, stopping rule) in the comments of each function.
 *   - EPIC interpolation of the sparse flow (Section 2, "Interpolation"; k from
 *     Section 3 "Parameters"): the reading is stated above oracle_epic_interpolate.
 *
 * Parity pins live in tests/test_oracle_*.py; functions without an independent pin
 * are marked "parity unpinned" below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_TRACKED = 0, OR_OOB = 1, OR_SMALL_EIG = 2, OR_SINGULAR = 3, OR_MAXITER = 4 };

/* ------------------------------------------------------------------ DeGraF */

/* Windows fully inside the image along one axis (Section 2: the window moves with
 * step delta; only positions where the whole window fits are used). */
static long grid_count(int n, int win, int step)
{
    if (n < win || win < 1 || step < 1) return 0;
    return (long)((n - win) / step) + 1;
}

long oracle_degraf_count(int W, int H, int win_w, int win_h, int step)
{
    return grid_count(W, win_w, step) * grid_count(H, win_h, step);
}

/*
 * One key-point per window, row-major over window positions (v outer, u inner).
 * Window (u, v) has its top-left pixel at (u*step, v*step); inside it i is the row
 * and j the column (Eq. 1-2). The image axis convention is x = column, y = row.
 *   S_pos = sum I,            C_pos = (sum j I, sum i I) / S_pos             (Eq. 1)
 *   m = max I over the window
 *   S_neg = sum (1+m-I),      C_neg = (sum j (1+m-I), sum i (1+m-I)) / S_neg (Eq. 2)
 *   key-point = C_neg if S_neg > S_pos, else C_pos (ties keep C_pos)
 * The point is returned in image coordinates: window origin + centroid, pixel
 * centres at integers.
 * sums (nullable, [N][7]) receives S_pos, sum j I, sum i I, m, S_neg, sum j (1+m-I),
 * sum i (1+m-I); neg (nullable, [N]) receives 1 where C_neg was chosen.
 */
int oracle_degraf_detect(const uint8_t* img, int W, int H, int pitch, int win_w, int win_h,
                         int step, double* pts, int64_t* sums, uint8_t* neg)
{
    if (!img || W < 1 || H < 1 || pitch < W || win_w < 1 || win_h < 1 || step < 1) return -1;
    long nu = grid_count(W, win_w, step), nv = grid_count(H, win_h, step);
    for (long v = 0; v < nv; ++v) {
        for (long u = 0; u < nu; ++u) {
            long k = v * nu + u;
            long ox = u * step, oy = v * step;
            int64_t S = 0, X = 0, Y = 0, m = 0;
            for (int i = 0; i < win_h; ++i)
                for (int j = 0; j < win_w; ++j) {
                    int64_t I = img[(oy + i) * (long)pitch + ox + j];
                    S += I;
                    X += (int64_t)j * I;
                    Y += (int64_t)i * I;
                    if (I > m) m = I;
                }
            int64_t Sn = 0, Xn = 0, Yn = 0;
            for (int i = 0; i < win_h; ++i)
                for (int j = 0; j < win_w; ++j) {
                    int64_t inv = 1 + m - (int64_t)img[(oy + i) * (long)pitch + ox + j];
                    Sn += inv;
                    Xn += (int64_t)j * inv;
                    Yn += (int64_t)i * inv;
                }
            int use_neg = Sn > S;
            double cx = use_neg ? (double)Xn / (double)Sn : (double)X / (double)S;
            double cy = use_neg ? (double)Yn / (double)Sn : (double)Y / (double)S;
            pts[2 * k + 0] = (double)ox + cx;
            pts[2 * k + 1] = (double)oy + cy;
            if (sums) {
                int64_t* o = sums + 7 * k;
                o[0] = S; o[1] = X; o[2] = Y; o[3] = m; o[4] = Sn; o[5] = Xn; o[6] = Yn;
            }
            if (neg) neg[k] = (uint8_t)use_neg;
        }
    }
    return 0;
}

/* ----------------------------------------------------------------- Pyramid */
/*
 * The paper names RLOF's image pyramid but does not define it. Reading used:
 * level 0 is the frame; level l+1 has size floor(W_l/2) x floor(H_l/2) and each
 * pixel is the mean of its 2x2 block, ((a+b)+(c+d)) * 0.25. Spatial gradients at
 * every level are the Sobel kernels divided by 8,
 *   Ix = [-1 0 1; -2 0 2; -1 0 1] / 8,  Iy = its transpose,
 * with coordinates clamped to the level's border.
 * Layout of `out`: for each level l in order, the planes I_l, Ix_l, Iy_l, each
 * W_l*H_l doubles, row-major.
 */
static void level_size(int W, int H, int l, int* Wl, int* Hl)
{
    int w = W, h = H;
    for (int k = 0; k < l; ++k) { w /= 2; h /= 2; }
    *Wl = w;
    *Hl = h;
}

long oracle_pyramid_size(int W, int H, int levels)
{
    long total = 0;
    for (int l = 0; l < levels; ++l) {
        int Wl, Hl;
        level_size(W, H, l, &Wl, &Hl);
        total += 3L * Wl * Hl;
    }
    return total;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_pyramid(const double* img, int W, int H, int levels, double* out)
{
    if (!img || !out || W < 1 || H < 1 || levels < 1) return -1;
    double* lev = out;
    const double* prev = NULL;
    int Wp = 0;
    for (int l = 0; l < levels; ++l) {
        int Wl, Hl;
        level_size(W, H, l, &Wl, &Hl);
        if (Wl < 1 || Hl < 1) return -1;
        double* I = lev;
        double* Ix = lev + (long)Wl * Hl;
        double* Iy = Ix + (long)Wl * Hl;
        for (int y = 0; y < Hl; ++y)
            for (int x = 0; x < Wl; ++x) {
                if (l == 0) {
                    I[(long)y * Wl + x] = img[(long)y * W + x];
                } else {
                    double a = prev[(long)(2 * y) * Wp + 2 * x];
                    double b = prev[(long)(2 * y) * Wp + 2 * x + 1];
                    double c = prev[(long)(2 * y + 1) * Wp + 2 * x];
                    double d = prev[(long)(2 * y + 1) * Wp + 2 * x + 1];
                    I[(long)y * Wl + x] = ((a + b) + (c + d)) * 0.25;
                }
            }
        static const int sobel_x[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
        for (int y = 0; y < Hl; ++y)
            for (int x = 0; x < Wl; ++x) {
                double gx = 0.0, gy = 0.0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        double v = I[(long)clampi(y + dy, 0, Hl - 1) * Wl + clampi(x + dx, 0, Wl - 1)];
                        gx += sobel_x[dy + 1][dx + 1] * v;
                        gy += sobel_x[dx + 1][dy + 1] * v; /* transposed kernel */
                    }
                Ix[(long)y * Wl + x] = gx / 8.0;
                Iy[(long)y * Wl + x] = gy / 8.0;
            }
        prev = I;
        Wp = Wl;
        lev += 3L * Wl * Hl;
    }
    return 0;
}

/* -------------------------------------------------------------------- RLOF */

/*
 * Arithmetic type of the tracking iteration (template sampling, residuals, robust
 * weights, normal equations, solve and update). It is double: this is the FP64
 * oracle. The test suite also compiles this file a second time with
 * -DORACLE_REAL=float, which rounds every tracking quantity to FP32 while taking
 * exactly the same steps; comparing that build with the FP64 one measures how far
 * FP32 rounding alone moves the iteration, the basis of the GPU parity bars. Pyramid
 * values are exact dyadic fractions in both types. Every literal below is cast to
 * `real` so that the FP32 build never computes in double.
 */
#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;
#define R(x) ((real)(x))

typedef struct {
    int levels;     /* pyramid levels, level 0 included */
    int radius;     /* support is (2 radius + 1)^2 pixels */
    int max_iter;   /* Gauss-Newton iterations per level */
    int model;      /* 2: translation only; 4: translation + gain/offset illumination */
    double eps;     /* stop when the translation update is shorter than eps (px) */
    double hampel_a, hampel_b, hampel_c; /* robust norm knots, 0 < a <= b < c */
    double min_eig; /* minimum eigenvalue of the gradient matrix per support pixel */
    double cross_tau; /* adaptive cross-based support threshold (intensity levels); <= 0: square support */
} oracle_rlof_params;

/*
 * Continuous three-part Hampel influence function (the robust norm of RLOF; the
 * paper names the method but not the norm, so this is the reading used):
 *   psi(r) = r                                  |r| <= a
 *          = a sgn(r)                           a < |r| <= b
 *          = a sgn(r) (c - |r|) / (c - b)       b < |r| <= c
 *          = 0                                  |r| > c
 */
static real hampel_psi(real r, real a, real b, real c)
{
    real ar = fabs(r), s = r < 0 ? R(-1) : R(1);
    if (ar <= a) return r;
    if (ar <= b) return a * s;
    if (ar <= c) return a * s * (c - ar) / (c - b);
    return R(0);
}

double oracle_hampel_psi(double r, double a, double b, double c)
{
    return (double)hampel_psi(R(r), R(a), R(b), R(c));
}

/* IRLS weight psi(r) / r, equal to 1 at r = 0. */
static real hampel_weight(real r, real a, real b, real c)
{
    if (fabs(r) <= a) return R(1);
    return hampel_psi(r, a, b, c) / r;
}

/* Bilinear interpolation of a W x H plane at (x, y); each of the four taps is
 * clamped to the border. */
static real bilinear(const double* P, int W, int H, real x, real y)
{
    real fx0 = floor(x), fy0 = floor(y);
    int x0 = (int)fx0, y0 = (int)fy0;
    real ax = x - fx0, ay = y - fy0;
    int xa = clampi(x0, 0, W - 1), xb = clampi(x0 + 1, 0, W - 1);
    int ya = clampi(y0, 0, H - 1), yb = clampi(y0 + 1, 0, H - 1);
    return (1 - ax) * (1 - ay) * R(P[(long)ya * W + xa]) + ax * (1 - ay) * R(P[(long)ya * W + xb])
         + (1 - ax) * ay * R(P[(long)yb * W + xa]) + ax * ay * R(P[(long)yb * W + xb]);
}

/* Cholesky solve of the n x n symmetric system A x = rhs (n <= 4). Returns 0 on a
 * non-positive pivot. */
static int cholesky_solve(int n, const real A[4][4], const real rhs[4], real x[4])
{
    real L[4][4] = {{0}};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            real s = A[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0)) return 0;
                L[i][i] = R(sqrt(s));  /* FP32 build: a double square root rounded once more is
                                           still the correctly rounded FP32 root */
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    real z[4];
    for (int i = 0; i < n; ++i) {
        real s = rhs[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * z[k];
        z[i] = s / L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        real s = z[i];
        for (int k = i + 1; k < n; ++k) s -= L[k][i] * x[k];
        x[i] = s / L[i][i];
    }
    return 1;
}

typedef struct {
    int W, H;
    const double *I, *Ix, *Iy;
} level_view;

static void pyramid_views(const double* pyr, int W, int H, int levels, level_view* v)
{
    const double* lev = pyr;
    for (int l = 0; l < levels; ++l) {
        level_size(W, H, l, &v[l].W, &v[l].H);
        long n = (long)v[l].W * v[l].H;
        v[l].I = lev;
        v[l].Ix = lev + n;
        v[l].Iy = lev + 2 * n;
        lev += 3 * n;
    }
}

/*
 * Tracks one point p (level-0 pixel coordinates) from frame 1 into frame 2.
 * Reading of RLOF used here (the paper gives only the method's name and its
 * options, Section 2 and Section 3 "Parameters"):
 *   g = 0 (or a given initial level-0 flow divided by 2^(L-1)), m = c = 0
 *   for l = L-1 .. 0:
 *     p_l = (p + 1/2) / 2^l - 1/2                      (centre-aligned pyramid map)
 *     template T_k, Tx_k, Ty_k = bilinear(I1_l, I1x_l, I1y_l) at p_l + k,
 *       k in [-r, r]^2
 *     if lambda_min(sum_k [Tx Ty]^T [Tx Ty]) / (2r+1)^2 < min_eig: SMALL_EIG, stop
 *       (with the cross-based support, cross_tau > 0: sums over the kept samples
 *       only, divided by their number, and every weight w_k below times the mask)
 *     d = 0; for it = 1 .. max_iter:
 *       q = p_l + g + d; if q is outside [0, W_l-1] x [0, H_l-1]: OOB, stop
 *       J_k = bilinear(I2_l) at q + k
 *       model 4: r_k = J_k - (1+m) T_k - c,  a_k = (Tx_k, Ty_k, -T_k, -1)
 *       model 2: r_k = J_k - T_k,            a_k = (Tx_k, Ty_k)
 *       w_k = psi(r_k) / r_k (Hampel, above)
 *       H = sum_k w_k a_k a_k^T, b = sum_k w_k a_k r_k
 *       solve H delta = -b by Cholesky (non-positive pivot: SINGULAR, stop)
 *       d += delta[0:2]; (m, c) += delta[2:4]
 *       if |delta[0:2]| < eps: converged, leave the loop
 *     if the loop ran out at level 0: status MAXITER (still a tracked point)
 *     if l > 0: g = 2 (g + d)         ((m, c) carry over unchanged)
 *   flow = g + d
 * Lost points (OOB, SMALL_EIG, SINGULAR) report flow 0 and illumination 0.
 * Returns the status; *iters counts the Gauss-Newton updates over all levels.
 */
/*
 * Adaptive cross-based support (Section 3 "Parameters": RLOF with the adaptive cross
 * based support region; the paper gives no formula, so this is the reading used).
 * Around the centre pixel c = p_l rounded half up (clamped into the level), in frame
 * 1's intensity plane of the level:
 *   the vertical arm runs from c up and down, at most r pixels each way, while each
 *   centre-column pixel differs from I(c) by at most tau;
 *   every row of the vertical arm runs left and right from its centre-column pixel
 *   a, at most r pixels each way, while each pixel differs from I(a) by at most tau.
 * Support sample k = (kx, ky) is kept (mask 1) iff pixel c + k lies in the cross: its
 * row inside the vertical arm and its column inside that row's horizontal arm.
 * Pixels outside the level are read clamped to the border. Returns the number of
 * kept samples (at least 1: the centre).
 */
static int cross_mask(const level_view* A, real plx, real ply, int r, double tau, unsigned char* mask)
{
    const int side = 2 * r + 1;
    const int cx = clampi((int)floor(plx + R(0.5)), 0, A->W - 1), cy = clampi((int)floor(ply + R(0.5)), 0, A->H - 1);
#define PIX(x, y) A->I[(long)clampi((y), 0, A->H - 1) * A->W + clampi((x), 0, A->W - 1)]
    const double vc = PIX(cx, cy);
    int up = 0, dn = 0, n = 0;
    while (up < r && fabs(PIX(cx, cy - up - 1) - vc) <= tau) ++up;
    while (dn < r && fabs(PIX(cx, cy + dn + 1) - vc) <= tau) ++dn;
    for (int ky = -r; ky <= r; ++ky) {
        int lf = -1, rt = -1;  /* row outside the vertical arm: nothing kept */
        if (ky >= -up && ky <= dn) {
            const double va = PIX(cx, cy + ky);
            lf = rt = 0;
            while (lf < r && fabs(PIX(cx - lf - 1, cy + ky) - va) <= tau) ++lf;
            while (rt < r && fabs(PIX(cx + rt + 1, cy + ky) - va) <= tau) ++rt;
        }
        for (int kx = -r; kx <= r; ++kx) {
            const int keep = lf >= 0 && kx >= -lf && kx <= rt;
            mask[(ky + r) * side + (kx + r)] = (unsigned char)keep;
            n += keep;
        }
    }
#undef PIX
    return n;
}

/* The cross mask of one point at level 0 of frame I1 (W x H doubles), for tests. */
int oracle_cross_mask(const double* I1, int W, int H, double px, double py, int r, double tau, uint8_t* mask)
{
    if (!I1 || W < 1 || H < 1 || r < 1 || r > 15 || !mask) return -1;
    level_view v = {W, H, I1, NULL, NULL};
    return cross_mask(&v, R(px), R(py), r, tau, mask);
}

static int track_point(const level_view* P1, const level_view* P2, const oracle_rlof_params* prm,
                       double px, double py, const double* init, double* flow, double* illum, int* iters)
{
    const int r = prm->radius, side = 2 * r + 1, npx = side * side;
    const int nm = prm->model == 4 ? 4 : 2;
    const real ha = R(prm->hampel_a), hb = R(prm->hampel_b), hc = R(prm->hampel_c);
    real* T = malloc(sizeof(real) * 4 * npx);
    real *Tx = T + npx, *Ty = T + 2 * npx, *Mk = T + 3 * npx;
    unsigned char* keep = malloc((size_t)npx);
    /* an initial level-0 flow u starts the coarsest level at g = u / 2^(L-1) */
    const real s0 = R(ldexp(1.0, -(prm->levels - 1)));
    real gx = init ? R(init[0]) * s0 : R(0), gy = init ? R(init[1]) * s0 : R(0), dx = 0, dy = 0, m = 0, c = 0;
    int status = OR_TRACKED;
    *iters = 0;
    for (int l = prm->levels - 1; l >= 0 && status == OR_TRACKED; --l) {
        const level_view* A = &P1[l];
        const level_view* B = &P2[l];
        real scale = R(ldexp(1.0, -l));
        real plx = (R(px) + R(0.5)) * scale - R(0.5), ply = (R(py) + R(0.5)) * scale - R(0.5);
        /* support mask: the cross (tau > 0) or the whole square */
        int n_keep = npx;
        if (prm->cross_tau > 0)
            n_keep = cross_mask(A, plx, ply, r, prm->cross_tau, keep);
        else
            memset(keep, 1, (size_t)npx);
        real G00 = 0, G01 = 0, G11 = 0;
        for (int ky = -r; ky <= r; ++ky)
            for (int kx = -r; kx <= r; ++kx) {
                int s = (ky + r) * side + (kx + r);
                T[s] = bilinear(A->I, A->W, A->H, plx + kx, ply + ky);
                Tx[s] = bilinear(A->Ix, A->W, A->H, plx + kx, ply + ky);
                Ty[s] = bilinear(A->Iy, A->W, A->H, plx + kx, ply + ky);
                Mk[s] = keep[s];
                G00 += Mk[s] * Tx[s] * Tx[s];
                G01 += Mk[s] * Tx[s] * Ty[s];
                G11 += Mk[s] * Ty[s] * Ty[s];
            }
        real half_tr = R(0.5) * (G00 + G11), half_df = R(0.5) * (G00 - G11);
        real lam_min = half_tr - R(sqrt(half_df * half_df + G01 * G01));
        if (lam_min / n_keep < R(prm->min_eig)) { status = OR_SMALL_EIG; break; }
        dx = dy = 0;
        int converged = 0;
        for (int it = 0; it < prm->max_iter; ++it) {
            real qx = plx + gx + dx, qy = ply + gy + dy;
            if (!(qx >= 0 && qx <= B->W - 1 && qy >= 0 && qy <= B->H - 1)) { status = OR_OOB; break; }
            real Hm[4][4] = {{0}}, bv[4] = {0};
            for (int ky = -r; ky <= r; ++ky)
                for (int kx = -r; kx <= r; ++kx) {
                    int s = (ky + r) * side + (kx + r);
                    real J = bilinear(B->I, B->W, B->H, qx + kx, qy + ky);
                    real res, a[4];
                    if (nm == 4) {
                        res = J - (1 + m) * T[s] - c;
                        a[0] = Tx[s]; a[1] = Ty[s]; a[2] = -T[s]; a[3] = R(-1);
                    } else {
                        res = J - T[s];
                        a[0] = Tx[s]; a[1] = Ty[s];
                    }
                    real w = Mk[s] * hampel_weight(res, ha, hb, hc);
                    for (int i = 0; i < nm; ++i) {
                        for (int j = 0; j < nm; ++j) Hm[i][j] += w * a[i] * a[j];
                        bv[i] += w * a[i] * res;
                    }
                }
            real rhs[4], delta[4];
            for (int i = 0; i < nm; ++i) rhs[i] = -bv[i];
            if (!cholesky_solve(nm, Hm, rhs, delta)) { status = OR_SINGULAR; break; }
            dx += delta[0];
            dy += delta[1];
            if (nm == 4) { m += delta[2]; c += delta[3]; }
            ++*iters;
            if (R(sqrt(delta[0] * delta[0] + delta[1] * delta[1])) < R(prm->eps)) { converged = 1; break; }
        }
        if (status != OR_TRACKED) break;
        if (l > 0) {
            gx = 2 * (gx + dx);
            gy = 2 * (gy + dy);
        } else if (!converged) {
            status = OR_MAXITER;
        }
    }
    free(T);
    free(keep);
    if (status == OR_TRACKED || status == OR_MAXITER) {
        flow[0] = (double)(gx + dx);
        flow[1] = (double)(gy + dy);
        if (illum) { illum[0] = (double)m; illum[1] = (double)c; }
    } else {
        flow[0] = flow[1] = 0;
        if (illum) illum[0] = illum[1] = 0;
    }
    return status;
}

static int rlof_params_ok(const oracle_rlof_params* p)
{
    return p && p->levels >= 1 && p->levels <= 12 && p->radius >= 1 && p->radius <= 15 &&
           p->max_iter >= 1 && (p->model == 2 || p->model == 4) && p->eps >= 0 &&
           p->hampel_a > 0 && p->hampel_b >= p->hampel_a && p->hampel_c > p->hampel_b;
}

/*
 * Tracks n points from frame I1 to frame I2 (both W x H doubles, row-major).
 * init_flow [n][2] (nullable): an initial level-0 flow per point (the global-motion
 * prior); NULL starts every point at zero motion.
 * Outputs: flow [n][2], status [n], iters [n] (nullable), illum [n][2] (gain m and
 * offset c; nullable). nthreads <= 0 uses the OpenMP default.
 */
int oracle_rlof_track_init(const double* I1, const double* I2, int W, int H, const double* pts, int n,
                           const oracle_rlof_params* prm, const double* init_flow, double* flow,
                           uint8_t* status, int32_t* iters, double* illum, int nthreads)
{
    if (!I1 || !I2 || W < 1 || H < 1 || n < 0 || (n > 0 && (!pts || !flow || !status)) ||
        !rlof_params_ok(prm))
        return -1;
    long sz = oracle_pyramid_size(W, H, prm->levels);
    double* pyr1 = malloc(sizeof(double) * sz);
    double* pyr2 = malloc(sizeof(double) * sz);
    level_view v1[12], v2[12];
    int rc = 0;
    if (!pyr1 || !pyr2 || oracle_pyramid(I1, W, H, prm->levels, pyr1) ||
        oracle_pyramid(I2, W, H, prm->levels, pyr2)) {
        rc = -1;
        goto done;
    }
    pyramid_views(pyr1, W, H, prm->levels, v1);
    pyramid_views(pyr2, W, H, prm->levels, v2);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int k = 0; k < n; ++k) {
        int it = 0;
        status[k] = (uint8_t)track_point(v1, v2, prm, pts[2 * k], pts[2 * k + 1],
                                         init_flow ? init_flow + 2 * k : NULL, flow + 2 * k,
                                         illum ? illum + 2 * k : NULL, &it);
        if (iters) iters[k] = it;
    }
done:
    free(pyr1);
    free(pyr2);
    return rc;
}

/*
 * Tracking on given pyramids (both in the layout of oracle_pyramid, levels prm->levels,
 * frame 1 with its gradient planes; frame 2's gradient planes are not read): the same
 * iteration as oracle_rlof_track_init, for pyramids whose values were rounded to a
 * storage format (FP16 storage) before tracking.
 */
int oracle_rlof_track_pyr(const double* pyr1, const double* pyr2, int W, int H, const double* pts, int n,
                          const oracle_rlof_params* prm, double* flow, uint8_t* status, int32_t* iters,
                          double* illum, int nthreads)
{
    if (!pyr1 || !pyr2 || W < 1 || H < 1 || n < 0 || (n > 0 && (!pts || !flow || !status)) ||
        !rlof_params_ok(prm))
        return -1;
    level_view v1[12], v2[12];
    pyramid_views(pyr1, W, H, prm->levels, v1);
    pyramid_views(pyr2, W, H, prm->levels, v2);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int k = 0; k < n; ++k) {
        int it = 0;
        status[k] = (uint8_t)track_point(v1, v2, prm, pts[2 * k], pts[2 * k + 1], NULL, flow + 2 * k,
                                         illum ? illum + 2 * k : NULL, &it);
        if (iters) iters[k] = it;
    }
    return 0;
}

int oracle_rlof_track(const double* I1, const double* I2, int W, int H, const double* pts, int n,
                      const oracle_rlof_params* prm, double* flow, uint8_t* status, int32_t* iters,
                      double* illum, int nthreads)
{
    return oracle_rlof_track_init(I1, I2, W, H, pts, n, prm, NULL, flow, status, iters, illum, nthreads);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------- DeGraF adjoint */

/*
 * DeGraF on a real-valued image (same definition as oracle_degraf_detect, FP64
 * sums). Used to take finite differences of the key-points; argmax ties resolve to
 * the first pixel in row-major order.
 */
int oracle_degraf_detect_f64(const double* img, int W, int H, int win_w, int win_h, int step, double* pts)
{
    if (!img || W < 1 || H < 1 || win_w < 1 || win_h < 1 || step < 1) return -1;
    long nu = grid_count(W, win_w, step), nv = grid_count(H, win_h, step);
    for (long v = 0; v < nv; ++v)
        for (long u = 0; u < nu; ++u) {
            long k = v * nu + u, ox = u * step, oy = v * step;
            double S = 0, X = 0, Y = 0, m = -1e300;
            for (int i = 0; i < win_h; ++i)
                for (int j = 0; j < win_w; ++j) {
                    double I = img[(oy + i) * (long)W + ox + j];
                    S += I; X += j * I; Y += i * I;
                    if (I > m) m = I;
                }
            double Sn = 0, Xn = 0, Yn = 0;
            for (int i = 0; i < win_h; ++i)
                for (int j = 0; j < win_w; ++j) {
                    double inv = 1 + m - img[(oy + i) * (long)W + ox + j];
                    Sn += inv; Xn += j * inv; Yn += i * inv;
                }
            int use_neg = Sn > S;
            pts[2 * k] = ox + (use_neg ? Xn / Sn : X / S);
            pts[2 * k + 1] = oy + (use_neg ? Yn / Sn : Y / S);
        }
    return 0;
}

/*
 * Vector-Jacobian product of DeGraF: grad_img += sum over key-points k of
 * grad_pts[k] . d(point_k)/d(img), valid wherever the selection and the window
 * maximum are locally constant. From Eq. 1: d(x_pos)/dI_ij = (j - x_pos) / S_pos
 * (likewise y with i). From Eq. 2 with weights 1 + m - I: d(x_neg)/dI_ij =
 * -(j - x_neg) / S_neg, plus, on the window's first maximum pixel (where m moves
 * with I), sum_ij (j - x_neg) / S_neg. The window origin is a constant.
 */
int oracle_degraf_vjp(const double* img, int W, int H, int win_w, int win_h, int step, const double* grad_pts,
                      double* grad_img)
{
    if (!img || !grad_pts || !grad_img || W < 1 || H < 1 || win_w < 1 || win_h < 1 || step < 1) return -1;
    long nu = grid_count(W, win_w, step), nv = grid_count(H, win_h, step);
    for (long v = 0; v < nv; ++v)
        for (long u = 0; u < nu; ++u) {
            long k = v * nu + u, ox = u * step, oy = v * step;
            double S = 0, X = 0, Y = 0, m = -1e300;
            int ai = 0, aj = 0;
            for (int i = 0; i < win_h; ++i)
                for (int j = 0; j < win_w; ++j) {
                    double I = img[(oy + i) * (long)W + ox + j];
                    S += I; X += j * I; Y += i * I;
                    if (I > m) { m = I; ai = i; aj = j; }
                }
            double Sn = 0, Xn = 0, Yn = 0;
            for (int i = 0; i < win_h; ++i)
                for (int j = 0; j < win_w; ++j) {
                    double inv = 1 + m - img[(oy + i) * (long)W + ox + j];
                    Sn += inv; Xn += j * inv; Yn += i * inv;
                }
            int use_neg = Sn > S;
            double gx = grad_pts[2 * k], gy = grad_pts[2 * k + 1];
            if (!use_neg) {
                double cx = X / S, cy = Y / S;
                for (int i = 0; i < win_h; ++i)
                    for (int j = 0; j < win_w; ++j)
                        grad_img[(oy + i) * (long)W + ox + j] += (gx * (j - cx) + gy * (i - cy)) / S;
            } else {
                double cx = Xn / Sn, cy = Yn / Sn, tot = 0;
                for (int i = 0; i < win_h; ++i)
                    for (int j = 0; j < win_w; ++j) {
                        double d = (gx * (j - cx) + gy * (i - cy)) / Sn;
                        grad_img[(oy + i) * (long)W + ox + j] -= d;
                        tot += d;
                    }
                grad_img[(oy + ai) * (long)W + ox + aj] += tot;
            }
        }
    return 0;
}

/* ------------------------------------------------------------ RLOF adjoint */

/* Derivative of the Hampel influence function (almost everywhere). */
static double hampel_dpsi(double r, double a, double b, double c)
{
    double ar = fabs(r);
    if (ar <= a) return 1.0;
    if (ar <= b) return 0.0;
    if (ar <= c) return -a / (c - b);
    return 0.0;
}

/* Solves the n x n system A x = rhs by Gaussian elimination with partial pivoting.
 * Returns 0 when A is singular. */
static int lu_solve(int n, double A[4][4], double rhs[4], double x[4])
{
    int perm[4] = {0, 1, 2, 3};
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return 0;
        if (piv != col) {
            for (int j = 0; j < n; ++j) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
            double t = rhs[col]; rhs[col] = rhs[piv]; rhs[piv] = t;
            int tp = perm[col]; perm[col] = perm[piv]; perm[piv] = tp;
        }
        for (int r = col + 1; r < n; ++r) {
            double f = A[r][col] / A[col][col];
            for (int j = col; j < n; ++j) A[r][j] -= f * A[col][j];
            rhs[r] -= f * rhs[col];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = rhs[i];
        for (int j = i + 1; j < n; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return 1;
}

/* Adds w * value at the four (clamped) bilinear taps of (x, y) in a W x H plane. */
static void scatter_bilinear(double* G, int W, int H, double x, double y, double value)
{
    double fx0 = floor(x), fy0 = floor(y);
    int x0 = (int)fx0, y0 = (int)fy0;
    double ax = x - fx0, ay = y - fy0;
    int xa = clampi(x0, 0, W - 1), xb = clampi(x0 + 1, 0, W - 1);
    int ya = clampi(y0, 0, H - 1), yb = clampi(y0 + 1, 0, H - 1);
    G[(long)ya * W + xa] += (1 - ax) * (1 - ay) * value;
    G[(long)ya * W + xb] += ax * (1 - ay) * value;
    G[(long)yb * W + xa] += (1 - ax) * ay * value;
    G[(long)yb * W + xb] += ax * ay * value;
}

/*
 * Vector-Jacobian product of RLOF tracking by implicit differentiation at the
 * converged level-0 state theta = (d, m, c) (the tracker's reading as in
 * oracle_rlof_track). The fixed point satisfies F(theta; I1, I2) = sum_k psi(r_k)
 * a_k = 0, so d(theta)/dI = -A^-1 dF/dI with A = dF/dtheta = sum_k psi'(r_k) a_k
 * s_k^T, s_k = dr_k/dtheta = (dJ_k/dx, dJ_k/dy, -T_k, -1) (exact derivatives of the
 * bilinear interpolant of I2). With A^T lambda = (grad_flow, grad_illum):
 *   grad_I2 += -sum_k psi'(r_k) (lambda . a_k) dJ_k/dI2
 *   grad_I1 += -sum_k [ mu_T dT_k/dI1 + psi(r_k) (lambda_0 dTx_k/dI1 + lambda_1 dTy_k/dI1) ]
 *     with mu_T = -(1+m) psi'(r_k) (lambda . a_k) - psi(r_k) lambda_2,
 * where T, Tx, Ty are bilinear samples of level-0 I1 and its Sobel/8 gradients (the
 * gradients' adjoint is the transposed Sobel stencil with the clamped border).
 * Model 2 drops m, c and the T, constant components. Coarse levels only choose
 * the basin, so they carry no gradient; points not TRACKED get none.
 * flow, illum, status are the forward outputs; grad_illum may be NULL.
 */
int oracle_rlof_vjp(const double* I1, const double* I2, int W, int H, const double* pts, int n,
                    const oracle_rlof_params* prm, const double* flow, const double* illum, const uint8_t* status,
                    const double* grad_flow, const double* grad_illum, double* grad_I1, double* grad_I2)
{
    /* the adjoint is defined for the square support only */
    if (!I1 || !I2 || W < 1 || H < 1 || n < 0 || !rlof_params_ok(prm) || prm->cross_tau > 0 || !grad_I1 || !grad_I2)
        return -1;
    const int r = prm->radius, nm = prm->model == 4 ? 4 : 2;
    double* gT = calloc((size_t)W * H, sizeof(double));   /* adjoint of the template plane */
    double* gTx = calloc((size_t)W * H, sizeof(double));  /* adjoint of the Sobel-x plane */
    double* gTy = calloc((size_t)W * H, sizeof(double));
    double* Ix = malloc(sizeof(double) * (size_t)W * H);
    double* Iy = malloc(sizeof(double) * (size_t)W * H);
    double* lev0 = malloc(sizeof(double) * 3 * (size_t)W * H);
    if (!gT || !gTx || !gTy || !Ix || !Iy || !lev0 || oracle_pyramid(I1, W, H, 1, lev0)) {
        free(gT); free(gTx); free(gTy); free(Ix); free(Iy); free(lev0);
        return -1;
    }
    memcpy(Ix, lev0 + (long)W * H, sizeof(double) * (size_t)W * H);
    memcpy(Iy, lev0 + 2L * W * H, sizeof(double) * (size_t)W * H);
    for (int k = 0; k < n; ++k) {
        if (status[k] != OR_TRACKED) continue;
        double px = pts[2 * k], py = pts[2 * k + 1];
        double qx = px + flow[2 * k], qy = py + flow[2 * k + 1];
        double m = nm == 4 ? illum[2 * k] : 0, c = nm == 4 ? illum[2 * k + 1] : 0;
        double A[4][4] = {{0}};
        for (int ky = -r; ky <= r; ++ky)
            for (int kx = -r; kx <= r; ++kx) {
                double T = bilinear(I1, W, H, px + kx, py + ky);
                double Tx = bilinear(Ix, W, H, px + kx, py + ky), Ty = bilinear(Iy, W, H, px + kx, py + ky);
                double x = qx + kx, y = qy + ky;
                double J = bilinear(I2, W, H, x, y);
                double fx0 = floor(x), fy0 = floor(y), ax = x - fx0, ay = y - fy0;
                int x0 = (int)fx0, y0 = (int)fy0;
                double v00 = I2[(long)clampi(y0, 0, H - 1) * W + clampi(x0, 0, W - 1)];
                double v01 = I2[(long)clampi(y0, 0, H - 1) * W + clampi(x0 + 1, 0, W - 1)];
                double v10 = I2[(long)clampi(y0 + 1, 0, H - 1) * W + clampi(x0, 0, W - 1)];
                double v11 = I2[(long)clampi(y0 + 1, 0, H - 1) * W + clampi(x0 + 1, 0, W - 1)];
                double Jx = (1 - ay) * (v01 - v00) + ay * (v11 - v10);
                double Jy = (1 - ax) * (v10 - v00) + ax * (v11 - v01);
                double res = nm == 4 ? J - (1 + m) * T - c : J - T;
                double dpsi = hampel_dpsi(res, prm->hampel_a, prm->hampel_b, prm->hampel_c);
                double a[4] = {Tx, Ty, -T, -1}, s[4] = {Jx, Jy, -T, -1};
                for (int i = 0; i < nm; ++i)
                    for (int j = 0; j < nm; ++j) A[i][j] += dpsi * a[i] * s[j];
            }
        double At[4][4], u[4] = {grad_flow[2 * k], grad_flow[2 * k + 1], 0, 0}, lam[4];
        if (nm == 4 && grad_illum) { u[2] = grad_illum[2 * k]; u[3] = grad_illum[2 * k + 1]; }
        for (int i = 0; i < nm; ++i)
            for (int j = 0; j < nm; ++j) At[i][j] = A[j][i];
        if (!lu_solve(nm, At, u, lam)) continue;
        for (int ky = -r; ky <= r; ++ky)
            for (int kx = -r; kx <= r; ++kx) {
                double T = bilinear(I1, W, H, px + kx, py + ky);
                double Tx = bilinear(Ix, W, H, px + kx, py + ky), Ty = bilinear(Iy, W, H, px + kx, py + ky);
                double x = qx + kx, y = qy + ky;
                double J = bilinear(I2, W, H, x, y);
                double res = nm == 4 ? J - (1 + m) * T - c : J - T;
                double psi = oracle_hampel_psi(res, prm->hampel_a, prm->hampel_b, prm->hampel_c);
                double dpsi = hampel_dpsi(res, prm->hampel_a, prm->hampel_b, prm->hampel_c);
                double la = lam[0] * Tx + lam[1] * Ty + (nm == 4 ? -lam[2] * T - lam[3] : 0.0);
                scatter_bilinear(grad_I2, W, H, x, y, -dpsi * la);
                double muT = nm == 4 ? -(1 + m) * dpsi * la - psi * lam[2] : -dpsi * la;
                scatter_bilinear(gT, W, H, px + kx, py + ky, -muT);
                scatter_bilinear(gTx, W, H, px + kx, py + ky, -psi * lam[0]);
                scatter_bilinear(gTy, W, H, px + kx, py + ky, -psi * lam[1]);
            }
    }
    /* I1 adjoint: the template plane directly, the gradient planes through the
     * transposed Sobel / 8 stencil (each output pixel's taps are clamped). */
    static const int sobel_x[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long o = (long)y * W + x;
            grad_I1[o] += gT[o];
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    long t = (long)clampi(y + dy, 0, H - 1) * W + clampi(x + dx, 0, W - 1);
                    grad_I1[t] += (sobel_x[dy + 1][dx + 1] * gTx[o] + sobel_x[dx + 1][dy + 1] * gTy[o]) / 8.0;
                }
        }
    free(gT); free(gTx); free(gTy); free(Ix); free(Iy); free(lev0);
    return 0;
}

/* ------------------------------------------------------ global-motion prior */

/*
 * Global-motion prior (Section 3 "Parameters": RLOF with the global motion model,
 * RLOF(IM-GM); the paper gives no formula, so the model is read as a global affine
 * motion q = A p + t fitted robustly to a first pass of tracked points and used as
 * every point's initial flow for a second pass).
 *
 * Affine parameters a[6]: q_x = a0 x + a1 y + a2, q_y = a3 x + a4 y + a5.
 * Points used: status TRACKED (converged) only; q_i = p_i + flow_i.
 * Iteratively reweighted least squares, iterations k = 0 .. iters-1:
 *   k = 0: all weights 1 (least squares);
 *   k > 0: e_i = |A p_i + t - q_i| with the previous estimate, Tukey biweight
 *          w_i = (1 - (e_i / c_k)^2)^2 for e_i < c_k, else 0,
 *          c_k = max(c_min, c0 / 2^(k-1));
 *   minimise sum w_i |A p_i + t - q_i|^2: the x and y rows share the normal matrix
 *   M = sum w [x y 1]^T [x y 1] with right-hand sides sum w [x y 1]^T q_x, q_y,
 *   solved by Cholesky.
 * A step with fewer than 3 weighted points or a singular normal matrix (a pivot
 * below 1e-10 of its diagonal entry) keeps the previous estimate and ends the
 * iterations. Returns 0 on success, 1 when no
 * estimate was made (then a = identity motion), -1 on bad arguments.
 */
/* Cholesky solve of the 3 x 3 normal equations; a pivot below 1e-10 of its
 * diagonal entry (collinear or repeated points) counts as singular: returns 0. */
static int solve3(const double M[3][3], const double b[3], double x[3])
{
    double L[3][3] = {{0}}, z[3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = M[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 1e-10 * M[i][i])) return 0;
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    for (int i = 0; i < 3; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * z[k];
        z[i] = s / L[i][i];
    }
    for (int i = 2; i >= 0; --i) {
        double s = z[i];
        for (int k = i + 1; k < 3; ++k) s -= L[k][i] * x[k];
        x[i] = s / L[i][i];
    }
    return 1;
}

int oracle_gm_fit_affine(const double* pts, const double* flow, const uint8_t* status, int n, int iters,
                         double c0, double c_min, double* a)
{
    if (!a || n < 0 || (n > 0 && (!pts || !flow || !status)) || iters < 1 || !(c0 > 0) || !(c_min > 0)) return -1;
    const double ident[6] = {1, 0, 0, 0, 1, 0};
    for (int i = 0; i < 6; ++i) a[i] = ident[i];
    int made = 0;
    for (int k = 0; k < iters; ++k) {
        const double ck = fmax(c_min, ldexp(c0, -(k - 1)));
        double M[3][3] = {{0}}, bx[3] = {0}, by[3] = {0};
        int used = 0;
        for (int i = 0; i < n; ++i) {
            if (status[i] != OR_TRACKED) continue;
            const double x = pts[2 * i], y = pts[2 * i + 1];
            const double qx = x + flow[2 * i], qy = y + flow[2 * i + 1];
            double w = 1.0;
            if (k > 0) {
                const double ex = a[0] * x + a[1] * y + a[2] - qx, ey = a[3] * x + a[4] * y + a[5] - qy;
                const double e = sqrt(ex * ex + ey * ey);
                if (e >= ck) continue;
                const double u = 1.0 - (e / ck) * (e / ck);
                w = u * u;
            }
            const double v[3] = {x, y, 1.0};
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c) M[r][c] += w * v[r] * v[c];
                bx[r] += w * v[r] * qx;
                by[r] += w * v[r] * qy;
            }
            ++used;
        }
        double sx[3], sy[3];
        if (used < 3 || !solve3(M, bx, sx) || !solve3(M, by, sy)) break;
        a[0] = sx[0]; a[1] = sx[1]; a[2] = sx[2];
        a[3] = sy[0]; a[4] = sy[1]; a[5] = sy[2];
        made = 1;
    }
    return made ? 0 : 1;
}

/* ----------------------------------------------------------- EPIC interpolation */

/*
 * Edge-preserving interpolation of the sparse flow into a dense field (Section 2,
 * "Interpolation": EPIC with an affine model fitted to the k nearest sparse
 * vectors under a geodesic distance that penalises crossing image edges, edges
 * taken from image gradients; Section 3 "Parameters": k = 128). The paper gives no
 * formulas, so this is the reading used, every distance an exact integer:
 *
 *  1. Edge cost of pixel x: C(x) = base + gain (|Gx| + |Gy|), Gx, Gy the integer
 *     Sobel responses [-1 0 1; -2 0 2; -1 0 1] (and its transpose) of frame 1 with
 *     clamped borders.
 *  2. Seeds: the matches with status TRACKED or MAXITER, each at pixel
 *     (floor(x + 1/2), floor(y + 1/2)) clamped into the image; a seed whose pixel
 *     holds a lower-index seed is not used.
 *  3. Geodesic distance on the 4-connected pixel grid, a step between neighbours x
 *     and y costing C(x) + C(y). Every pixel gets the lexicographically smallest
 *     (distance, seed index) over all seeds: distance D(x) and label s(x).
 *  4. Seed graph: 4-adjacent pixels x, y with s(x) != s(y) link the two seeds with
 *     weight D(x) + C(x) + C(y) + D(y); the edge keeps the smallest such weight.
 *  5. Neighbourhood of seed s: the k seeds with the smallest (graph distance,
 *     index), s itself first at distance 0 (all reachable seeds if fewer than k).
 *  6. Fit: weights w_t = exp(-a d_t / (2 base)) (a per flat pixel of travel).
 *     model 1 (affine): minimise sum w_t |A (p_t - p_s) + b - f_t|^2; the normal
 *     matrix M = sum w v v^T, v = (x_t - x_s, y_t - y_s, 1), is solved by Cholesky;
 *     it is used when there are at least 3 neighbours and the smallest eigenvalue
 *     of the weighted covariance of their positions is at least min_spread^2
 *     (px^2); otherwise (too few, or too close to a point or a line for a stable
 *     slope) the fit falls back to the weighted mean (A = 0). model 0: the
 *     weighted mean always.
 *  7. Dense flow of pixel x: A_s(x) (x - p_s(x)) + b_s(x); 0 where no seed exists.
 */
typedef struct {
    int k, model, cost_base, cost_gain;
    double a, min_spread;
} oracle_epic_params;

int oracle_epic_cost(const uint8_t* img, int W, int H, int base, int gain, int64_t* cost)
{
    if (!img || !cost || W < 1 || H < 1) return -1;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long gx = 0, gy = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const long v = img[(long)clampi(y + dy, 0, H - 1) * W + clampi(x + dx, 0, W - 1)];
                    const int wc = dy == 0 ? 2 : 1, wr = dx == 0 ? 2 : 1;  /* smoothing across the axis */
                    gx += dx * wc * v;
                    gy += dy * wr * v;
                }
            cost[(long)y * W + x] = base + (int64_t)gain * (labs(gx) + labs(gy));
        }
    return 0;
}

/* Binary min-heap of (d, s, v) entries ordered by (d, s). */
typedef struct {
    int64_t d;
    int32_t s, v;
} ep_item;
typedef struct {
    ep_item* a;
    long n, cap;
} ep_heap;

static int ep_less(const ep_item* x, const ep_item* y) { return x->d < y->d || (x->d == y->d && x->s < y->s); }

static int ep_push(ep_heap* h, ep_item it)
{
    if (h->n == h->cap) {
        long cap = h->cap ? 2 * h->cap : 1024;
        ep_item* a = (ep_item*)realloc(h->a, (size_t)cap * sizeof(ep_item));
        if (!a) return 0;
        h->a = a;
        h->cap = cap;
    }
    long i = h->n++;
    while (i > 0) {
        long p = (i - 1) / 2;
        if (!ep_less(&it, &h->a[p])) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i] = it;
    return 1;
}

static ep_item ep_pop(ep_heap* h)
{
    ep_item top = h->a[0], last = h->a[--h->n];
    long i = 0;
    for (;;) {
        long c = 2 * i + 1;
        if (c >= h->n) break;
        if (c + 1 < h->n && ep_less(&h->a[c + 1], &h->a[c])) ++c;
        if (!ep_less(&h->a[c], &last)) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->n > 0) h->a[i] = last;
    return top;
}

typedef struct {
    int32_t s, t;
    int64_t w;
} ep_edge;

static int ep_edge_cmp(const void* x, const void* y)
{
    const ep_edge *a = (const ep_edge*)x, *b = (const ep_edge*)y;
    if (a->s != b->s) return a->s < b->s ? -1 : 1;
    if (a->t != b->t) return a->t < b->t ? -1 : 1;
    return a->w < b->w ? -1 : (a->w > b->w);
}

int oracle_epic_interpolate(const uint8_t* img, int W, int H, const double* pts, const double* flow,
                            const uint8_t* status, int n, const oracle_epic_params* p, double* dense,
                            int32_t* labels, int64_t* dist, int32_t* knn_idx, int64_t* knn_dist,
                            int32_t* knn_count, double* models, uint8_t* fit_kind)
{
    if (!img || !p || !dense || W < 1 || H < 1 || n < 0 || (n > 0 && (!pts || !flow || !status)) || p->k < 1 ||
        (p->model != 0 && p->model != 1) || p->cost_base < 1 || p->cost_gain < 0 || !(p->a >= 0) ||
        !(p->min_spread >= 0))
        return -1;
    const long NP = (long)W * H;
    const int k = p->k;
    int64_t* C = (int64_t*)malloc((size_t)NP * sizeof(int64_t));
    int64_t* D = (int64_t*)malloc((size_t)NP * sizeof(int64_t));
    int32_t* S = (int32_t*)malloc((size_t)NP * sizeof(int32_t));
    char* done = (char*)calloc((size_t)NP, 1);
    int32_t* own = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));  /* seed's pixel, -1: not used */
    ep_heap h = {0};
    int rc = 0;
    if (!C || !D || !S || !done || !own) { rc = -2; goto out; }
    oracle_epic_cost(img, W, H, p->cost_base, p->cost_gain, C);

    /* 2-3. seeds and the multi-source geodesic distance (Dijkstra on (distance, seed)) */
    for (long i = 0; i < NP; ++i) { D[i] = INT64_MAX; S[i] = -1; }
    for (int i = 0; i < n; ++i) {
        own[i] = -1;
        if (status[i] != OR_TRACKED && status[i] != OR_MAXITER) continue;
        const int x = clampi((int)floor(pts[2 * i] + 0.5), 0, W - 1);
        const int y = clampi((int)floor(pts[2 * i + 1] + 0.5), 0, H - 1);
        const long o = (long)y * W + x;
        if (S[o] >= 0) continue;  /* a lower-index seed holds the pixel */
        S[o] = i;
        D[o] = 0;
        own[i] = (int32_t)o;
        if (!ep_push(&h, (ep_item){0, i, (int32_t)o})) { rc = -2; goto out; }
    }
    while (h.n > 0) {
        const ep_item it = ep_pop(&h);
        if (done[it.v]) continue;
        if (it.d != D[it.v] || it.s != S[it.v]) continue;  /* superseded entry */
        done[it.v] = 1;
        const int x = it.v % W, y = it.v / W;
        const int nx[4] = {x - 1, x + 1, x, x}, ny[4] = {y, y, y - 1, y + 1};
        for (int q = 0; q < 4; ++q) {
            if (nx[q] < 0 || nx[q] >= W || ny[q] < 0 || ny[q] >= H) continue;
            const long o = (long)ny[q] * W + nx[q];
            if (done[o]) continue;
            const ep_item c = {it.d + C[it.v] + C[o], it.s, (int32_t)o};
            if (S[o] < 0 || c.d < D[o] || (c.d == D[o] && c.s < S[o])) {
                D[o] = c.d;
                S[o] = c.s;
                if (!ep_push(&h, c)) { rc = -2; goto out; }
            }
        }
    }

    /* 4. seed graph: candidate links of 4-adjacent pixels in different cells, the
     * smallest weight per seed pair kept, stored both ways in CSR form */
    long ne = 0, ecap = 1024;
    ep_edge* E = (ep_edge*)malloc((size_t)ecap * sizeof(ep_edge));
    if (!E) { rc = -2; goto out; }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const long o = (long)y * W + x;
            const long nb[2] = {x + 1 < W ? o + 1 : -1, y + 1 < H ? o + W : -1};
            for (int q = 0; q < 2; ++q) {
                if (nb[q] < 0 || S[o] < 0 || S[nb[q]] < 0 || S[o] == S[nb[q]]) continue;
                const int64_t w = D[o] + C[o] + C[nb[q]] + D[nb[q]];
                if (ne + 2 > ecap) {
                    ecap *= 2;
                    ep_edge* e2 = (ep_edge*)realloc(E, (size_t)ecap * sizeof(ep_edge));
                    if (!e2) { free(E); rc = -2; goto out; }
                    E = e2;
                }
                E[ne++] = (ep_edge){S[o], S[nb[q]], w};
                E[ne++] = (ep_edge){S[nb[q]], S[o], w};
            }
        }
    qsort(E, (size_t)ne, sizeof(ep_edge), ep_edge_cmp);
    long nu = 0;  /* keep the first (smallest weight) entry of each (s, t) */
    for (long i = 0; i < ne; ++i)
        if (nu == 0 || E[i].s != E[nu - 1].s || E[i].t != E[nu - 1].t) E[nu++] = E[i];
    long* first = (long*)calloc((size_t)n + 1, sizeof(long));
    if (!first) { free(E); rc = -2; goto out; }
    for (long i = 0; i < nu; ++i) first[E[i].s + 1]++;
    for (int i = 0; i < n; ++i) first[i + 1] += first[i];

    /* 5-6. per-seed neighbourhood (Dijkstra on the seed graph, stopped after k
     * settled seeds) and the weighted fit; model of seed s in mod[6 s ..]:
     * (A00, A01, A10, A11, b0, b1) */
    double* mod = models ? models : (double*)malloc((size_t)(n > 0 ? n : 1) * 6 * sizeof(double));
    int failed = !mod;
    if (!failed)
#pragma omp parallel
    {
        ep_heap g = {0};
        int64_t* best = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        char* fin = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
        int32_t* touched = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        if (!best || !fin || !touched) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int i = 0; i < n; ++i) best[i] = INT64_MAX;
#pragma omp for schedule(dynamic, 64)
            for (int s = 0; s < n; ++s) {
                double* mo = mod + 6L * s;
                for (int j = 0; j < 6; ++j) mo[j] = 0.0;
                if (fit_kind) fit_kind[s] = 0;
                if (knn_count) knn_count[s] = 0;
                if (own[s] < 0) continue;
                int nt = 0, cnt = 0, oom = 0;
                g.n = 0;
                best[s] = 0;
                touched[nt++] = s;
                if (!ep_push(&g, (ep_item){0, s, s})) oom = 1;
                double M[3][3] = {{0}}, bu[3] = {0}, bv[3] = {0}, sw = 0, su = 0, sv = 0;
                const double xs = pts[2 * s], ys = pts[2 * s + 1];
                while (!oom && g.n > 0 && cnt < k) {
                    const ep_item it = ep_pop(&g);
                    if (fin[it.s] || it.d != best[it.s]) continue;  /* superseded entry */
                    fin[it.s] = 1;
                    const int t = it.s;
                    if (knn_idx) knn_idx[(long)s * k + cnt] = t;
                    if (knn_dist) knn_dist[(long)s * k + cnt] = it.d;
                    ++cnt;
                    const double w = exp(-p->a * (double)it.d / (2.0 * p->cost_base));
                    const double v[3] = {pts[2 * t] - xs, pts[2 * t + 1] - ys, 1.0};
                    const double fu = flow[2 * t], fv = flow[2 * t + 1];
                    for (int r = 0; r < 3; ++r) {
                        for (int c = 0; c < 3; ++c) M[r][c] += w * v[r] * v[c];
                        bu[r] += w * v[r] * fu;
                        bv[r] += w * v[r] * fv;
                    }
                    sw += w;
                    su += w * fu;
                    sv += w * fv;
                    for (long e = first[t]; e < first[t + 1]; ++e) {
                        const int u = E[e].t;
                        const int64_t d = it.d + E[e].w;
                        if (fin[u] || d >= best[u]) continue;
                        if (best[u] == INT64_MAX) touched[nt++] = u;
                        best[u] = d;
                        if (!ep_push(&g, (ep_item){d, u, u})) { oom = 1; break; }
                    }
                }
                for (int i = 0; i < nt; ++i) { best[touched[i]] = INT64_MAX; fin[touched[i]] = 0; }
                if (oom) {
#pragma omp atomic write
                    failed = 1;
                    continue;
                }
                if (knn_count) knn_count[s] = cnt;
                double xu[3] = {0, 0, 0}, xv[3] = {0, 0, 0};
                /* weighted covariance of the neighbours' positions: the Schur
                 * complement of M's constant term over sum w */
                int affine = p->model == 1 && cnt >= 3;
                if (affine) {
                    const double mx = M[0][2] / sw, my = M[1][2] / sw;
                    const double cxx = M[0][0] / sw - mx * mx, cxy = M[0][1] / sw - mx * my;
                    const double cyy = M[1][1] / sw - my * my;
                    const double h = 0.5 * (cxx - cyy);
                    const double lmin = 0.5 * (cxx + cyy) - sqrt(h * h + cxy * cxy);
                    affine = lmin >= p->min_spread * p->min_spread;
                }
                if (affine) {
                    double L[3][3] = {{0}}, zu[3], zv[3];
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j <= i; ++j) {
                            double a = M[i][j];
                            for (int q = 0; q < j; ++q) a -= L[i][q] * L[j][q];
                            if (i == j)
                                L[i][i] = sqrt(a);
                            else
                                L[i][j] = a / L[j][j];
                        }
                    for (int i = 0; i < 3; ++i) {
                        double a = bu[i], b = bv[i];
                        for (int q = 0; q < i; ++q) { a -= L[i][q] * zu[q]; b -= L[i][q] * zv[q]; }
                        zu[i] = a / L[i][i];
                        zv[i] = b / L[i][i];
                    }
                    for (int i = 2; i >= 0; --i) {
                        double a = zu[i], b = zv[i];
                        for (int q = i + 1; q < 3; ++q) { a -= L[q][i] * xu[q]; b -= L[q][i] * xv[q]; }
                        xu[i] = a / L[i][i];
                        xv[i] = b / L[i][i];
                    }
                }
                if (!affine) {
                    xu[0] = xu[1] = xv[0] = xv[1] = 0.0;
                    xu[2] = su / sw;
                    xv[2] = sv / sw;
                }
                mo[0] = xu[0]; mo[1] = xu[1]; mo[2] = xv[0]; mo[3] = xv[1]; mo[4] = xu[2]; mo[5] = xv[2];
                if (fit_kind) fit_kind[s] = affine ? 1 : 2;
            }
        }
        free(g.a); free(best); free(fin); free(touched);
    }
    free(first);
    free(E);

    /* 7. dense flow: every pixel takes its seed's model */
    if (!failed)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const long o = (long)y * W + x;
                const int s = S[o];
                if (labels) labels[o] = s;
                if (dist) dist[o] = s >= 0 ? D[o] : -1;
                if (s < 0) { dense[2 * o] = dense[2 * o + 1] = 0.0; continue; }
                const double* mo = mod + 6L * s;
                const double dx = x - pts[2 * s], dy = y - pts[2 * s + 1];
                dense[2 * o] = mo[0] * dx + mo[1] * dy + mo[4];
                dense[2 * o + 1] = mo[2] * dx + mo[3] * dy + mo[5];
            }
    if (mod != models) free(mod);
    if (failed) rc = -2;
out:
    free(h.a); free(C); free(D); free(S); free(done); free(own);
    return rc;
}
