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

typedef struct {
    int levels;     /* pyramid levels, level 0 included */
    int radius;     /* support is (2 radius + 1)^2 pixels */
    int max_iter;   /* Gauss-Newton iterations per level */
    int model;      /* 2: translation only; 4: translation + gain/offset illumination */
    double eps;     /* stop when the translation update is shorter than eps (px) */
    double hampel_a, hampel_b, hampel_c; /* robust norm knots, 0 < a <= b < c */
    double min_eig; /* minimum eigenvalue of the gradient matrix per support pixel */
} oracle_rlof_params;

/*
 * Continuous three-part Hampel influence function (the robust norm of RLOF; the
 * paper names the method but not the norm, so this is the reading used):
 *   psi(r) = r                                  |r| <= a
 *          = a sgn(r)                           a < |r| <= b
 *          = a sgn(r) (c - |r|) / (c - b)       b < |r| <= c
 *          = 0                                  |r| > c
 */
double oracle_hampel_psi(double r, double a, double b, double c)
{
    double ar = fabs(r), s = r < 0 ? -1.0 : 1.0;
    if (ar <= a) return r;
    if (ar <= b) return a * s;
    if (ar <= c) return a * s * (c - ar) / (c - b);
    return 0.0;
}

/* IRLS weight psi(r) / r, equal to 1 at r = 0. */
static double hampel_weight(double r, double a, double b, double c)
{
    if (fabs(r) <= a) return 1.0;
    return oracle_hampel_psi(r, a, b, c) / r;
}

/* Bilinear interpolation of a W x H plane at (x, y); each of the four taps is
 * clamped to the border. */
static double bilinear(const double* P, int W, int H, double x, double y)
{
    double fx0 = floor(x), fy0 = floor(y);
    int x0 = (int)fx0, y0 = (int)fy0;
    double ax = x - fx0, ay = y - fy0;
    int xa = clampi(x0, 0, W - 1), xb = clampi(x0 + 1, 0, W - 1);
    int ya = clampi(y0, 0, H - 1), yb = clampi(y0 + 1, 0, H - 1);
    return (1 - ax) * (1 - ay) * P[(long)ya * W + xa] + ax * (1 - ay) * P[(long)ya * W + xb]
         + (1 - ax) * ay * P[(long)yb * W + xa] + ax * ay * P[(long)yb * W + xb];
}

/* Cholesky solve of the n x n symmetric system A x = rhs (n <= 4). Returns 0 on a
 * non-positive pivot. */
static int cholesky_solve(int n, const double A[4][4], const double rhs[4], double x[4])
{
    double L[4][4] = {{0}};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0)) return 0;
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    double z[4];
    for (int i = 0; i < n; ++i) {
        double s = rhs[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * z[k];
        z[i] = s / L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = z[i];
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
 *   for l = L-1 .. 0:
 *     p_l = (p + 1/2) / 2^l - 1/2                      (centre-aligned pyramid map)
 *     template T_k, Tx_k, Ty_k = bilinear(I1_l, I1x_l, I1y_l) at p_l + k,
 *       k in [-r, r]^2
 *     if lambda_min(sum_k [Tx Ty]^T [Tx Ty]) / (2r+1)^2 < min_eig: SMALL_EIG, stop
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
static int track_point(const level_view* P1, const level_view* P2, const oracle_rlof_params* prm,
                       double px, double py, double* flow, double* illum, int* iters)
{
    const int r = prm->radius, side = 2 * r + 1, npx = side * side;
    const int nm = prm->model == 4 ? 4 : 2;
    double* T = malloc(sizeof(double) * 3 * npx);
    double *Tx = T + npx, *Ty = T + 2 * npx;
    double gx = 0, gy = 0, dx = 0, dy = 0, m = 0, c = 0;
    int status = OR_TRACKED;
    *iters = 0;
    for (int l = prm->levels - 1; l >= 0 && status == OR_TRACKED; --l) {
        const level_view* A = &P1[l];
        const level_view* B = &P2[l];
        double scale = ldexp(1.0, -l);
        double plx = (px + 0.5) * scale - 0.5, ply = (py + 0.5) * scale - 0.5;
        double G00 = 0, G01 = 0, G11 = 0;
        for (int ky = -r; ky <= r; ++ky)
            for (int kx = -r; kx <= r; ++kx) {
                int s = (ky + r) * side + (kx + r);
                T[s] = bilinear(A->I, A->W, A->H, plx + kx, ply + ky);
                Tx[s] = bilinear(A->Ix, A->W, A->H, plx + kx, ply + ky);
                Ty[s] = bilinear(A->Iy, A->W, A->H, plx + kx, ply + ky);
                G00 += Tx[s] * Tx[s];
                G01 += Tx[s] * Ty[s];
                G11 += Ty[s] * Ty[s];
            }
        double half_tr = 0.5 * (G00 + G11), half_df = 0.5 * (G00 - G11);
        double lam_min = half_tr - sqrt(half_df * half_df + G01 * G01);
        if (lam_min / npx < prm->min_eig) { status = OR_SMALL_EIG; break; }
        dx = dy = 0;
        int converged = 0;
        for (int it = 0; it < prm->max_iter; ++it) {
            double qx = plx + gx + dx, qy = ply + gy + dy;
            if (!(qx >= 0 && qx <= B->W - 1 && qy >= 0 && qy <= B->H - 1)) { status = OR_OOB; break; }
            double Hm[4][4] = {{0}}, bv[4] = {0};
            for (int ky = -r; ky <= r; ++ky)
                for (int kx = -r; kx <= r; ++kx) {
                    int s = (ky + r) * side + (kx + r);
                    double J = bilinear(B->I, B->W, B->H, qx + kx, qy + ky);
                    double res, a[4];
                    if (nm == 4) {
                        res = J - (1 + m) * T[s] - c;
                        a[0] = Tx[s]; a[1] = Ty[s]; a[2] = -T[s]; a[3] = -1.0;
                    } else {
                        res = J - T[s];
                        a[0] = Tx[s]; a[1] = Ty[s];
                    }
                    double w = hampel_weight(res, prm->hampel_a, prm->hampel_b, prm->hampel_c);
                    for (int i = 0; i < nm; ++i) {
                        for (int j = 0; j < nm; ++j) Hm[i][j] += w * a[i] * a[j];
                        bv[i] += w * a[i] * res;
                    }
                }
            double rhs[4], delta[4];
            for (int i = 0; i < nm; ++i) rhs[i] = -bv[i];
            if (!cholesky_solve(nm, Hm, rhs, delta)) { status = OR_SINGULAR; break; }
            dx += delta[0];
            dy += delta[1];
            if (nm == 4) { m += delta[2]; c += delta[3]; }
            ++*iters;
            if (sqrt(delta[0] * delta[0] + delta[1] * delta[1]) < prm->eps) { converged = 1; break; }
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
    if (status == OR_TRACKED || status == OR_MAXITER) {
        flow[0] = gx + dx;
        flow[1] = gy + dy;
        if (illum) { illum[0] = m; illum[1] = c; }
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
 * Outputs: flow [n][2], status [n], iters [n] (nullable), illum [n][2] (gain m and
 * offset c; nullable). nthreads <= 0 uses the OpenMP default.
 */
int oracle_rlof_track(const double* I1, const double* I2, int W, int H, const double* pts, int n,
                      const oracle_rlof_params* prm, double* flow, uint8_t* status, int32_t* iters,
                      double* illum, int nthreads)
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
        status[k] = (uint8_t)track_point(v1, v2, prm, pts[2 * k], pts[2 * k + 1], flow + 2 * k,
                                         illum ? illum + 2 * k : NULL, &it);
        if (iters) iters[k] = it;
    }
done:
    free(pyr1);
    free(pyr2);
    return rc;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
