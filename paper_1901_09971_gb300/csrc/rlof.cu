// RLOF sparse point tracking (arXiv 1901.09971, Section 2 "Sparse point tracking";
// Section 3 "Parameters": RLOF with the illumination model).
//
// Work mapping: a group of G consecutive lanes (G = 8, 16 or 32) owns one point
// for its whole coarse-to-fine trajectory. Each lane holds SL support samples in
// registers (slot s = lane + G * j of the (2r+1)^2 support, row-major), so the
// template T, Tx, Ty of a level is sampled once and stays in registers for all of
// that level's Gauss-Newton iterations. Per iteration every lane samples frame 2
// at its slots (bilinear, FP32, all slots share one set of fractional weights),
// forms the Hampel weight and its partial sums of the 4x4 (or 2x2) normal
// equations, and the group reduces them with xor shuffles. The butterfly leaves
// bit-identical sums in every lane, so the FP32 Cholesky solve, the update and
// the convergence test run redundantly and the group's control flow stays
// uniform; points converge and exit independently.
#include "common.cuh"

namespace {

struct LevelPlanes {
    const void *I1, *I1x, *I1y, *I2;
    int W, H, pitch;
};

struct RlofArgs {
    LevelPlanes lv[DGF_MAX_LEVELS];
    int levels, radius, max_iter, n;
    float eps2, ha, hb, hc, inv_cb, min_eig;
    const float* pts;
    float* flow;
    uint8_t* status;
    uint8_t* iters;
    float* illum;
};

template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// Bilinear sample with clamped taps at integer base (xi, yi) and weights (ax, ay).
template <typename TS>
__device__ __forceinline__ float sample_clamped(const TS* P, int pitch, int W, int H, int xi, int yi, float ax,
                                                float ay)
{
    const int xa = min(max(xi, 0), W - 1), xb = min(max(xi + 1, 0), W - 1);
    const int ya = min(max(yi, 0), H - 1), yb = min(max(yi + 1, 0), H - 1);
    const TS* r0 = P + (size_t)ya * pitch;
    const TS* r1 = P + (size_t)yb * pitch;
    const float v00 = dgf::ld(r0 + xa), v01 = dgf::ld(r0 + xb);
    const float v10 = dgf::ld(r1 + xa), v11 = dgf::ld(r1 + xb);
    const float top = fmaf(ax, v01 - v00, v00);
    const float bot = fmaf(ax, v11 - v10, v10);
    return fmaf(ay, bot - top, top);
}

// Bilinear sample of four in-bounds taps starting at p (row stride pitch).
template <typename TS>
__device__ __forceinline__ float sample_inside(const TS* p, int pitch, float ax, float ay)
{
    const float v00 = dgf::ld(p), v01 = dgf::ld(p + 1);
    const float v10 = dgf::ld(p + pitch), v11 = dgf::ld(p + pitch + 1);
    const float top = fmaf(ax, v01 - v00, v00);
    const float bot = fmaf(ax, v11 - v10, v10);
    return fmaf(ay, bot - top, top);
}

// Hampel IRLS weight psi(r) / r (continuous three-part Hampel).
__device__ __forceinline__ float hampel_weight(float r, float ha, float hb, float hc, float inv_cb)
{
    const float ar = fabsf(r);
    const float inv = __frcp_rn(fmaxf(ar, ha));
    float w = ha * inv;
    w = ar <= hb ? w : w * fmaxf((hc - ar) * inv_cb, 0.f);
    return ar <= ha ? 1.f : w;
}

// Cholesky solve of the symmetric positive definite N x N system H x = rhs.
// Returns false on a non-positive pivot.
template <int N>
__device__ __forceinline__ bool chol_solve(float (&H)[N][N], const float (&rhs)[N], float (&x)[N])
{
    float L[N][N];
    float inv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float s = H[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) s = fmaf(-L[i][k], L[j][k], s);
            if (i == j) {
                if (!(s > 0.f)) return false;
                inv[i] = rsqrtf(s);
                L[i][i] = s * inv[i];
            } else {
                L[i][j] = s * inv[j];
            }
        }
    }
    float z[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float s = rhs[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s = fmaf(-L[i][k], z[k], s);
        z[i] = s * inv[i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        float s = z[i];
#pragma unroll
        for (int k = i + 1; k < N; ++k) s = fmaf(-L[k][i], x[k], s);
        x[i] = s * inv[i];
    }
    return true;
}

template <typename TS, int G, int SL, int MODEL>
__global__ void __launch_bounds__(256) rlof_kernel(const RlofArgs a)
{
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int pt = gtid / G;
    const int lane = threadIdx.x & (G - 1);
    if (pt >= a.n) return;
    const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int R = a.radius, side = 2 * R + 1, npx = side * side;

    const float2 p = reinterpret_cast<const float2*>(a.pts)[pt];
    float gx = 0.f, gy = 0.f, dx = 0.f, dy = 0.f, m = 0.f, c = 0.f;
    int status = DGF_TRACKED, iters = 0;

    float T[SL], Tx[SL], Ty[SL];
    int off[SL];

    for (int l = a.levels - 1; l >= 0; --l) {
        const LevelPlanes L = a.lv[l];
        const TS* I1 = static_cast<const TS*>(L.I1);
        const TS* I1x = static_cast<const TS*>(L.I1x);
        const TS* I1y = static_cast<const TS*>(L.I1y);
        const TS* I2 = static_cast<const TS*>(L.I2);
        const float scale = __int_as_float((127 - l) << 23);  // 2^-l
        const float plx = (p.x + 0.5f) * scale - 0.5f, ply = (p.y + 0.5f) * scale - 0.5f;

        // level set-up: template and its gradients at p_l + k
        {
            const float fx0 = floorf(plx), fy0 = floorf(ply);
            const int x0 = (int)fx0, y0 = (int)fy0;
            const float ax = plx - fx0, ay = ply - fy0;
            float g00 = 0.f, g01 = 0.f, g11 = 0.f;
#pragma unroll
            for (int j = 0; j < SL; ++j) {
                const int s = lane + G * j;
                const int ky = s / side, kx = s - ky * side;
                off[j] = (ky - R) * L.pitch + (kx - R);
                if (s < npx) {
                    const int xi = x0 + kx - R, yi = y0 + ky - R;
                    T[j] = sample_clamped(I1, L.pitch, L.W, L.H, xi, yi, ax, ay);
                    Tx[j] = sample_clamped(I1x, L.pitch, L.W, L.H, xi, yi, ax, ay);
                    Ty[j] = sample_clamped(I1y, L.pitch, L.W, L.H, xi, yi, ax, ay);
                    g00 = fmaf(Tx[j], Tx[j], g00);
                    g01 = fmaf(Tx[j], Ty[j], g01);
                    g11 = fmaf(Ty[j], Ty[j], g11);
                } else {
                    T[j] = Tx[j] = Ty[j] = 0.f;
                }
            }
            g00 = group_sum<G>(g00, mask);
            g01 = group_sum<G>(g01, mask);
            g11 = group_sum<G>(g11, mask);
            const float ht = 0.5f * (g00 + g11), hd = 0.5f * (g00 - g11);
            const float lam = ht - sqrtf(hd * hd + g01 * g01);
            if (lam / (float)npx < a.min_eig) {
                status = DGF_SMALL_EIG;
                break;
            }
        }

        dx = 0.f;
        dy = 0.f;
        bool converged = false;
        for (int it = 0; it < a.max_iter; ++it) {
            const float qx = plx + gx + dx, qy = ply + gy + dy;
            if (!(qx >= 0.f && qx <= (float)(L.W - 1) && qy >= 0.f && qy <= (float)(L.H - 1))) {
                status = DGF_OOB;
                break;
            }
            const float fx0 = floorf(qx), fy0 = floorf(qy);
            const int x0 = (int)fx0, y0 = (int)fy0;
            const float ax = qx - fx0, ay = qy - fy0;
            const bool inside = x0 - R >= 0 && x0 + R + 1 <= L.W - 1 && y0 - R >= 0 && y0 + R + 1 <= L.H - 1;
            const TS* base = I2 + (size_t)y0 * L.pitch + x0;
            const float g1 = 1.f + m;
            float h[10], b[4];
#pragma unroll
            for (int k = 0; k < 10; ++k) h[k] = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) b[k] = 0.f;
#pragma unroll
            for (int j = 0; j < SL; ++j) {
                const int s = lane + G * j;
                if (s < npx) {
                    float J;
                    if (inside) {
                        J = sample_inside(base + off[j], L.pitch, ax, ay);
                    } else {
                        const int ky = s / side, kx = s - ky * side;
                        J = sample_clamped(I2, L.pitch, L.W, L.H, x0 + kx - R, y0 + ky - R, ax, ay);
                    }
                    const float r = MODEL == 4 ? (J - g1 * T[j]) - c : J - T[j];
                    const float w = hampel_weight(r, a.ha, a.hb, a.hc, a.inv_cb);
                    const float wTx = w * Tx[j], wTy = w * Ty[j];
                    h[0] = fmaf(wTx, Tx[j], h[0]);
                    h[1] = fmaf(wTx, Ty[j], h[1]);
                    h[4] = fmaf(wTy, Ty[j], h[4]);
                    b[0] = fmaf(wTx, r, b[0]);
                    b[1] = fmaf(wTy, r, b[1]);
                    if (MODEL == 4) {
                        const float wT = w * T[j];
                        h[2] = fmaf(wTx, T[j], h[2]);
                        h[3] += wTx;
                        h[5] = fmaf(wTy, T[j], h[5]);
                        h[6] += wTy;
                        h[7] = fmaf(wT, T[j], h[7]);
                        h[8] += wT;
                        h[9] += w;
                        b[2] = fmaf(wT, r, b[2]);
                        b[3] = fmaf(w, r, b[3]);
                    }
                }
            }
            float delta[4];
            bool ok;
            if (MODEL == 4) {
#pragma unroll
                for (int k = 0; k < 10; ++k) h[k] = group_sum<G>(h[k], mask);
#pragma unroll
                for (int k = 0; k < 4; ++k) b[k] = group_sum<G>(b[k], mask);
                // a = (Tx, Ty, -T, -1): fold the signs of the T and constant columns
                float Hm[4][4] = {{h[0], h[1], -h[2], -h[3]},
                                  {h[1], h[4], -h[5], -h[6]},
                                  {-h[2], -h[5], h[7], h[8]},
                                  {-h[3], -h[6], h[8], h[9]}};
                const float rhs[4] = {-b[0], -b[1], b[2], b[3]};
                float x[4];
                ok = chol_solve<4>(Hm, rhs, x);
#pragma unroll
                for (int k = 0; k < 4; ++k) delta[k] = x[k];
            } else {
                h[0] = group_sum<G>(h[0], mask);
                h[1] = group_sum<G>(h[1], mask);
                h[4] = group_sum<G>(h[4], mask);
                b[0] = group_sum<G>(b[0], mask);
                b[1] = group_sum<G>(b[1], mask);
                float Hm[2][2] = {{h[0], h[1]}, {h[1], h[4]}};
                const float rhs[2] = {-b[0], -b[1]};
                float x[2];
                ok = chol_solve<2>(Hm, rhs, x);
                delta[0] = x[0];
                delta[1] = x[1];
            }
            if (!ok) {
                status = DGF_SINGULAR;
                break;
            }
            dx += delta[0];
            dy += delta[1];
            if (MODEL == 4) {
                m += delta[2];
                c += delta[3];
            }
            ++iters;
            if (delta[0] * delta[0] + delta[1] * delta[1] < a.eps2) {
                converged = true;
                break;
            }
        }
        if (status != DGF_TRACKED) break;
        if (l > 0) {
            gx = 2.f * (gx + dx);
            gy = 2.f * (gy + dy);
        } else if (!converged) {
            status = DGF_MAXITER;
        }
    }

    if (lane == 0) {
        const bool ok = status == DGF_TRACKED || status == DGF_MAXITER;
        reinterpret_cast<float2*>(a.flow)[pt] = ok ? make_float2(gx + dx, gy + dy) : make_float2(0.f, 0.f);
        a.status[pt] = (uint8_t)status;
        if (a.iters) a.iters[pt] = (uint8_t)min(iters, 255);
        if (a.illum)
            reinterpret_cast<float2*>(a.illum)[pt] = ok && MODEL == 4 ? make_float2(m, c) : make_float2(0.f, 0.f);
    }
}

int g_lanes_override = 0;

template <typename TS, int MODEL>
int launch(const RlofArgs& a, int lanes, cudaStream_t stream)
{
    const int npx = (2 * a.radius + 1) * (2 * a.radius + 1);
    const int threads = 256;
    const long long total = (long long)a.n * lanes;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads);
#define DGF_LAUNCH(G, SL)                                                                       \
    if (lanes == G && npx <= G * SL) {                                                          \
        rlof_kernel<TS, G, SL, MODEL><<<blocks, threads, 0, stream>>>(a);                      \
        return dgf::launch_status();                                                            \
    }
    DGF_LAUNCH(8, 11)   // radius 4 (81 samples)
    DGF_LAUNCH(8, 16)   // radius 5 (121)
    DGF_LAUNCH(16, 6)   // radius 4
    DGF_LAUNCH(16, 8)   // radius 5
    DGF_LAUNCH(32, 3)   // radius 4
    DGF_LAUNCH(32, 4)   // radius 5
    DGF_LAUNCH(32, 8)   // radius 6, 7
#undef DGF_LAUNCH
    return DGF_ERR_ARG;
}

int choose_lanes(int radius)
{
    if (g_lanes_override) return radius <= 5 || g_lanes_override == 32 ? g_lanes_override : 32;
    return radius <= 5 ? 8 : 32;
}

}  // namespace

extern "C" void dgf_rlof_params_default(dgf_rlof_params* p)
{
    if (!p) return;
    p->version = DGF_RLOF_PARAMS_VERSION;
    p->levels = 3;
    p->radius = 4;
    p->max_iter = 30;
    p->model = 4;
    p->storage = DGF_F32;
    p->eps = 1e-3f;
    p->hampel_a = 8.f;
    p->hampel_b = 16.f;
    p->hampel_c = 32.f;
    p->min_eig = 1e-3f;
}

// Tuning hook: lanes per point (8, 16 or 32; 0 restores the automatic choice).
// Returns the previous setting, or DGF_ERR_ARG for an unsupported value.
extern "C" int dgf_rlof_set_lanes(int lanes)
{
    if (lanes != 0 && lanes != 8 && lanes != 16 && lanes != 32) return DGF_ERR_ARG;
    const int prev = g_lanes_override;
    g_lanes_override = lanes;
    return prev;
}

extern "C" int rlof_track(const void* pyr1, const void* pyr2, int W, int H, const float* pts, int n,
                          const dgf_rlof_params* p, float* flow, uint8_t* status, uint8_t* iters, float* illum,
                          cudaStream_t stream)
{
    if (!p || p->version != DGF_RLOF_PARAMS_VERSION || n < 0) return DGF_ERR_ARG;
    if (p->radius < 1 || p->radius > DGF_MAX_RADIUS || p->max_iter < 1 || p->max_iter > 255 ||
        (p->model != 2 && p->model != 4) || !(p->eps >= 0.f) || !(p->hampel_a > 0.f) ||
        !(p->hampel_b >= p->hampel_a) || !(p->hampel_c > p->hampel_b) || !(p->min_eig >= 0.f))
        return DGF_ERR_ARG;
    dgf_pyramid_layout L1;
    int rc = dgf_pyramid_layout_get(W, H, p->levels, p->storage, 1, &L1);
    if (rc != DGF_OK) return rc;
    const int need = 2 * p->radius + 2;
    if (L1.W[p->levels - 1] < need || L1.H[p->levels - 1] < need) return DGF_ERR_LEVELS;
    if (n == 0) return DGF_OK;
    if (!pyr1 || !pyr2 || !pts || !flow || !status || !dgf::aligned(pyr1, 256) || !dgf::aligned(pyr2, 256) ||
        !dgf::aligned(pts, 8) || !dgf::aligned(flow, 8) || (illum && !dgf::aligned(illum, 8)))
        return DGF_ERR_ARG;
    RlofArgs a = {};
    for (int l = 0; l < p->levels; ++l) {
        const char* b1 = static_cast<const char*>(pyr1);
        const char* b2 = static_cast<const char*>(pyr2);
        a.lv[l].I1 = b1 + L1.off_I[l];
        a.lv[l].I1x = b1 + L1.off_Ix[l];
        a.lv[l].I1y = b1 + L1.off_Iy[l];
        a.lv[l].I2 = b2 + L1.off_I[l];  // intensity planes sit at the same offsets with or without gradients
        a.lv[l].W = L1.W[l];
        a.lv[l].H = L1.H[l];
        a.lv[l].pitch = L1.pitch[l];
    }
    a.levels = p->levels;
    a.radius = p->radius;
    a.max_iter = p->max_iter;
    a.n = n;
    a.eps2 = p->eps * p->eps;
    a.ha = p->hampel_a;
    a.hb = p->hampel_b;
    a.hc = p->hampel_c;
    a.inv_cb = 1.f / (p->hampel_c - p->hampel_b);
    a.min_eig = p->min_eig;
    a.pts = pts;
    a.flow = flow;
    a.status = status;
    a.iters = iters;
    a.illum = illum;
    const int lanes = choose_lanes(p->radius);
    if (p->storage == DGF_F32)
        return p->model == 4 ? launch<float, 4>(a, lanes, stream) : launch<float, 2>(a, lanes, stream);
    return p->model == 4 ? launch<__half, 4>(a, lanes, stream) : launch<__half, 2>(a, lanes, stream);
}
