// Adjoints: gradients of DeGraF key-points (Section 2, Eq. 1-2) and of RLOF flow
// with respect to the frames. The paper differentiates neither; both follow from
// the forward definitions:
//
//  - DeGraF: the positive centroid x = sum j I / S has dx/dI_ij = (j - x) / S; the
//    negative one (weights 1 + m - I) has -(j - x) / S_neg, plus, on the window's
//    first maximum (where m follows I), sum_ij (j - x) / S_neg. Per window this is an
//    affine function of the local pixel position plus one extra term, so pass 1
//    stores (A, B, C0, E, argmax) per window and pass 2 gathers, for every pixel, the
//    windows covering it in a fixed order (deterministic, no atomics).
//  - RLOF: implicit differentiation at the converged level-0 state theta = (d, m, c):
//    F = sum_k psi(r_k) a_k = 0 there, so with A = dF/dtheta = sum_k psi'(r_k) a_k s_k^T
//    (s_k = dr_k/dtheta uses the exact derivative of the bilinear interpolant) and
//    A^T lambda = upstream gradient, grad I = -lambda^T dF/dI. One warp per point
//    forms and reduces A, solves for lambda (partial-pivoting LU in FP32) and
//    scatters with atomics into grad I2, and into the adjoints of the template plane
//    and of the two Sobel planes (workspace); a per-pixel pass then adds the
//    template adjoint and the transposed Sobel / 8 stencil into grad I1. Atomic
//    order makes the last bits of the result vary between runs.
#include <initializer_list>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------- DeGraF

struct WindowRecord {
    float4 coef;  // A, B, C0, E: contribution A j + B i + C0 (+ E at the argmax)
};

__global__ void __launch_bounds__(kThreads) degraf_records_kernel(const uint8_t* img, int pitch, int ww, int wh,
                                                                   int step, int nu, int nv, const float* grad_pts,
                                                                   float4* coef, int* argmax)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nu * nv) return;
    const int u = k % nu, v = k / nu;
    const uint8_t* w0 = img + (size_t)(v * step) * pitch + u * step;
    int S = 0, X = 0, Y = 0, m = -1, a = 0;
    for (int i = 0; i < wh; ++i)
        for (int j = 0; j < ww; ++j) {
            const int I = w0[(size_t)i * pitch + j];
            S += I;
            X += j * I;
            Y += i * I;
            if (I > m) {  // first maximum in row-major order
                m = I;
                a = i * ww + j;
            }
        }
    const int n = ww * wh, m1 = m + 1, Sn = n * m1 - S;
    const float gx = grad_pts[2 * k], gy = grad_pts[2 * k + 1];
    float A, B, C0, E = 0.f;
    if (Sn > S) {
        const float sj = (float)(wh * (ww * (ww - 1) / 2)), si = (float)(ww * (wh * (wh - 1) / 2));
        const float cx = ((float)m1 * sj - (float)X) / (float)Sn, cy = ((float)m1 * si - (float)Y) / (float)Sn;
        A = -gx / (float)Sn;
        B = -gy / (float)Sn;
        C0 = -(A * cx + B * cy);
        E = (gx * (sj - (float)n * cx) + gy * (si - (float)n * cy)) / (float)Sn;
    } else {
        const float cx = (float)X / (float)S, cy = (float)Y / (float)S;
        A = gx / (float)S;
        B = gy / (float)S;
        C0 = -(A * cx + B * cy);
        a = -1;
    }
    coef[k] = make_float4(A, B, C0, E);
    argmax[k] = a;
}

__global__ void __launch_bounds__(kThreads) degraf_gather_kernel(int W, int H, int ww, int wh, int step, int nu, int nv,
                                                                  const float4* coef, const int* argmax, float* grad,
                                                                  int grad_pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const int u_lo = x >= ww ? (x - ww) / step + 1 : 0, u_hi = min(x / step, nu - 1);
    const int v_lo = y >= wh ? (y - wh) / step + 1 : 0, v_hi = min(y / step, nv - 1);
    float acc = 0.f;
    for (int v = v_lo; v <= v_hi; ++v) {
        const int i = y - v * step;
        for (int u = u_lo; u <= u_hi; ++u) {
            const int j = x - u * step, k = v * nu + u;
            const float4 c = coef[k];
            acc += fmaf(c.x, (float)j, fmaf(c.y, (float)i, c.z)) + (argmax[k] == i * ww + j ? c.w : 0.f);
        }
    }
    grad[(size_t)y * grad_pitch + x] += acc;
}

// ------------------------------------------------------------------ RLOF

template <typename TS>
__device__ __forceinline__ float tap(const TS* P, int pitch, int W, int H, int x, int y)
{
    return dgf::ld(P + (size_t)min(max(y, 0), H - 1) * pitch + min(max(x, 0), W - 1));
}

// Bilinear sample at (x, y) with its four (clamped) taps and weights.
struct Bilin {
    int xa, xb, ya, yb;
    float ax, ay;
    __device__ __forceinline__ Bilin(float x, float y, int W, int H)
    {
        const float fx = floorf(x), fy = floorf(y);
        const int x0 = (int)fx, y0 = (int)fy;
        ax = x - fx;
        ay = y - fy;
        xa = min(max(x0, 0), W - 1);
        xb = min(max(x0 + 1, 0), W - 1);
        ya = min(max(y0, 0), H - 1);
        yb = min(max(y0 + 1, 0), H - 1);
    }
    template <typename TS>
    __device__ __forceinline__ float sample(const TS* P, int pitch, float* dx = nullptr, float* dy = nullptr) const
    {
        const float v00 = dgf::ld(P + (size_t)ya * pitch + xa), v01 = dgf::ld(P + (size_t)ya * pitch + xb);
        const float v10 = dgf::ld(P + (size_t)yb * pitch + xa), v11 = dgf::ld(P + (size_t)yb * pitch + xb);
        if (dx) *dx = (1.f - ay) * (v01 - v00) + ay * (v11 - v10);
        if (dy) *dy = (1.f - ax) * (v10 - v00) + ax * (v11 - v01);
        return (1.f - ax) * (1.f - ay) * v00 + ax * (1.f - ay) * v01 + (1.f - ax) * ay * v10 + ax * ay * v11;
    }
    __device__ __forceinline__ void scatter(float* G, int gpitch, float value) const
    {
        atomicAdd(G + (size_t)ya * gpitch + xa, (1.f - ax) * (1.f - ay) * value);
        atomicAdd(G + (size_t)ya * gpitch + xb, ax * (1.f - ay) * value);
        atomicAdd(G + (size_t)yb * gpitch + xa, (1.f - ax) * ay * value);
        atomicAdd(G + (size_t)yb * gpitch + xb, ax * ay * value);
    }
};

__device__ __forceinline__ float hampel_psi(float r, float ha, float hb, float hc)
{
    const float ar = fabsf(r);
    const float s = r < 0.f ? -1.f : 1.f;
    if (ar <= ha) return r;
    if (ar <= hb) return ha * s;
    if (ar <= hc) return ha * s * (hc - ar) / (hc - hb);
    return 0.f;
}

__device__ __forceinline__ float hampel_dpsi(float r, float ha, float hb, float hc)
{
    const float ar = fabsf(r);
    if (ar <= ha) return 1.f;
    if (ar <= hb) return 0.f;
    if (ar <= hc) return -ha / (hc - hb);
    return 0.f;
}

// Partial-pivoting LU solve of the N x N system M x = rhs; false when singular.
template <int N>
__device__ __forceinline__ bool lu_solve(float (&M)[N][N], float (&rhs)[N], float (&x)[N])
{
#pragma unroll
    for (int col = 0; col < N; ++col) {
        int piv = col;
#pragma unroll
        for (int r = col + 1; r < N; ++r)
            if (fabsf(M[r][col]) > fabsf(M[piv][col])) piv = r;
        if (M[piv][col] == 0.f) return false;
#pragma unroll
        for (int r = 0; r < N; ++r) {  // swap rows col and piv (unrolled, no dynamic indexing)
            if (r == piv && r != col) {
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const float t = M[col][j];
                    M[col][j] = M[r][j];
                    M[r][j] = t;
                }
                const float t = rhs[col];
                rhs[col] = rhs[r];
                rhs[r] = t;
            }
        }
        const float inv = 1.f / M[col][col];
#pragma unroll
        for (int r = col + 1; r < N; ++r) {
            const float f = M[r][col] * inv;
#pragma unroll
            for (int j = col; j < N; ++j) M[r][j] -= f * M[col][j];
            rhs[r] -= f * rhs[col];
        }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        float s = rhs[i];
#pragma unroll
        for (int j = i + 1; j < N; ++j) s -= M[i][j] * x[j];
        x[i] = s / M[i][i];
    }
    return true;
}

struct BackArgs {
    const void *I1, *I1x, *I1y, *I2;  // level-0 planes
    int W, H, pitch;
    int n, radius, model;
    float ha, hb, hc;
    const float *pts, *flow, *illum, *grad_flow, *grad_illum;
    const uint8_t* status;
    float *gT, *gTx, *gTy, *grad_I2;  // W x H planes (pitch W)
    int grad_pitch;
};

template <typename TS, int MODEL>
__global__ void __launch_bounds__(kThreads) rlof_backward_kernel(const BackArgs a)
{
    const int pt = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (pt >= a.n || a.status[pt] != DGF_TRACKED) return;  // whole warps leave together
    constexpr int NM = MODEL == 4 ? 4 : 2;
    const TS* I1 = static_cast<const TS*>(a.I1);
    const TS* I1x = static_cast<const TS*>(a.I1x);
    const TS* I1y = static_cast<const TS*>(a.I1y);
    const TS* I2 = static_cast<const TS*>(a.I2);
    const int R = a.radius, side = 2 * R + 1, npx = side * side;
    const float px = a.pts[2 * pt], py = a.pts[2 * pt + 1];
    const float qx = px + a.flow[2 * pt], qy = py + a.flow[2 * pt + 1];
    const float m = MODEL == 4 ? a.illum[2 * pt] : 0.f, c = MODEL == 4 ? a.illum[2 * pt + 1] : 0.f;

    // A = sum_k psi'(r_k) a_k s_k^T
    float A[NM][NM];
#pragma unroll
    for (int i = 0; i < NM; ++i)
#pragma unroll
        for (int j = 0; j < NM; ++j) A[i][j] = 0.f;
    for (int s = lane; s < npx; s += 32) {
        const int ky = s / side - R, kx = s % side - R;
        const Bilin bt(px + kx, py + ky, a.W, a.H);
        const float T = bt.sample(I1, a.pitch), Tx = bt.sample(I1x, a.pitch), Ty = bt.sample(I1y, a.pitch);
        const Bilin bj(qx + kx, qy + ky, a.W, a.H);
        float Jx, Jy;
        const float J = bj.sample(I2, a.pitch, &Jx, &Jy);
        const float r = MODEL == 4 ? J - (1.f + m) * T - c : J - T;
        const float dpsi = hampel_dpsi(r, a.ha, a.hb, a.hc);
        const float av[4] = {Tx, Ty, -T, -1.f}, sv[4] = {Jx, Jy, -T, -1.f};
#pragma unroll
        for (int i = 0; i < NM; ++i)
#pragma unroll
            for (int j = 0; j < NM; ++j) A[i][j] = fmaf(dpsi * av[i], sv[j], A[i][j]);
    }
#pragma unroll
    for (int i = 0; i < NM; ++i)
#pragma unroll
        for (int j = 0; j < NM; ++j)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) A[i][j] += __shfl_xor_sync(0xffffffffu, A[i][j], o);

    // A^T lambda = upstream (flow, and illumination for model 4)
    float At[NM][NM], u[NM], lam[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i)
#pragma unroll
        for (int j = 0; j < NM; ++j) At[i][j] = A[j][i];
    u[0] = a.grad_flow[2 * pt];
    u[1] = a.grad_flow[2 * pt + 1];
    if (MODEL == 4) {
        u[NM > 2 ? 2 : 0] = a.grad_illum ? a.grad_illum[2 * pt] : 0.f;
        u[NM > 3 ? 3 : 1] = a.grad_illum ? a.grad_illum[2 * pt + 1] : 0.f;
    }
    if (!lu_solve<NM>(At, u, lam)) return;

    for (int s = lane; s < npx; s += 32) {
        const int ky = s / side - R, kx = s % side - R;
        const Bilin bt(px + kx, py + ky, a.W, a.H);
        const float T = bt.sample(I1, a.pitch), Tx = bt.sample(I1x, a.pitch), Ty = bt.sample(I1y, a.pitch);
        const Bilin bj(qx + kx, qy + ky, a.W, a.H);
        const float J = bj.sample(I2, a.pitch);
        const float r = MODEL == 4 ? J - (1.f + m) * T - c : J - T;
        const float psi = hampel_psi(r, a.ha, a.hb, a.hc), dpsi = hampel_dpsi(r, a.ha, a.hb, a.hc);
        const float la = MODEL == 4 ? lam[0] * Tx + lam[1] * Ty - lam[NM > 2 ? 2 : 0] * T - lam[NM > 3 ? 3 : 1]
                                    : lam[0] * Tx + lam[1] * Ty;
        const float muT = MODEL == 4 ? -(1.f + m) * dpsi * la - psi * lam[NM > 2 ? 2 : 0] : -dpsi * la;
        bj.scatter(a.grad_I2, a.grad_pitch, -dpsi * la);
        bt.scatter(a.gT, a.W, -muT);
        bt.scatter(a.gTx, a.W, -psi * lam[0]);
        bt.scatter(a.gTy, a.W, -psi * lam[1]);
    }
}

// grad_I1 += gT + transposed Sobel / 8 of (gTx, gTy), with the forward's clamped
// taps: output pixel o read I1 at clamp(o + d), so t collects from every o whose
// clamped neighbour d lands on t.
__global__ void __launch_bounds__(kThreads) sobel_adjoint_kernel(int W, int H, const float* gT, const float* gTx,
                                                                  const float* gTy, float* grad, int grad_pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    float acc = gT[(size_t)y * W + x];
    for (int dy = -1; dy <= 1; ++dy) {
        // rows o_y with clamp(o_y + dy) == y
        const int ylo = max(0, (y == 0 ? -1000000 : y) - dy), yhi = min(H - 1, (y == H - 1 ? 1000000 : y) - dy);
        for (int oy = ylo; oy <= yhi; ++oy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int xlo = max(0, (x == 0 ? -1000000 : x) - dx), xhi = min(W - 1, (x == W - 1 ? 1000000 : x) - dx);
                const float sx = (float)(dx * (dy == 0 ? 2 : 1)) * 0.125f;  // Sobel-x weight of offset (dx, dy)
                const float sy = (float)(dy * (dx == 0 ? 2 : 1)) * 0.125f;  // Sobel-y weight
                if (sx == 0.f && sy == 0.f) continue;
                for (int ox = xlo; ox <= xhi; ++ox)
                    acc = fmaf(sx, gTx[(size_t)oy * W + ox], fmaf(sy, gTy[(size_t)oy * W + ox], acc));
            }
    }
    grad[(size_t)y * grad_pitch + x] += acc;
}

long long grid_count(int n, int win, int step) { return n < win ? 0 : (long long)((n - win) / step) + 1; }

}  // namespace

extern "C" size_t dgf_degraf_backward_workspace(int W, int H, int win_w, int win_h, int step)
{
    const long long n = dgf_degraf_count(W, H, win_w, win_h, step);
    if (n < 0) return 0;
    return dgf::round_up((size_t)n * sizeof(float4), 256) + dgf::round_up((size_t)n * sizeof(int), 256) + 256;
}

extern "C" int degraf_detect_backward(const uint8_t* img, int W, int H, int pitch, int win_w, int win_h, int step,
                                      const float* grad_pts, void* workspace, size_t ws_bytes, float* grad_img,
                                      int grad_pitch, cudaStream_t stream)
{
    const long long n = dgf_degraf_count(W, H, win_w, win_h, step);
    if (n < 0 || !img || pitch < W || !grad_img || grad_pitch < W) return DGF_ERR_ARG;
    if (n == 0) return DGF_OK;
    if (!grad_pts || !workspace || !dgf::aligned(workspace, 256) || n > (1LL << 30) || !dgf::aligned(grad_pts, 4) ||
        !dgf::aligned(grad_img, 4))
        return DGF_ERR_ARG;
    if (ws_bytes < dgf_degraf_backward_workspace(W, H, win_w, win_h, step)) return DGF_ERR_WORKSPACE;
    float4* coef = static_cast<float4*>(workspace);
    int* argmax = reinterpret_cast<int*>(static_cast<char*>(workspace) + dgf::round_up((size_t)n * sizeof(float4), 256));
    const int nu = (int)grid_count(W, win_w, step), nv = (int)grid_count(H, win_h, step);
    degraf_records_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, stream>>>(
        img, pitch, win_w, win_h, step, nu, nv, grad_pts, coef, argmax);
    degraf_gather_kernel<<<dim3((W + kThreads - 1) / kThreads, H), kThreads, 0, stream>>>(
        W, H, win_w, win_h, step, nu, nv, coef, argmax, grad_img, grad_pitch);
    return dgf::launch_status();
}

extern "C" size_t dgf_rlof_backward_workspace(int W, int H)
{
    if (W < 1 || H < 1) return 0;
    return 3 * dgf::round_up((size_t)W * H * sizeof(float), 256);
}

extern "C" int rlof_track_backward(const void* pyr1, const void* pyr2, int W, int H, const float* pts, int n,
                                   const dgf_rlof_params* p, const float* flow, const float* illum,
                                   const uint8_t* status, const float* grad_flow, const float* grad_illum,
                                   void* workspace, size_t ws_bytes, float* grad_I1, float* grad_I2, int grad_pitch,
                                   cudaStream_t stream)
{
    if (!p || p->version != DGF_RLOF_PARAMS_VERSION || n < 0 || W < 1 || H < 1) return DGF_ERR_ARG;
    if (p->levels < 1 || p->levels > DGF_MAX_LEVELS || p->radius < 1 || p->radius > DGF_MAX_RADIUS ||
        (p->model != 2 && p->model != 4) || (p->storage != DGF_F32 && p->storage != DGF_F16) ||
        !(p->hampel_a > 0.f) || !(p->hampel_b >= p->hampel_a) || !(p->hampel_c > p->hampel_b) ||
        p->cross_tau != 0.f)  // the adjoint is defined for the square support
        return DGF_ERR_ARG;
    if (!grad_I1 || !grad_I2 || grad_pitch < W) return DGF_ERR_ARG;
    if (n == 0) return DGF_OK;
    if (!pyr1 || !pyr2 || !pts || !flow || !status || !grad_flow || (p->model == 4 && !illum) || !workspace ||
        !dgf::aligned(workspace, 256) || !dgf::aligned(pyr1, 256) || !dgf::aligned(pyr2, 256))
        return DGF_ERR_ARG;
    for (const void* f : {(const void*)pts, (const void*)flow, (const void*)illum, (const void*)grad_flow,
                          (const void*)grad_illum, (const void*)grad_I1, (const void*)grad_I2})
        if (f && !dgf::aligned(f, 4)) return DGF_ERR_ARG;  // float arrays (null where optional)
    const size_t plane = dgf::round_up((size_t)W * H * sizeof(float), 256);
    if (ws_bytes < dgf_rlof_backward_workspace(W, H)) return DGF_ERR_WORKSPACE;
    dgf::LevelGeom g;
    const int es = p->storage == DGF_F32 ? 4 : 2;
    if (!dgf::level_geom(W, H, p->levels, es, 0, &g)) return DGF_ERR_ARG;
    char* ws = static_cast<char*>(workspace);
    if (cudaMemsetAsync(ws, 0, 3 * plane, stream) != cudaSuccess) return DGF_ERR_CUDA;
    BackArgs a;
    a.I1 = static_cast<const char*>(pyr1) + g.off_I;
    a.I1x = static_cast<const char*>(pyr1) + g.off_Ix;
    a.I1y = static_cast<const char*>(pyr1) + g.off_Iy;
    a.I2 = static_cast<const char*>(pyr2) + g.off_I;
    a.W = W;
    a.H = H;
    a.pitch = g.pitch;
    a.n = n;
    a.radius = p->radius;
    a.model = p->model;
    a.ha = p->hampel_a;
    a.hb = p->hampel_b;
    a.hc = p->hampel_c;
    a.pts = pts;
    a.flow = flow;
    a.illum = illum;
    a.grad_flow = grad_flow;
    a.grad_illum = grad_illum;
    a.status = status;
    a.gT = reinterpret_cast<float*>(ws);
    a.gTx = reinterpret_cast<float*>(ws + plane);
    a.gTy = reinterpret_cast<float*>(ws + 2 * plane);
    a.grad_I2 = grad_I2;
    a.grad_pitch = grad_pitch;
    const unsigned blocks = (unsigned)(((long long)n * 32 + kThreads - 1) / kThreads);
    if (p->storage == DGF_F32) {
        if (p->model == 4)
            rlof_backward_kernel<float, 4><<<blocks, kThreads, 0, stream>>>(a);
        else
            rlof_backward_kernel<float, 2><<<blocks, kThreads, 0, stream>>>(a);
    } else {
        if (p->model == 4)
            rlof_backward_kernel<__half, 4><<<blocks, kThreads, 0, stream>>>(a);
        else
            rlof_backward_kernel<__half, 2><<<blocks, kThreads, 0, stream>>>(a);
    }
    sobel_adjoint_kernel<<<dim3((W + kThreads - 1) / kThreads, H), kThreads, 0, stream>>>(
        W, H, a.gT, a.gTx, a.gTy, grad_I1, grad_pitch);
    return dgf::launch_status();
}
