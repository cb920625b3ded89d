// Global-motion prior for RLOF tracking (arXiv 1901.09971, Section 3 "Parameters":
// RLOF with the global motion model, RLOF(IM-GM)). The paper prints no formula; the
// model used is a global affine motion fitted robustly to a sparse first pass and
// used as every point's initial flow in the main pass.
//
// The fit runs in one CTA: per IRLS iteration every thread accumulates the weighted
// normal-equation sums of its points in FP64, the CTA reduces them in a fixed tree
// order (deterministic), and one thread solves the two 3 x 3 systems. It is tiny
// next to tracking (a few sums per first-pass point), so one CTA is enough and no
// host round trip separates the three stages: the main pass reads the fitted
// parameters from device memory.
#include "common.cuh"
#include "batch.cuh"

namespace {

constexpr int kFitThreads = 1024;
constexpr int kSums = 12;  // xx xy x yy y w | x qx, y qx, qx | x qy, y qy, qy

// Cholesky solve of the 3 x 3 normal equations (row-major m[9]); a pivot below
// 1e-10 of its diagonal entry counts as singular.
__device__ bool solve3(const double* m, const double* b, double* x)
{
    double L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, z[3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = m[3 * i + j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 1e-10 * m[3 * i + i])) return false;
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
    return true;
}

// Robust affine fit over the n first-pass points (point k at pts[k * stride]).
// out: a[6] then an int flag at byte 48 (1 = fitted).
__global__ void __launch_bounds__(kFitThreads) gm_fit_kernel(const float* pts, int stride, const float* flow,
                                                             const uint8_t* status, int n, int iters, double c0,
                                                             double c_min, double* out)
{
    __shared__ double part[kFitThreads / 32][kSums];
    __shared__ int used_part[kFitThreads / 32];
    __shared__ double a[6];
    __shared__ int go, made;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        a[0] = 1; a[1] = 0; a[2] = 0;
        a[3] = 0; a[4] = 1; a[5] = 0;
        go = 1;
        made = 0;
    }
    __syncthreads();
    for (int k = 0; k < iters; ++k) {
        if (!go) break;  // uniform: every thread reads it after the same barrier
        const double ck = fmax(c_min, ldexp(c0, -(k - 1)));
        double s[kSums];
#pragma unroll
        for (int j = 0; j < kSums; ++j) s[j] = 0.0;
        int used = 0;
        for (int i = threadIdx.x; i < n; i += kFitThreads) {
            if (status[i] != DGF_TRACKED) continue;
            const float2 p = reinterpret_cast<const float2*>(pts)[(long long)i * stride];
            const float2 f = reinterpret_cast<const float2*>(flow)[i];
            const double x = p.x, y = p.y, qx = x + (double)f.x, qy = y + (double)f.y;
            double w = 1.0;
            if (k > 0) {
                const double ex = a[0] * x + a[1] * y + a[2] - qx, ey = a[3] * x + a[4] * y + a[5] - qy;
                const double e = sqrt(ex * ex + ey * ey);
                if (e >= ck) continue;
                const double u = 1.0 - (e / ck) * (e / ck);
                w = u * u;
            }
            s[0] += w * x * x;
            s[1] += w * x * y;
            s[2] += w * x;
            s[3] += w * y * y;
            s[4] += w * y;
            s[5] += w;
            s[6] += w * x * qx;
            s[7] += w * y * qx;
            s[8] += w * qx;
            s[9] += w * x * qy;
            s[10] += w * y * qy;
            s[11] += w * qy;
            ++used;
        }
        // fixed-order reduction: xor butterfly in each warp, then one thread over the warps
#pragma unroll
        for (int j = 0; j < kSums; ++j)
            for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
        for (int o = 16; o > 0; o >>= 1) used += __shfl_xor_sync(0xffffffffu, used, o);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < kSums; ++j) part[warp][j] = s[j];
            used_part[warp] = used;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t[kSums];
            int u = 0;
            for (int j = 0; j < kSums; ++j) t[j] = 0.0;
            for (int w = 0; w < kFitThreads / 32; ++w) {
                for (int j = 0; j < kSums; ++j) t[j] += part[w][j];
                u += used_part[w];
            }
            const double m[9] = {t[0], t[1], t[2], t[1], t[3], t[4], t[2], t[4], t[5]};
            const double bx[3] = {t[6], t[7], t[8]}, by[3] = {t[9], t[10], t[11]};
            double sx[3], sy[3];
            if (u < 3 || !solve3(m, bx, sx) || !solve3(m, by, sy)) {
                go = 0;  // keep the previous estimate
            } else {
                a[0] = sx[0]; a[1] = sx[1]; a[2] = sx[2];
                a[3] = sy[0]; a[4] = sy[1]; a[5] = sy[2];
                made = 1;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = a[threadIdx.x];
    if (threadIdx.x == 0) reinterpret_cast<int*>(out + 6)[0] = made;
}

bool gm_params_ok(const dgf_gm_params* g)
{
    return g && g->version == DGF_GM_PARAMS_VERSION && g->stride >= 1 && g->extra_levels >= 0 && g->iters >= 1 &&
           g->iters <= 64 && g->c0 > 0 && g->c_min > 0;
}

// Workspace layout: [a[6], flag; 256 B] [first-pass flow, n_sub x 8 B] [first-pass status, n_sub B]
size_t flow_offset() { return 256; }
size_t status_offset(long long n_sub) { return dgf::round_up(flow_offset() + (size_t)n_sub * 8, 256); }

}  // namespace

extern "C" void dgf_gm_params_default(dgf_gm_params* g)
{
    if (!g) return;
    g->version = DGF_GM_PARAMS_VERSION;
    g->stride = 4;
    g->extra_levels = 2;
    g->iters = 8;
    g->c0 = 32.0;
    g->c_min = 2.0;
}

extern "C" size_t dgf_gm_workspace(int n, const dgf_gm_params* g)
{
    if (n < 0 || !gm_params_ok(g)) return 0;
    const long long n_sub = ((long long)n + g->stride - 1) / g->stride;
    return dgf::round_up(status_offset(n_sub) + (size_t)n_sub, 256);
}

extern "C" int rlof_track_gm(const void* pyr1, const void* pyr2, int W, int H, int pyr_levels, const float* pts, int n,
                             const dgf_rlof_params* p, const dgf_gm_params* g, float* flow, uint8_t* status,
                             uint8_t* iters, float* illum, void* workspace, size_t ws_bytes, cudaStream_t stream)
{
    dgf::TrackBatch main = {};
    int rc = dgf::prepare_params(p, main);
    if (rc != DGF_OK) return rc;
    if (!gm_params_ok(g) || n < 0 || W < 1 || H < 1 || pyr_levels > DGF_MAX_LEVELS ||
        pyr_levels < p->levels + g->extra_levels)
        return DGF_ERR_ARG;
    dgf_rlof_params deep = *p;
    deep.levels = p->levels + g->extra_levels;
    if ((rc = dgf::check_levels(W, H, &deep)) != DGF_OK) return rc;
    if (n == 0) return DGF_OK;
    if (!pyr1 || !pyr2 || !pts || !flow || !status || !workspace || !dgf::aligned(pyr1, 256) ||
        !dgf::aligned(pyr2, 256) || !dgf::aligned(pts, 8) || !dgf::aligned(flow, 8) ||
        (illum && !dgf::aligned(illum, 8)) || !dgf::aligned(workspace, 256))
        return DGF_ERR_ARG;
    if (ws_bytes < dgf_gm_workspace(n, g)) return DGF_ERR_WORKSPACE;
    const long long n_sub = ((long long)n + g->stride - 1) / g->stride;
    char* ws = static_cast<char*>(workspace);
    double* affine = reinterpret_cast<double*>(ws);
    float* sub_flow = reinterpret_cast<float*>(ws + flow_offset());
    uint8_t* sub_status = reinterpret_cast<uint8_t*>(ws + status_offset(n_sub));

    // 1. sparse first pass with the deeper pyramid (deep.levels <= pyr_levels <= DGF_MAX_LEVELS)
    dgf::TrackBatch first = {};
    if ((rc = dgf::prepare_params(&deep, first)) != DGF_OK) return rc;
    first.pyr_levels = pyr_levels;
    first.n_jobs = 1;
    first.total = (int)n_sub;
    first.jobs[0] = dgf::TrackJob{static_cast<const char*>(pyr1), static_cast<const char*>(pyr2), W, H, pts, sub_flow,
                                  sub_status, nullptr, nullptr, 0, g->stride, nullptr};
    if ((rc = dgf::launch_track(first, &deep, stream)) != DGF_OK) return rc;
    // 2. robust affine fit
    gm_fit_kernel<<<1, kFitThreads, 0, stream>>>(pts, g->stride, sub_flow, sub_status, (int)n_sub, g->iters, g->c0,
                                                 g->c_min, affine);
    if ((rc = dgf::launch_status()) != DGF_OK) return rc;
    // 3. main pass from the prior
    main.pyr_levels = pyr_levels;
    main.n_jobs = 1;
    main.total = n;
    main.jobs[0] = dgf::TrackJob{static_cast<const char*>(pyr1), static_cast<const char*>(pyr2), W, H, pts, flow, status,
                                 iters, illum, 0, 1, affine};
    return dgf::launch_track(main, p, stream);
}
