// Global-motion prior for RLOF tracking (arXiv 1901.09971, Section 3 "Parameters":
// RLOF with the global motion model, RLOF(IM-GM)). The paper prints no formula; the
// model used is a global affine motion fitted robustly to a sparse first pass and
// used as every point's initial flow in the main pass.
//
// The fit is an IRLS loop of a few iterations, one launch each: 64 CTAs sum the
// weighted normal equations of their points in FP64 (GB300's FP64 pipe is narrow,
// so the sums are spread over the SMs) into per-CTA partials; the CTA that finishes
// last (a ticket counter) adds the partials in CTA order, one thread per sum
// (deterministic), and solves the two 3 x 3 systems. The state (affine, fitted flag,
// go-on flag, ticket) lives in the workspace, so no host round trip separates the
// stages: the main pass reads the fitted parameters from device memory.
#include "common.cuh"
#include "batch.cuh"

namespace {

constexpr int kPartThreads = 256, kPartBlocks = 64;
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

// State at the start of the workspace: a[6] (doubles), then int flags at byte 48
// (1 = fitted) and byte 52 (1 = iterating), and the CTAs' ticket counter at byte 56.
__global__ void gm_init_kernel(double* state)
{
    state[0] = 1; state[1] = 0; state[2] = 0;
    state[3] = 0; state[4] = 1; state[5] = 0;
    reinterpret_cast<int*>(state + 6)[0] = 0;
    reinterpret_cast<int*>(state + 6)[1] = 1;
    reinterpret_cast<unsigned*>(state + 7)[0] = 0;
}

// IRLS iteration k: per-CTA sums over the points of the CTA's grid stride (point i
// at pts[i * stride]); partial[blockIdx.x][0..11] = the 12 sums, [12] = the number of
// weighted points. The last CTA to finish adds the partials in CTA order and solves
// the two 3 x 3 systems; a step with fewer than 3 weighted points or a singular
// matrix keeps the previous estimate and stops the loop.
__global__ void __launch_bounds__(kPartThreads) gm_iteration_kernel(const float* pts, int stride, const float* flow,
                                                                    const uint8_t* status, int n, int k, double c0,
                                                                    double c_min, double* state, double* partial)
{
    __shared__ double part[kPartThreads / 32][kSums + 1];
    __shared__ double tot[kSums + 1];
    __shared__ int last;
    int* flags = reinterpret_cast<int*>(state + 6);
    unsigned* ticket = reinterpret_cast<unsigned*>(state + 7);
    if (!flags[1]) return;  // uniform: the fit has stopped
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double a[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) a[j] = state[j];
    const double ck = fmax(c_min, ldexp(c0, -(k - 1)));
    double s[kSums + 1];
#pragma unroll
    for (int j = 0; j <= kSums; ++j) s[j] = 0.0;
    for (int i = blockIdx.x * kPartThreads + threadIdx.x; i < n; i += kPartBlocks * kPartThreads) {
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
        s[12] += 1.0;
    }
    // fixed-order reduction: xor butterfly in each warp, then one thread a sum over the warps
#pragma unroll
    for (int j = 0; j <= kSums; ++j)
        for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j <= kSums; ++j) part[warp][j] = s[j];
    __syncthreads();
    if (threadIdx.x <= kSums) {
        double t = 0.0;
        for (int w = 0; w < kPartThreads / 32; ++w) t += part[w][threadIdx.x];
        partial[blockIdx.x * (kSums + 1) + threadIdx.x] = t;
        __threadfence();  // the partial is visible device-wide before this CTA's ticket
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    // the last CTA: every other CTA's partial was written before its ticket
    __threadfence();
    if (threadIdx.x <= kSums) {
        double t = 0.0;
#pragma unroll 8
        for (int b = 0; b < kPartBlocks; ++b) t += __ldcg(partial + b * (kSums + 1) + threadIdx.x);
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    *ticket = 0;  // for the next iteration's launch
    const double m[9] = {tot[0], tot[1], tot[2], tot[1], tot[3], tot[4], tot[2], tot[4], tot[5]};
    const double bx[3] = {tot[6], tot[7], tot[8]}, by[3] = {tot[9], tot[10], tot[11]};
    double sx[3], sy[3];
    if (tot[12] < 3.0 || !solve3(m, bx, sx) || !solve3(m, by, sy)) {
        flags[1] = 0;  // keep the previous estimate
        return;
    }
    state[0] = sx[0]; state[1] = sx[1]; state[2] = sx[2];
    state[3] = sy[0]; state[4] = sy[1]; state[5] = sy[2];
    flags[0] = 1;
}

bool gm_params_ok(const dgf_gm_params* g)
{
    return g && g->version == DGF_GM_PARAMS_VERSION && g->stride >= 1 && g->extra_levels >= 0 && g->iters >= 1 &&
           g->iters <= 64 && g->c0 > 0 && g->c_min > 0;
}

// Workspace layout: [a[6], flags, ticket; 256 B] [first-pass flow, n_sub x 8 B] [first-pass status, n_sub B]
// [per-CTA partial sums, 64 x 13 doubles]
size_t flow_offset() { return 256; }
size_t status_offset(long long n_sub) { return dgf::round_up(flow_offset() + (size_t)n_sub * 8, 256); }
size_t partial_offset(long long n_sub) { return dgf::round_up(status_offset(n_sub) + (size_t)n_sub, 256); }
constexpr size_t kPartialBytes = (size_t)kPartBlocks * (kSums + 1) * 8;

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
    return dgf::round_up(partial_offset(n_sub) + kPartialBytes, 256);
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
    double* partial = reinterpret_cast<double*>(ws + partial_offset(n_sub));
    gm_init_kernel<<<1, 1, 0, stream>>>(affine);
    for (int k = 0; k < g->iters; ++k) {
        gm_iteration_kernel<<<kPartBlocks, kPartThreads, 0, stream>>>(pts, g->stride, sub_flow, sub_status,
                                                                       (int)n_sub, k, g->c0, g->c_min, affine, partial);
    }
    if ((rc = dgf::launch_status()) != DGF_OK) return rc;
    // 3. main pass from the prior
    main.pyr_levels = pyr_levels;
    main.n_jobs = 1;
    main.total = n;
    main.jobs[0] = dgf::TrackJob{static_cast<const char*>(pyr1), static_cast<const char*>(pyr2), W, H, pts, flow, status,
                                 iters, illum, 0, 1, affine};
    return dgf::launch_track(main, p, stream);
}
