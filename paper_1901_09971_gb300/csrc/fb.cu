// Forward-backward consistency filter on tracked points. The paper does not describe
// one; it is the common check on sparse tracks before interpolation: track forward,
// track the end points backward with the same parameters, and measure how far the
// round trip lands from the start.
//
// Four launches on the caller's stream: forward tracking, the end points p + f, the
// backward tracking (frame 2's pyramid as the template; points the forward pass
// lost are gated out), and the round-trip error with the status update. The two
// element-wise kernels move 17 and 25 bytes per point.
#include "common.cuh"
#include "batch.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fb_endpoints_kernel(const float2* pts, const float2* flow, float2* q,
                                                                int n)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const float2 p = pts[i], f = flow[i];
    q[i] = make_float2(p.x + f.x, p.y + f.y);
}

__device__ __forceinline__ bool tracked(uint8_t s) { return s == DGF_TRACKED || s == DGF_MAXITER; }

__global__ void __launch_bounds__(kThreads) fb_finish_kernel(const float2* flow, uint8_t* status, const float2* bflow,
                                                             const uint8_t* bstatus, float* fb_err, float fb_max,
                                                             int n)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint8_t s = status[i];
    float e = __int_as_float(0x7f800000);  // +inf
    if (tracked(s) && tracked(bstatus[i])) {
        const float2 f = flow[i], b = bflow[i];
        const float dx = f.x + b.x, dy = f.y + b.y;
        e = sqrtf(dx * dx + dy * dy);
    }
    if (fb_err) fb_err[i] = e;
    if (fb_max > 0.f && tracked(s) && e > fb_max) status[i] = DGF_FB_REJECTED;
}

// Workspace layout: [end points, n x 8 B] [backward flow, n x 8 B] [backward status, n B]
size_t bflow_offset(int n) { return dgf::round_up((size_t)n * 8, 256); }
size_t bstatus_offset(int n) { return bflow_offset(n) + dgf::round_up((size_t)n * 8, 256); }

}  // namespace

extern "C" size_t dgf_fb_workspace(int n)
{
    if (n < 0) return 0;
    return dgf::round_up(bstatus_offset(n) + (size_t)n, 256);
}

extern "C" int rlof_track_fb(const void* pyr1, const void* pyr2, size_t pyr_bytes, int W, int H, const float* pts,
                             int n, const dgf_rlof_params* p, float fb_max, float* flow, uint8_t* status,
                             float* fb_err, void* workspace, size_t ws_bytes, cudaStream_t stream)
{
    dgf::TrackBatch a = {};
    int rc = dgf::prepare_params(p, a);
    if (rc != DGF_OK) return rc;
    if (n < 0 || W < 1 || H < 1 || !(fb_max >= 0.f)) return DGF_ERR_ARG;
    if ((rc = dgf::check_levels(W, H, p)) != DGF_OK) return rc;
    const size_t need = dgf_pyramid_bytes(W, H, p->levels, p->storage, 1);
    if (need == 0 || pyr_bytes < need) return DGF_ERR_ARG;  // both pyramids need their gradient planes
    if (n == 0) return DGF_OK;
    if (!pyr1 || !pyr2 || !pts || !flow || !status || !workspace || !dgf::aligned(pyr1, 256) ||
        !dgf::aligned(pyr2, 256) || !dgf::aligned(pts, 8) || !dgf::aligned(flow, 8) ||
        (fb_err && !dgf::aligned(fb_err, 4)) || !dgf::aligned(workspace, 256))
        return DGF_ERR_ARG;
    if (ws_bytes < dgf_fb_workspace(n)) return DGF_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    float2* q = reinterpret_cast<float2*>(ws);
    float2* bflow = reinterpret_cast<float2*>(ws + bflow_offset(n));
    uint8_t* bstatus = reinterpret_cast<uint8_t*>(ws + bstatus_offset(n));
    const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);

    a.n_jobs = 1;
    a.total = n;
    a.jobs[0] = dgf::TrackJob{static_cast<const char*>(pyr1), static_cast<const char*>(pyr2), W, H, pts, flow, status,
                              nullptr, nullptr, 0, 1, nullptr};
    if ((rc = dgf::launch_track(a, p, stream)) != DGF_OK) return rc;
    fb_endpoints_kernel<<<grid, kThreads, 0, stream>>>(reinterpret_cast<const float2*>(pts),
                                                       reinterpret_cast<const float2*>(flow), q, n);
    if ((rc = dgf::launch_status()) != DGF_OK) return rc;
    // backward pass only for forward-tracked points (a point the forward pass lost
    // has an infinite round-trip error whatever the backward pass finds)
    a.jobs[0] = dgf::TrackJob{static_cast<const char*>(pyr2), static_cast<const char*>(pyr1), W, H,
                              reinterpret_cast<const float*>(q), reinterpret_cast<float*>(bflow), bstatus, nullptr,
                              nullptr, 0, 1, nullptr, status};
    if ((rc = dgf::launch_track(a, p, stream)) != DGF_OK) return rc;
    fb_finish_kernel<<<grid, kThreads, 0, stream>>>(reinterpret_cast<const float2*>(flow), status, bflow, bstatus,
                                                    fb_err, fb_max, n);
    return dgf::launch_status();
}
