// Batched DeGraF + pyramid + RLOF over many frame pairs of uneven size and point
// count (the paper's pipeline, Section 2, applied to a batch of pairs).
//
// Per chunk of up to 64 pairs the stream receives three kinds of launch: one
// detection launch over every frame 1 (per distinct window size), one pyramid
// launch over all 2 x pairs frames, and one tracking launch over every point of
// the chunk (one lane group per point, blocks of eight points, so uneven pairs
// and iteration counts balance through the block scheduler). In a captured graph
// detection runs on a forked branch beside the pyramids. Descriptors travel
// as kernel parameters, so the sequence needs no host-to-device copy and can be
// captured into a CUDA graph; with use_graph = 1 the library captures it once per
// distinct argument set and replays the instantiated graph afterwards.
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "batch.cuh"
#include "common.cuh"

namespace {

struct PairPlan {
    long long n;              // key-points
    size_t pyr1, pyr2;        // workspace offsets of the two pyramids
    size_t pyr1_bytes, pyr2_bytes;
};

// Validates the batch and lays out the workspace: the two pyramids of every pair.
// Returns the bytes needed, or 0 on error.
size_t plan(const dgf_pair* pairs, int n_pairs, const dgf_rlof_params* p, PairPlan* out, int* rc)
{
    *rc = DGF_ERR_ARG;
    if (!pairs || n_pairs < 1 || !p) return 0;
    dgf::TrackBatch probe = {};
    if ((*rc = dgf::prepare_params(p, probe)) != DGF_OK) return 0;
    size_t off = 0;
    for (int i = 0; i < n_pairs; ++i) {
        const dgf_pair& P = pairs[i];
        *rc = DGF_ERR_ARG;
        if (!P.frame1 || !P.frame2 || P.W < 1 || P.H < 1 || P.pitch < P.W) return 0;
        const long long n = dgf_degraf_count(P.W, P.H, P.win, P.win, P.step);
        if (n < 0 || n > 0x7fffffffLL) return 0;
        if (n > 0 && (!P.pts || !P.flow || !P.status || !dgf::aligned(P.pts, 8) || !dgf::aligned(P.flow, 8)))
            return 0;
        if ((*rc = dgf::check_levels(P.W, P.H, p)) != DGF_OK) return 0;
        const size_t b1 = dgf_pyramid_bytes(P.W, P.H, p->levels, p->storage, 1);
        const size_t b2 = dgf_pyramid_bytes(P.W, P.H, p->levels, p->storage, 0);
        if (out) out[i] = PairPlan{n, off, off + b1, b1, b2};
        off += b1 + b2;  // both multiples of 256
    }
    *rc = DGF_OK;
    return off;
}

// Optional fork of detection onto a second stream (used while capturing a graph):
// detection and the pyramids read the frames only, so they become parallel graph
// branches that join before tracking.
struct Fork {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

int enqueue(const dgf_pair* pairs, int n_pairs, const dgf_rlof_params* p, const PairPlan* plans, char* ws,
            int stages, int lanes_set, cudaStream_t stream, const Fork& fk = Fork())
{
    for (int c0 = 0; c0 < n_pairs; c0 += dgf::kMaxBatchPairs) {
        const int cn = n_pairs - c0 < dgf::kMaxBatchPairs ? n_pairs - c0 : dgf::kMaxBatchPairs;
        // detection, one launch per distinct window size (on the side stream when forked)
        const bool forked = fk.side && (stages & DGF_STAGE_DETECT) && (stages & DGF_STAGE_PYRAMID);
        cudaStream_t ds = stream;
        if (forked) {
            if (cudaEventRecord(fk.fork, stream) != cudaSuccess || cudaStreamWaitEvent(fk.side, fk.fork, 0) != cudaSuccess)
                return DGF_ERR_CUDA;
            ds = fk.side;
        }
        bool done[dgf::kMaxBatchPairs] = {};
        for (int i = 0; i < cn && (stages & DGF_STAGE_DETECT); ++i) {
            if (done[i]) continue;
            dgf::DetectBatch d = {};
            d.ww = d.wh = pairs[c0 + i].win;
            for (int j = i; j < cn; ++j) {
                const dgf_pair& P = pairs[c0 + j];
                if (done[j] || P.win != d.ww) continue;
                done[j] = true;
                if (plans[c0 + j].n == 0) continue;
                dgf::DetectJob& J = d.jobs[d.n_jobs++];
                J.img = P.frame1;
                J.W = P.W;
                J.H = P.H;
                J.pitch = P.pitch;
                J.step = P.step;
                J.nu = (P.W - P.win) / P.step + 1;
                J.nv = (P.H - P.win) / P.step + 1;
                J.pts = P.pts;
                J.sums = nullptr;
            }
            if (d.n_jobs) {
                const int rc = dgf::launch_detect(d, ds);
                if (rc != DGF_OK) return rc;
            }
        }
        if (forked && cudaEventRecord(fk.join, fk.side) != cudaSuccess) return DGF_ERR_CUDA;
        // pyramids of both frames of every pair
        dgf::PyrBatch y = {};
        y.levels = p->levels;
        for (int i = 0; i < cn; ++i) {
            const dgf_pair& P = pairs[c0 + i];
            const PairPlan& Q = plans[c0 + i];
            y.frames[y.n_frames++] = dgf::PyrFrame{P.frame1, P.W, P.H, P.pitch, 1, ws + Q.pyr1, 0};
            y.frames[y.n_frames++] = dgf::PyrFrame{P.frame2, P.W, P.H, P.pitch, 0, ws + Q.pyr2, 0};
        }
        int rc = (stages & DGF_STAGE_PYRAMID) ? dgf::launch_pyramids(y, p->storage, stream) : DGF_OK;
        if (rc != DGF_OK) return rc;
        if (forked && cudaStreamWaitEvent(stream, fk.join, 0) != cudaSuccess) return DGF_ERR_CUDA;
        if (!(stages & DGF_STAGE_TRACK)) continue;
        // tracking of every point of the chunk
        dgf::TrackBatch t = {};
        dgf::prepare_params(p, t);
        long long total = 0;
        for (int i = 0; i < cn; ++i) {
            const dgf_pair& P = pairs[c0 + i];
            if (plans[c0 + i].n == 0) continue;
            t.jobs[t.n_jobs++] = dgf::TrackJob{ws + plans[c0 + i].pyr1, ws + plans[c0 + i].pyr2, P.W, P.H, P.pts,
                                               P.flow, P.status, P.iters, nullptr, (int)total, 1, nullptr};
            total += plans[c0 + i].n;
        }
        if (total > 0x7fffffffLL) return DGF_ERR_ARG;
        t.total = (int)total;
        if (total > 0 && (rc = dgf::launch_track(t, p, stream, lanes_set)) != DGF_OK) return rc;
    }
    return DGF_OK;
}

// Instantiated graphs keyed by everything the launches bake in (graph_key).
struct GraphCache {
    std::mutex mu;
    std::unordered_map<std::string, cudaGraphExec_t> map;
};

// Capture happens on a private non-blocking stream per device (the legacy default
// stream cannot be captured); the instantiated graph then runs on the caller's.
// The side stream and events of the fork, created once per device.
Fork capture_fork(int dev)
{
    static Fork forks[64] = {};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) return Fork();
    Fork& f = forks[dev];
    if (!f.side) {
        Fork t;
        if (cudaStreamCreateWithFlags(&t.side, cudaStreamNonBlocking) != cudaSuccess) return Fork();
        if (cudaEventCreateWithFlags(&t.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&t.join, cudaEventDisableTiming) != cudaSuccess) {
            if (t.fork) cudaEventDestroy(t.fork);
            cudaStreamDestroy(t.side);
            return Fork();  // no fork: detection stays on the capture stream
        }
        f = t;
    }
    return f;
}

cudaStream_t capture_stream(int dev)
{
    static cudaStream_t streams[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}

GraphCache& cache()
{
    static GraphCache* c = new GraphCache();  // never destroyed: outlives late callers
    return *c;
}

// The exact argument set a captured graph bakes in, written out field by field (so
// struct padding never enters it): a cache hit replays launches whose arguments all
// equal the caller's.
std::string graph_key(const dgf_pair* pairs, int n_pairs, const dgf_rlof_params* p, const char* ws, int dev,
                      int stages, int lanes)
{
    std::string k;
    k.reserve((size_t)n_pairs * 68 + sizeof(*p) + 24);
    const auto put = [&k](const void* v, size_t n) { k.append(static_cast<const char*>(v), n); };
    for (int i = 0; i < n_pairs; ++i) {
        const dgf_pair& P = pairs[i];
        const void* ptrs[6] = {P.frame1, P.frame2, P.pts, P.flow, P.status, P.iters};
        const int dims[5] = {P.W, P.H, P.pitch, P.win, P.step};
        put(ptrs, sizeof(ptrs));
        put(dims, sizeof(dims));
    }
    put(p, sizeof(*p));  // ints and floats only: no padding
    put(&ws, sizeof(ws));
    const int rest[3] = {dev, stages, lanes};
    put(rest, sizeof(rest));
    return k;
}

}  // namespace

extern "C" size_t dgf_track_many_workspace(const dgf_pair* pairs, int n_pairs, const dgf_rlof_params* p)
{
    int rc;
    return plan(pairs, n_pairs, p, nullptr, &rc);
}

extern "C" int rlof_track_many(const dgf_pair* pairs, int n_pairs, const dgf_rlof_params* p, void* workspace,
                               size_t ws_bytes, int stages, int use_graph, cudaStream_t stream)
{
    if (n_pairs == 0) return DGF_OK;
    if (n_pairs < 0 || stages < 1 || stages > DGF_STAGE_ALL) return DGF_ERR_ARG;
    int rc;
    PairPlan* plans = new PairPlan[n_pairs];
    const size_t need = plan(pairs, n_pairs, p, plans, &rc);
    if (rc == DGF_OK && (!workspace || !dgf::aligned(workspace, 256))) rc = DGF_ERR_ARG;
    if (rc == DGF_OK && ws_bytes < need) rc = DGF_ERR_WORKSPACE;
    if (rc != DGF_OK) {
        delete[] plans;
        return rc;
    }
    char* ws = static_cast<char*>(workspace);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        delete[] plans;
        return DGF_ERR_CUDA;
    }
    // the lanes setting is read once: the graph key and the launches use the same value
    const int lanes_set = dgf::lanes_setting();
    if (!use_graph || cap != cudaStreamCaptureStatusNone) {  // plain launches (also inside a caller's capture)
        rc = enqueue(pairs, n_pairs, p, plans, ws, stages, lanes_set, stream);
        delete[] plans;
        return rc;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    const std::string key =
        graph_key(pairs, n_pairs, p, ws, dev, stages, lanes_set);  // the lanes setting is baked in too
    GraphCache& C = cache();
    std::lock_guard<std::mutex> lock(C.mu);
    auto it = C.map.find(key);
    if (it == C.map.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cs = capture_stream(dev);
        if (!cs || cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            delete[] plans;
            return DGF_ERR_CUDA;
        }
        rc = enqueue(pairs, n_pairs, p, plans, ws, stages, lanes_set, cs, capture_fork(dev));
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        delete[] plans;
        if (rc != DGF_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc != DGF_OK ? rc : DGF_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return DGF_ERR_CUDA;
        if (C.map.size() >= 16) {  // bounded cache: drop everything on overflow
            for (auto& kv : C.map) cudaGraphExecDestroy(kv.second);
            C.map.clear();
        }
        it = C.map.emplace(key, exec).first;
    } else {
        delete[] plans;
    }
    return cudaGraphLaunch(it->second, stream) == cudaSuccess ? DGF_OK : DGF_ERR_CUDA;
}

// ---- single pair without any allocation ------------------------------------
//
// Some callers cannot allocate device memory when they want to track: code that
// must not call cudaMalloc after start-up (real-time loops where an allocation
// could stall or fail, plug-ins whose host application owns all device memory,
// code whose rules forbid dynamic allocation once running). They still own their
// frames and output buffers; what they cannot provide is the pyramid workspace.
// This entry point uses a fixed scratch array compiled into the library instead.
// Every GPU that loads the library holds the array until the process exits.

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)24 << 20;  // DGF_NOALLOC_SCRATCH_BYTES
static_assert(kNoAllocScratchBytes == (size_t)DGF_NOALLOC_SCRATCH_BYTES, "scratch size and header disagree");

// The pyramids of the pair being tracked. Shared by every call: nothing in it
// needs to start at zero (each call rewrites every byte it later reads).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;

// Device address of the scratch array on the current device. The host-side name
// of a __device__ array is only a stand-in, so the address is looked up once per
// device (with that device current) and kept.
void* scratch_address(int dev)
{
    static void* addr[kMaxDevices] = {};
    static std::mutex mu;
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        addr[dev] = p;
    }
    return addr[dev];
}

}  // namespace

extern "C" int rlof_track_pair_noalloc(const dgf_pair* pair, const dgf_rlof_params* p, cudaStream_t stream)
{
    PairPlan plan1;
    int rc;
    const size_t need = plan(pair, 1, p, &plan1, &rc);
    if (rc != DGF_OK) return rc;
    if (need > kNoAllocScratchBytes) return DGF_ERR_WORKSPACE;  // frames too large for the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DGF_ERR_CUDA;
    char* ws = static_cast<char*>(scratch_address(dev));
    if (!ws) return DGF_ERR_CUDA;
    return enqueue(pair, 1, p, &plan1, ws, DGF_STAGE_ALL, dgf::lanes_setting(), stream);
}
