// Launch descriptors shared by the single-frame entry points and the batched
// pipeline: every kernel takes its jobs as a __grid_constant__ parameter block, so
// a batch needs no descriptor copy to device memory (and stays capturable in a
// CUDA graph).
#pragma once
#include "common.cuh"

namespace dgf {

constexpr int kMaxBatchPairs = 64;  // pairs per batched launch (longer batches are split)

// One frame's pyramid build.
struct PyrFrame {
    const uint8_t* img;
    int W, H, pitch, with_grad;
    char* base;     // pyramid buffer
    int cta_begin;  // first CTA of this frame in the launch
    int bulk;       // set by launch_pyramids: frame base, pitch and width multiples of 16 (bulk row copies)
};

struct PyrBatch {
    int levels, n_frames;
    unsigned* status;  // the device status word (nullable)
    PyrFrame frames[2 * kMaxBatchPairs];
};

int launch_pyramids(PyrBatch& a, int storage, cudaStream_t stream);

// One frame's DeGraF detection.
struct DetectJob {
    const uint8_t* img;
    int W, H, pitch, step, nu, nv;
    float* pts;
    int32_t* sums;
    int cta_begin;  // first CTA of this frame in the launch
    int tiles_x;    // CTAs per row of windows
    int bulk;       // set by launch_detect: frame base, pitch and width multiples of 16 (bulk row copies)
};

struct DetectBatch {
    int ww, wh, by, vr, staged, tile_w, tile_h, n_jobs;  // vr: windows per thread along y
    unsigned* status;  // the device status word (nullable)
    DetectJob jobs[kMaxBatchPairs];
};

int launch_detect(DetectBatch& a, cudaStream_t stream);

// One pair's tracking job: pyramids of both frames, start points and outputs.
struct TrackJob {
    const char* pyr1;  // frame 1 pyramid with gradients
    const char* pyr2;  // frame 2 pyramid (intensity planes used)
    int W, H;
    const float* pts;
    float* flow;
    uint8_t* status;
    uint8_t* iters;
    float* illum;
    int pt_begin;         // prefix count of points over the jobs of the launch
    int pt_stride;        // point k of the job is pts[k * pt_stride] (1: all points)
    const double* prior;  // global affine motion (6 doubles, device) or null
    const uint8_t* gate;  // nullable: point k is tracked only if gate[k] is TRACKED or MAXITER;
                          // otherwise its status is gate[k] and its flow 0
};

// Parameters and jobs of one tracking launch (a single pair or a batch).
struct TrackBatch {
    int levels, pyr_levels, radius, max_iter, es;  // pyr_levels: levels the pyramids were built with
    float eps2, ha, hc, inv_cb, min_eig, cross_tau;  // cross_tau > 0: adaptive cross-based support
    int n_jobs, total;  // jobs, and points over all jobs
    TrackJob jobs[kMaxBatchPairs];
};

int prepare_params(const dgf_rlof_params* p, TrackBatch& a);
int check_levels(int W, int H, const dgf_rlof_params* p);
// lanes_set: the lanes-per-point setting to launch with (dgf_rlof_set_lanes; 0 is the
// automatic choice); -1 reads the current setting.
int launch_track(const TrackBatch& a, const dgf_rlof_params* p, cudaStream_t stream, int lanes_set = -1);
int lanes_setting();

}  // namespace dgf
