// FP32 throughput probe: the measured ceiling of the tracking kernel's roofline.
//
// The tracking iteration is bound by FP32 issue, not by memory, so its roofline
// denominator is the rate at which this GPU retires fused multiply-adds. The probe
// runs independent FMA chains in every thread of a full grid, either as scalar FFMA
// or as packed FP32x2 FMA (fma.rn.f32x2, sm_100+), the form the tracking kernel
// uses. The caller times the launch and divides dgf_fp32_probe_flops() by it.
#include "common.cuh"

namespace {

constexpr int kChains = 8;   // independent accumulators per thread
constexpr int kRepeat = 8;   // chain steps per loop trip (keeps loop overhead near 2%)

template <bool PACKED>
__global__ void __launch_bounds__(256) fp32_probe_kernel(float* out, int iters, float m, float c)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (PACKED) {
        float2 v[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) v[k] = make_float2(0.25f * k + tid * 1e-7f, 0.5f - 0.125f * k);
        const float2 mm = make_float2(m, m), cc = make_float2(c, c);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kRepeat; ++r) {
#pragma unroll
                for (int k = 0; k < kChains; ++k) v[k] = __ffma2_rn(v[k], mm, cc);
            }
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += v[k].x + v[k].y;
        out[tid] = s;
    } else {
        float v[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) v[k] = 0.25f * k + tid * 1e-7f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kRepeat; ++r) {
#pragma unroll
                for (int k = 0; k < kChains; ++k) v[k] = fmaf(v[k], m, c);
            }
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += v[k];
        out[tid] = s;
    }
}

}  // namespace

extern "C" double dgf_fp32_probe_flops(int blocks, int threads, int iters, int packed)
{
    return 2.0 * (packed ? 2.0 : 1.0) * kChains * kRepeat * (double)iters * (double)threads * (double)blocks;
}

extern "C" int dgf_fp32_probe(float* out, int blocks, int threads, int iters, int packed, cudaStream_t stream)
{
    if (!out || blocks < 1 || threads < 32 || threads > 256 || threads % 32 != 0 || iters < 1) return DGF_ERR_ARG;
    // v <- v m + c with m = 1/2, c = 1 stays in [0.5, 2]: no overflow, no subnormals
    if (packed)
        fp32_probe_kernel<true><<<blocks, threads, 0, stream>>>(out, iters, 0.5f, 1.0f);
    else
        fp32_probe_kernel<false><<<blocks, threads, 0, stream>>>(out, iters, 0.5f, 1.0f);
    return dgf::launch_status();
}
