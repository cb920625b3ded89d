// Shared helpers of the CUDA library: the public ABI, the pyramid geometry used by
// host and device code alike, storage-type loads and stores, and launch-error
// mapping.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "degraf.h"

namespace dgf {

// Loads and stores of pyramid samples; both storage types widen to FP32.
__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }

// Asynchronous 4-byte global-to-shared copy (cp.async, sm_80+) and the wait for all of
// the thread's outstanding copies. Both addresses must be 4-byte aligned.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bulk asynchronous copies (cp.async.bulk: the tensor-memory-access engine's
// untiled form, sm_90+) of contiguous global bytes into shared memory, completed
// on a shared-memory mbarrier that counts the bytes. Source and destination must
// be 16-byte aligned and the size a multiple of 16.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// One arrival that also announces the bytes the phase's copies will deliver.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_to_smem(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Waits for phase `parity` of the barrier to complete, giving up after max_tries
// polls (each may suspend the thread for a short while); returns false then.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned max_tries)
{
    const unsigned a = smem_addr(bar);
    for (unsigned i = 0; i < max_tries; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// Polls of a staging wait before a block gives up on its copies (far beyond the
// microseconds a copy takes; reaching it means the copy engine stopped answering).
constexpr unsigned kStageWaitTries = 1u << 22;

// Device address of the library's status word on the current device (the DGF_DEV_*
// bits of the device-side failures since the last reset; read by
// dgf_device_status), or null if it cannot be looked up. The first call on a device
// looks the address up (outside any stream capture); later calls return the cached
// value.
unsigned* status_word();

// Rounds v up to a multiple of a, a power of two.
__host__ __device__ __forceinline__ size_t round_up(size_t v, size_t a) { return (v + a - 1) & ~(a - 1); }

// Width of the replicated border (apron) around every pyramid plane, in pixels
// (DGF_PYR_APRON): pixel (x, y) of a plane may be read for x in [-A, W + A) and
// y in [-A, H + A), and outside [0, W) x [0, H) it holds the value at the clamped
// position. Tracking reads its bilinear taps without clamping; A covers the taps of
// the largest support (radius 7) around any position in, or half a pixel beyond, a
// level. Each row starts 128 bytes before its pixel 0 (the left apron in the last
// A elements of that space), so every row of the level itself starts on a 128-byte
// boundary, as the builder's full-line stores want.
constexpr int kApron = DGF_PYR_APRON;

// Geometry of one pyramid level inside a pyramid buffer (see dgf_pyramid_layout):
// planes I_0..I_{L-1}, then Ix_0..Ix_{L-1}, Iy_0..Iy_{L-1}; each plane (its apron
// included) starts on a 256-byte boundary, rows are padded to 128 bytes.
struct LevelGeom {
    int W, H, pitch;            // size and row pitch (elements)
    size_t off_I, off_Ix, off_Iy;  // byte offsets of pixel (0, 0) (gradient offsets valid when built with them)
    size_t bytes_all, bytes_intensity;  // buffer size with / without gradient planes
};

// Level l of a W x H frame with `levels` levels of element size es (4 or 2).
// Returns false when a level up to `levels - 1` is empty.
__host__ __device__ inline bool level_geom(int W, int H, int levels, int es, int l, LevelGeom* g)
{
    size_t pre = 0, tot = 0;
    int w = W, h = H;
    for (int k = 0; k < levels; ++k) {
        if (w < 1 || h < 1) return false;
        const int lead = 128 / es;  // elements before pixel 0 of a row (>= kApron)
        const int pitch = (int)round_up((size_t)w + lead + kApron, (size_t)(128 / es));
        const size_t plane = round_up((size_t)pitch * (h + 2 * kApron) * es, 256);
        if (k == l) {
            g->W = w;
            g->H = h;
            g->pitch = pitch;
            pre = tot + ((size_t)kApron * pitch + lead) * es;
        }
        tot += plane;
        w /= 2;
        h /= 2;
    }
    g->off_I = pre;
    g->off_Ix = tot + pre;
    g->off_Iy = 2 * tot + pre;
    g->bytes_all = 3 * tot;
    g->bytes_intensity = tot;
    return true;
}

inline int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DGF_OK : DGF_ERR_CUDA;
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace dgf
