// Status strings, version query and the device status word of the C ABI.
#include <mutex>

#include "common.cuh"

extern "C" const char* dgf_strerror(int code)
{
    switch (code) {
        case DGF_OK: return "ok";
        case DGF_ERR_ARG: return "invalid argument";
        case DGF_ERR_WORKSPACE: return "buffer smaller than the size query requires";
        case DGF_ERR_LEVELS: return "coarsest pyramid level smaller than the support";
        case DGF_ERR_CUDA: return "CUDA launch or runtime error";
        case DGF_ERR_TIMEOUT: return "bounded wait expired";
        case DGF_ERR_DEVICE: return "kernel reported an error";
        default: return "unknown status";
    }
}

extern "C" int dgf_version(void) { return 100; }

namespace {

// DGF_DEV_* bits of the device-side failures on each device that loaded the library.
__device__ unsigned g_status_word;

constexpr int kMaxDevices = 64;

}  // namespace

unsigned* dgf::status_word()
{
    static unsigned* addr[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
        addr[dev] = static_cast<unsigned*>(p);
    }
    return addr[dev];
}

extern "C" int dgf_device_status(unsigned* bits, int reset)
{
    if (!bits) return DGF_ERR_ARG;
    if (!dgf::status_word()) return DGF_ERR_CUDA;
    if (cudaMemcpyFromSymbol(bits, g_status_word, sizeof(unsigned)) != cudaSuccess) return DGF_ERR_CUDA;
    if (reset) {
        const unsigned zero = 0;
        if (cudaMemcpyToSymbol(g_status_word, &zero, sizeof(unsigned)) != cudaSuccess) return DGF_ERR_CUDA;
    }
    return DGF_OK;
}
