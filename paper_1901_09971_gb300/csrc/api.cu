// Status strings and version query of the C ABI.
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
