// Status strings, version and the host-mapping query of the C ABI.
#include "tf_host.cuh"

extern "C" const char *twofold_strerror(int status) {
    switch (status) {
    case TF_OK: return "ok";
    case TF_EINVAL: return "invalid argument";
    case TF_ENOSPC: return "workspace too small";
    case TF_ECUDA: return "CUDA error";
    case TF_ETIMEOUT: return "device-side wait timed out";
    case TF_EUNSUPPORTED: return "unsupported request";
    default: return "unknown status";
    }
}

extern "C" int twofold_version(void) { return 100; }

extern "C" int twofold_host_mapped(const void *ptr) {
    if (!ptr) return 0;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == ptr ? 1 : 0;
}
