// Status strings and version of the C ABI.
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
