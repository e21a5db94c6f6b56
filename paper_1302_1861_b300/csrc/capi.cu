// Error reporting and small C-ABI helpers of the PSL library.
#include <cuda_runtime.h>

#include <string>

#include "psl_internal.cuh"

static thread_local std::string g_last_error;

void psl_set_error(const std::string &msg) { g_last_error = msg; }

int psl_fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

extern "C" const char *psl_last_error(void) { return g_last_error.c_str(); }

extern "C" void psl_physics_default(psl_physics_t *out) {
    if (!out) return;
    out->photon_cut = 0.010f;                        // Sec. 2.6
    out->electron_cut = (float)(0.700 - 0.51099895);  // 0.700 MeV total energy, Sec. 2.6
    out->wcc = 0.200f;
    out->wcb = 0.200f;
    out->flags = 0u;
}
