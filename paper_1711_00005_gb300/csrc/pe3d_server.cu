// pe3d_server.cu -- request loop (continuous batching); placeholder until built.
#include "pe3d_internal.h"

using namespace pe3d_host;

extern "C" {
int pe3d_server_create(size_t, int, int, pe3d_server_t* out) {
    if (out) *out = nullptr;
    return fail(PE3D_ERR_STATE, "request loop not built yet");
}
int pe3d_submit(pe3d_server_t, const pe3d_request*, uint64_t*) { return fail(PE3D_ERR_STATE, "request loop not built yet"); }
int pe3d_poll(pe3d_server_t, uint64_t, int*, void*, double*) { return fail(PE3D_ERR_STATE, "request loop not built yet"); }
int pe3d_server_destroy(pe3d_server_t) { return PE3D_OK; }
int pe3d_server_stats(pe3d_server_t, int64_t*, int) { return fail(PE3D_ERR_STATE, "request loop not built yet"); }
}
