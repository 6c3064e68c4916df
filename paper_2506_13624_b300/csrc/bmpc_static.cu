/*
 * Batch creation with the solver scratch held inside the library.
 *
 * Some callers cannot allocate device memory at solve time: real-time control
 * loops whose safety rules forbid dynamic allocation once the controller runs,
 * plug-ins whose host framework owns every device buffer, and embedded targets
 * that size all memory statically.  bmpc_create_batch_static lets them run the
 * solver without a scratch arena: the per-node Jacobians, Riccati factors and
 * search directions live in one file-scope device array of fixed size that is
 * part of the library image.  The caller still provides the data arena
 * (problem tables, inputs, outputs, statistics) exactly as for
 * bmpc_create_batch, and uses bmpc_set_problems / bmpc_solve_batch /
 * bmpc_get_solutions unchanged on the returned handle.
 */
#include <cuda_runtime.h>

#include "../../include/bmpc.h"

namespace {

/* Fixed solver scratch: BMPC_STATIC_SCRATCH_BYTES, kept by every GPU that loads the library until
 * the process exits.  Nothing in it has to start at zero: every solve writes each scratch entry
 * before reading it. */
static __device__ __align__(256) unsigned char g_static_scratch[BMPC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};

/* Device address of the scratch array on the current device, looked up once per device. */
int static_scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BMPC_ERR_CUDA;
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return BMPC_ERR_CUDA;
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return BMPC_OK;
}

}  // namespace

extern "C" int bmpc_create_batch_static(const bmpc_tree_desc *descs, int32_t n, void *dev_data, size_t data_bytes,
                                        void *host_staging, size_t staging_bytes, void *stream, bmpc_batch **out) {
    if (!out) return BMPC_ERR_INVALID;
    *out = nullptr;
    size_t need_d = 0, need_s = 0, need_h = 0;
    int st = bmpc_batch_bytes(descs, n, &need_d, &need_s, &need_h);
    if (st != BMPC_OK) return st;
    if (need_s > (size_t)BMPC_STATIC_SCRATCH_BYTES) return BMPC_ERR_SPACE;   /* batch too large for the array */
    void *scratch = nullptr;
    st = static_scratch_address(&scratch);
    if (st != BMPC_OK) return st;
    return bmpc_create_batch(descs, n, dev_data, data_bytes, scratch, (size_t)BMPC_STATIC_SCRATCH_BYTES,
                             host_staging, staging_bytes, stream, out);
}
