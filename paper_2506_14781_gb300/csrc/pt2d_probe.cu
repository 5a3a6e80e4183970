// Read-bandwidth probe (include/pt2d.h, pt2d_diag_read_bandwidth): the L2 and
// HBM read ceilings against which the memory traffic of the sweep kernels is
// judged (the measured HBM copy peak of the machine has no L2 counterpart).
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/pt2d.h"

namespace {

// `iters` passes of 16-byte loads over the buffer, cached in L2 only (.cg), so
// a buffer well below the L2 size is served by L2 after the first pass.  The
// loaded words are folded into one value per thread, which is stored only when
// it equals a fixed constant: the loads cannot be dropped, the store almost
// never happens and the result does not matter.
__global__ void k_read_probe(const uint4 *__restrict__ buf, int64_t n16, int32_t iters, uint32_t *out) {
    uint32_t acc = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t first = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int32_t it = 0; it < iters; ++it) {
        for (int64_t i = first; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9E3779B9u) out[0] = acc;
}

}  // namespace

extern "C" int pt2d_diag_read_bandwidth(const void *device_buf, size_t bytes, int32_t iters, void *device_out,
                                        float *ms) {
    if (!device_buf || !device_out || !ms || bytes < 16 || bytes % 16 || iters < 1 ||
        reinterpret_cast<uintptr_t>(device_buf) % 16 || reinterpret_cast<uintptr_t>(device_out) % 4)
        return PT2D_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return PT2D_ERR_UNSUPPORTED;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
        k_read_probe<<<static_cast<unsigned>(sms) * 8, 256>>>(static_cast<const uint4 *>(device_buf),
                                                               static_cast<int64_t>(bytes / 16), iters,
                                                               static_cast<uint32_t *>(device_out));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e == cudaSuccess ? PT2D_OK : PT2D_ERR_CUDA;
}
