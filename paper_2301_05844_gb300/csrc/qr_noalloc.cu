// bbp_qr_batched_noalloc: the batched QR of bbp_qr_batched without any device
// allocation.  Its workspace and task descriptors live in a file-scope device array.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "bbp.h"
#include "bbp_internal.h"
#include "engine.h"

using namespace bbp;

// Fixed workspace: task descriptors followed by 2*m*n scalars per matrix.  Every GPU
// that loads the library holds these 16 MiB until the process exits.
static __device__ __align__(256) unsigned char g_qr_scratch[BBP_QR_NOALLOC_SCRATCH_BYTES];

// The header states the descriptor bytes a request needs (144 per matrix).
static_assert(sizeof(QRTask) == 144, "bbp.h states 144 descriptor bytes per matrix");

namespace {
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_qr_scratch, per device
std::mutex g_setup_mu;                   // serialises the first call on each device

// Task descriptors are built on the device, so the call needs no host staging buffer.
__global__ void k_build_qr_tasks(QRTask* tasks, int batch, int m, int n, size_t ss, const double* A, double* Q,
                                 double* loss, unsigned char* work) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const size_t mat = (size_t)m * n;
    QRTask t{};
    t.in = (const unsigned char*)A + b * mat * ss;
    t.out = (unsigned char*)Q + b * mat * ss;
    t.work = work + b * 2 * mat * ss;
    t.loss = loss ? loss + b : nullptr;
    t.m = m;
    t.n = n;
    t.in_rs = n;
    t.in_cs = 1;
    t.out_rs = n;
    t.out_cs = 1;
    tasks[b] = t;
}
}  // namespace

extern "C" int bbp_qr_batched_noalloc(int batch, int m, int n, int complex_values, const double* A, double* Q,
                                      double* loss, void* stream) try {
    if (batch < 1 || n < 1 || m < n || n > 512 || !A || !Q)
        return fail(BBP_ERR_INVALID, "qr_batched_noalloc: need batch >= 1, 1 <= n <= m, n <= 512 and non-NULL A, Q");
    const size_t ss = complex_values ? 16 : 8;
    const size_t task_bytes = ((size_t)batch * sizeof(QRTask) + 255) & ~(size_t)255;
    const size_t need = task_bytes + (size_t)batch * 2 * m * (size_t)n * ss;
    if (need > BBP_QR_NOALLOC_SCRATCH_BYTES)
        return fail(BBP_ERR_INVALID, "qr_batched_noalloc: batch * (2*m*n scalars) exceeds the fixed " +
                                         std::to_string(BBP_QR_NOALLOC_SCRATCH_BYTES) + "-byte workspace");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(BBP_ERR_CUDA, std::string("qr_batched_noalloc: no current device: ") + cudaGetErrorString(e));
    void* addr = nullptr;
    {
        std::lock_guard<std::mutex> guard(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            // first call on this device: resolve the device address of the array (the host-side
            // symbol is only a stand-in; under lazy module loading this also loads the module and
            // commits the array) and raise the QR kernels' shared-memory limits for both scalar
            // types, so that no later call changes a kernel attribute
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_qr_scratch);
            if (e != cudaSuccess || !p) {
                const bool oom = e == cudaErrorMemoryAllocation;
                return fail(oom ? BBP_ERR_OOM : BBP_ERR_CUDA,
                            std::string("qr_batched_noalloc: workspace address: ") + cudaGetErrorString(e));
            }
            e = qr_prepare(512, false);
            if (e == cudaSuccess) e = qr_prepare(512, true);
            if (e != cudaSuccess)
                return fail(e == cudaErrorMemoryAllocation ? BBP_ERR_OOM : BBP_ERR_CUDA,
                            std::string("qr_batched_noalloc: ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        addr = g_scratch_addr[dev];
    }
    // a no-op unless m is above the 512 rows prepared at the first call (the limit only grows)
    e = qr_prepare(m, complex_values != 0);
    if (e != cudaSuccess) return fail(BBP_ERR_CUDA, std::string("qr_batched_noalloc: ") + cudaGetErrorString(e));
    unsigned char* base = (unsigned char*)addr;
    QRTask* tasks = (QRTask*)base;
    cudaStream_t st = (cudaStream_t)stream;
    k_build_qr_tasks<<<(batch + 127) / 128, 128, 0, st>>>(tasks, batch, m, n, ss, A, Q, loss, base + task_bytes);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_qr(tasks, batch, m, (long long)m * n, complex_values != 0, st);
    if (e != cudaSuccess) return fail(BBP_ERR_CUDA, std::string("qr_batched_noalloc: ") + cudaGetErrorString(e));
    return BBP_OK;
} catch (...) {
    return abi_error();
}
