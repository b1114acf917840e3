// bbp_qr_batched: the truncation step of the zip-up fit (App. A) as a standalone call.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "bbp.h"
#include "bbp_internal.h"
#include "engine.h"

using namespace bbp;

extern "C" int bbp_qr_batched(int batch, int m, int n, int complex_values, const double* A, double* Q, double* loss,
                              void* stream) try {
    if (batch < 1 || n < 1 || m < n || n > 512 || !A || !Q)
        return fail(BBP_ERR_INVALID, "qr_batched: need batch >= 1, 1 <= n <= m, n <= 512 and non-NULL A, Q");
    const size_t ss = complex_values ? 16 : 8;
    const size_t mat = (size_t)m * n;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<QRTask> ts(batch);
    void* work = nullptr;
    QRTask* d_ts = nullptr;
    cudaError_t e = cudaMallocAsync(&work, (size_t)batch * 2 * mat * ss, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_ts, (size_t)batch * sizeof(QRTask), st);
    if (e != cudaSuccess) {
        if (work) cudaFreeAsync(work, st);
        return fail(BBP_ERR_OOM, std::string("qr_batched: ") + cudaGetErrorString(e));
    }
    for (int b = 0; b < batch; ++b) {
        QRTask& t = ts[b];
        t = QRTask{};
        t.in = (const char*)A + b * mat * ss;
        t.out = (char*)Q + b * mat * ss;
        t.work = (char*)work + b * 2 * mat * ss;
        t.loss = loss ? loss + b : nullptr;
        t.m = m;
        t.n = n;
        t.in_rs = n; t.in_cs = 1; t.out_rs = n; t.out_cs = 1;
    }
    e = cudaMemcpyAsync(d_ts, ts.data(), ts.size() * sizeof(QRTask), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = qr_prepare(m, complex_values != 0);
    if (e == cudaSuccess) e = launch_qr(d_ts, batch, m, (long long)m * n, complex_values != 0, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // ts is released on return
    cudaFreeAsync(d_ts, st);
    cudaFreeAsync(work, st);
    if (e != cudaSuccess) return fail(BBP_ERR_CUDA, std::string("qr_batched: ") + cudaGetErrorString(e));
    return BBP_OK;
} catch (...) {
    return abi_error();
}
