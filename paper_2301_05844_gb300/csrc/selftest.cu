// bbp_selftest_gemm: runs the tensor-core GEMM on host matrices (diagnostics).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "bbp.h"
#include "engine.h"
#include "tc_gemm.h"

using namespace bbp;

// The GEMM of bbp_selftest_gemm; stall: launch with the producer's copies withheld.
static int selftest_gemm(int M, int N, int K, int prec, const float* A, const float* B, float* C, int stall) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || (prec != BBP_PREC_TF32 && prec != BBP_PREC_BF16))
        return fail(BBP_ERR_INVALID, "selftest: bad arguments");
    const int kind = prec == BBP_PREC_TF32 ? 0 : 1;
    const int esz = kind == 0 ? 4 : 2;
    const long long ld = ((long long)K * esz + 15) / 16 * 16 / esz;  // 16-byte row pitch
    std::vector<unsigned char> ha((size_t)M * ld * esz, 0), hb((size_t)N * ld * esz, 0);
    for (long long i = 0; i < M; ++i)
        for (long long k = 0; k < K; ++k) {
            if (kind == 0) ((float*)ha.data())[i * ld + k] = A[i * K + k];
            else ((__nv_bfloat16*)ha.data())[i * ld + k] = __float2bfloat16_rn(A[i * K + k]);
        }
    for (long long i = 0; i < N; ++i)
        for (long long k = 0; k < K; ++k) {
            if (kind == 0) ((float*)hb.data())[i * ld + k] = B[i * K + k];
            else ((__nv_bfloat16*)hb.data())[i * ld + k] = __float2bfloat16_rn(B[i * K + k]);
        }
    void *da = nullptr, *db = nullptr, *dc = nullptr, *dt = nullptr;
    int* derr = nullptr;
    int rc = BBP_OK;
    const int bn = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    cudaError_t e = cudaMalloc(&da, ha.size());
    if (!e) e = cudaMalloc(&db, hb.size());
    if (!e) e = cudaMalloc(&dc, (size_t)M * N * 4);
    if (!e) e = cudaMalloc(&dt, sizeof(TCTask));
    if (!e) e = cudaMalloc((void**)&derr, sizeof(int));
    if (!e) e = cudaMemcpy(da, ha.data(), ha.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(db, hb.data(), hb.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(dc, 0, (size_t)M * N * 4);
    if (!e) e = cudaMemset(derr, 0, sizeof(int));
    TCTask t{};
    if (!e) e = tc_make_map(&t.map_a, da, kind, M, K, ld, 128);
    if (!e) e = tc_make_map(&t.map_b, db, kind, N, K, ld, bn);
    t.M = M; t.N = N; t.K = K; t.M2 = M; t.N2 = N; t.out_kind = 0;
    t.nseg = 1;
    t.c_m1 = 0; t.c_m2 = N; t.c_n1 = 0; t.c_n2 = 1;
    t.C = dc; t.C2 = nullptr; t.active = nullptr; t.alpha = 1.0f;
    if (!e) e = cudaMemcpy(dt, &t, sizeof(t), cudaMemcpyHostToDevice);
    if (!e) e = tc_prepare();
    const int tiles = ((M + 127) / 128) * ((N + bn - 1) / bn);
    const int ek = kind == 0 ? 32 : 64;
    const int nk = (K + ek - 1) / ek;
    if (!e) e = launch_tc_gemm((const TCTask*)dt, 1, kind, bn, tiles, tc_default_stages(bn, nk), derr, 0, 1, stall);
    if (!e) e = cudaDeviceSynchronize();
    int herr = 0;
    if (!e) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(C, dc, (size_t)M * N * 4, cudaMemcpyDeviceToHost);
    if (e) rc = fail(BBP_ERR_CUDA, std::string("selftest: ") + cudaGetErrorString(e));
    else if (herr) rc = fail(BBP_ERR_TIMEOUT, "selftest: a pipeline wait timed out");
    cudaFree(da); cudaFree(db); cudaFree(dc); cudaFree(dt); cudaFree(derr);
    return rc;
}

extern "C" int bbp_selftest_gemm(int M, int N, int K, int prec, const float* A, const float* B, float* C) try {
    return selftest_gemm(M, N, K, prec, A, B, C, 0);
} catch (...) {
    return abi_error();
}

extern "C" int bbp_selftest_gemm_timeout(void) try {
    // a 256 x 64 x 64 TF32 GEMM (two tiles) whose operands are never loaded
    std::vector<float> a(256 * 64, 1.0f), b(64 * 64, 1.0f), c(256 * 64, 0.0f);
    return selftest_gemm(256, 64, 64, BBP_PREC_TF32, a.data(), b.data(), c.data(), 1);
} catch (...) {
    return abi_error();
}

extern "C" int bbp_selftest_scalar(long long n, const double* x, double* rsqrt_ours, double* rcp_ours,
                                   double* rsqrt_cuda, double* rcp_cuda) try {
    if (n < 1 || !x || !rsqrt_ours || !rcp_ours || !rsqrt_cuda || !rcp_cuda)
        return fail(BBP_ERR_INVALID, "selftest_scalar: bad arguments");
    for (long long i = 0; i < n; ++i)
        if (!(x[i] >= 0x1p-100 && x[i] <= 0x1p100)) return fail(BBP_ERR_INVALID, "selftest_scalar: x outside [2^-100, 2^100]");
    double* d = nullptr;
    const size_t bytes = (size_t)n * sizeof(double);
    cudaError_t e = cudaMalloc((void**)&d, 5 * bytes);
    if (e) return fail(BBP_ERR_OOM, std::string("selftest_scalar: ") + cudaGetErrorString(e));
    e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
    if (!e) e = launch_scalar_selftest(d, n, d + n, d + 2 * n, d + 3 * n, d + 4 * n, 0);
    if (!e) e = cudaDeviceSynchronize();
    double* outs[4] = {rsqrt_ours, rcp_ours, rsqrt_cuda, rcp_cuda};
    for (int k = 0; k < 4 && !e; ++k) e = cudaMemcpy(outs[k], d + (k + 1) * n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e) return fail(BBP_ERR_CUDA, std::string("selftest_scalar: ") + cudaGetErrorString(e));
    return BBP_OK;
} catch (...) {
    return abi_error();
}

extern "C" int bbp_selftest_qr_fp32(int batch, int m, int n, const float* A, double* Q, double* loss,
                                    int* workspace_intact) try {
    if (batch < 1 || n < 1 || m < n || n > 512 || !A || !Q || !workspace_intact)
        return fail(BBP_ERR_INVALID, "selftest_qr_fp32: need batch >= 1, 1 <= n <= m, n <= 512, non-NULL arrays");
    const size_t mat = (size_t)m * n;
    const size_t guard = 512;                    // doubles after each task's 2 m n workspace
    const size_t per = 2 * mat + guard;
    const double pattern = -0x1.5p+77;            // a value no QR writes
    std::vector<QRTask> ts(batch);
    char* d = nullptr;
    const size_t in_b = (size_t)batch * mat * sizeof(float), out_b = (size_t)batch * mat * sizeof(double);
    const size_t work_b = (size_t)batch * per * sizeof(double), loss_b = (size_t)batch * sizeof(double);
    cudaError_t e = cudaMalloc((void**)&d, in_b + out_b + work_b + loss_b + batch * sizeof(QRTask) + 1024);
    if (e) return fail(BBP_ERR_OOM, std::string("selftest_qr_fp32: ") + cudaGetErrorString(e));
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* d_in = d;
    char* d_out = d + al(in_b);
    double* d_work = (double*)(d_out + al(out_b));
    double* d_loss = (double*)((char*)d_work + al(work_b));
    QRTask* d_ts = (QRTask*)((char*)d_loss + al(loss_b));
    std::vector<double> wk((size_t)batch * per, pattern);
    for (int b = 0; b < batch; ++b) {
        QRTask& t = ts[b];
        t = QRTask{};
        t.in = d_in + b * mat * sizeof(float);
        t.in_float = 2;
        t.out = d_out + b * mat * sizeof(double);
        t.work = d_work + b * per;
        t.loss = d_loss + b;
        t.m = m;
        t.n = n;
        t.in_rs = n; t.in_cs = 1; t.out_rs = n; t.out_cs = 1;
    }
    e = cudaMemcpy(d_in, A, in_b, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_work, wk.data(), wk.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_ts, ts.data(), ts.size() * sizeof(QRTask), cudaMemcpyHostToDevice);
    if (!e) e = qr_prepare(m, false);
    if (!e) e = launch_qr(d_ts, batch, m, (long long)mat, false, 0, QR_F32);
    if (!e) e = cudaDeviceSynchronize();
    if (!e) e = cudaMemcpy(Q, d_out, out_b, cudaMemcpyDeviceToHost);
    if (!e && loss) e = cudaMemcpy(loss, d_loss, loss_b, cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(wk.data(), d_work, wk.size() * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e) return fail(BBP_ERR_CUDA, std::string("selftest_qr_fp32: ") + cudaGetErrorString(e));
    int ok = 1;
    for (int b = 0; b < batch; ++b)
        for (size_t i = 2 * mat; i < per; ++i) ok &= wk[(size_t)b * per + i] == pattern;
    *workspace_intact = ok;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

// Layered pair contraction (the read-out's layered site rows) on host arrays: X in the
// layout of a downward row's first intermediate, [(k1 k1')][m1][(k2 k2')][m2], Tk and Tb as
// [p][k1][k2][n1][n2] (placed side by side on the device, the bra at a fixed offset from
// the ket, as the read-out places O T and T), Y as [m1][m2][(n1 n1')][(n2 n2')].
extern "C" int bbp_selftest_layer(int f32, int d, int K1, int K2, int N1, int N2, int M1, int M2, const double* X,
                                  const double* Tk, const double* Tb, double* Y) try {
    if (d < 1 || K1 < 1 || K2 < 1 || N1 < 1 || N2 < 1 || M1 < 1 || M2 < 1 || !X || !Tk || !Tb || !Y)
        return fail(BBP_ERR_INVALID, "selftest_layer: bad arguments");
    const int UL = K1 * K2, DR = N1 * N2;
    const size_t smem = layer_smem_bytes(d, UL, DR, f32 != 0);
    if (UL > 32 || DR > 32 || smem > LAYER_SMEM_MAX) return fail(BBP_ERR_INVALID, "selftest_layer: shape beyond the kernel");
    const long long K1q = (long long)K1 * K1, K2q = (long long)K2 * K2, vol = (long long)UL * DR;
    const size_t nx = (size_t)(K1q * M1 * K2q * M2), nt = (size_t)(d * vol), ny = (size_t)M1 * M2 * DR * DR;
    GTask t{};
    t.layer_d = d;
    t.tb_off = (long long)nt;
    t.M1 = M1; t.M2 = M2; t.K1 = K1; t.K2 = K2; t.N1 = N1; t.N2 = N2;
    t.a_k1 = (long long)M1 * K2q * M2; t.a_m1 = K2q * M2; t.a_k2 = M2; t.a_m2 = 1;
    t.b_k1 = (long long)K2 * DR; t.b_k2 = DR; t.b_n1 = N2; t.b_n2 = 1;
    t.c_m1 = (long long)M2 * DR * DR; t.c_m2 = (long long)DR * DR; t.c_n1 = (long long)N2 * N2; t.c_n2 = 1;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t xb = nx * 8, tb = 2 * nt * 8, yb = ny * 8;
    char* dmem = nullptr;
    cudaError_t e = cudaMalloc((void**)&dmem, al(xb) + al(tb) + al(yb) + al(sizeof(GTask)));
    if (e) return fail(BBP_ERR_OOM, std::string("selftest_layer: ") + cudaGetErrorString(e));
    double* dx = (double*)dmem;
    double* dt = (double*)(dmem + al(xb));
    double* dy = (double*)(dmem + al(xb) + al(tb));
    GTask* dtask = (GTask*)(dmem + al(xb) + al(tb) + al(yb));
    t.A = dx; t.B = dt; t.C = dy;
    e = cudaMemcpy(dx, X, xb, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dt, Tk, nt * 8, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dt + nt, Tb, nt * 8, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dtask, &t, sizeof(GTask), cudaMemcpyHostToDevice);
    if (!e) e = layer_prepare();
    const int apt = f32 ? LAYER_APT_F32 : LAYER_APT_F64;
    const int tiles = M1 * ((M2 + apt - 1) / apt);
    if (!e) e = launch_gcontract(dtask, 1, tiles, false, 0, GC_LAYER | (f32 ? GC_F32 : 0), (long long)smem);
    if (!e) e = cudaDeviceSynchronize();
    if (!e) e = cudaMemcpy(Y, dy, yb, cudaMemcpyDeviceToHost);
    cudaFree(dmem);
    if (e) return fail(BBP_ERR_CUDA, std::string("selftest_layer: ") + cudaGetErrorString(e));
    return BBP_OK;
} catch (...) {
    return abi_error();
}

extern "C" int bbp_selftest_rng(unsigned long long seed, unsigned long long stream, long long n, double* out) try {
    if (n < 0 || (n > 0 && !out)) return fail(BBP_ERR_INVALID, "selftest_rng: bad arguments");
    for (long long i = 0; i < n; ++i) out[i] = bbp::uniform_pm1(seed, stream, (uint64_t)i);
    return BBP_OK;
} catch (...) {
    return abi_error();
}
