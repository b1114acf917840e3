// Internal declarations shared by the blockBP CUDA kernels and the host engine.
//
// Every grouped kernel takes a device array of task descriptors; one launch runs
// the same step (for example "left-to-right site update, step 2") for every
// message being computed in the sweep, each with its own pointers and shapes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bbp {

// Strided two-level contraction  C[m][n] (+)= sum_k op(A)[m][k] * B[k][n]
// with m = m1*M2 + m2, n = n1*N2 + n2, k = k1*K2 + k2 and an arbitrary element
// stride for each of the six sub-indices of A and B and four of C.  Every
// contraction of the zip-up fit (Eq. "update", the A/B recurrences), of the MPS
// overlaps and of the read-out closing is one of these.
struct GTask {
    const void* A;
    const void* B;
    void* C;
    int M1, M2, N1, N2, K1, K2;
    long long a_m1, a_m2, a_k1, a_k2;
    long long b_k1, b_k2, b_n1, b_n2;
    long long c_m1, c_m2, c_n1, c_n2;
    int conjA;       // complex: use conj(A)
    int accumulate;  // 1: C += result, 0: C = result
    const int* active;  // task skipped when *active == 0 (nullptr: always runs)
    // layer_d > 0: a layered pair contraction (steps with mode GC_LAYER, real operands) over
    // layer_d physical values instead of the product above.  For every pair (m1, m2) the task
    // reads a matrix over two contracted double legs,
    //   X[(k1 k1')][(k2 k2')] = A[m1 a_m1 + m2 a_m2 + (k1 K1 + k1') a_k1 + (k2 K2 + k2') a_k2],
    // and writes
    //   Y[(n1 n1')][(n2 n2')] = sum_p sum_{k1 k2 k1' k2'} Tk_p[k1 k2 n1 n2] X[(k1 k1')][(k2 k2')] Tb_p[k1' k2' n1' n2']
    // to C[m1 c_m1 + m2 c_m2 + (n1 N1 + n1') c_n1 + (n2 N2 + n2') c_n2]: the contraction of X
    // with the double layer E = sum_p Tk_p (x) Tb_p, without forming E.  Tk_p[k1 k2 n1 n2] is
    // B[p vol + k1 b_k1 + k2 b_k2 + n1 b_n1 + n2 b_n2] (vol = K1 K2 N1 N2), Tb the same view
    // tb_off elements from B (0: the same tensor).  K1 K2 and N1 N2 are at most 32.
    int layer_d;
    long long tb_off;
};

// Householder QR of an m x n matrix (m >= n) read with element (i, j) at
// in[i*in_rs + j*in_cs] (conjugated if conj_io); writes the thin Q, columns scaled
// so that diag(R) is real non-negative, to out[i*out_rs + j*out_cs] (conjugated
// if conj_io).  conj_io with transposed strides turns this into the LQ of the
// right-to-left half sweep.  Also writes -||in||^2 (the fit loss of App. A).
struct QRTask {
    const void* in;
    void* out;
    void* work;      // 2*m*n elements of scratch
    double* loss;    // may be nullptr
    const int* active;
    int m, n;
    long long in_rs, in_cs, out_rs, out_cs;
    int conj_io;
    int in_float;    // 0: input in the FP64 scalar type; 1: FP32 input (mixed path), FP64
                     // arithmetic; 2: FP32 input and FP32 arithmetic (see QR_F32)
    void* out2;      // optional second copy of Q in a low-precision operand layout:
                     // element (i, k) at (i / out2_M2) * out2_rs + (i % out2_M2) * out2_rs2 + k * out2_cs
    long long out2_rs, out2_cs, out2_rs2;
    int out2_kind;   // element kind of out2 (see RelayoutTask)
    int out2_M2;     // >= 1
    int out2_x3;     // split operand (see RelayoutTask); out2_kseg = elements between its planes
    long long out2_kseg;
};

// Strided copy with type conversion over a 4-D index space (dims d0 x d1 x d2 x d3):
//   dst[sum_i i_k * ds_k] = convert(src[sum_i i_k * ss_k]).
// Element kinds: 0 FP64, 2 FP32, 3 BF16, 4 FP32 rounded to TF32 (store only).
struct RelayoutTask {
    const void* src;
    void* dst;
    int d[4];
    long long ss[4];
    long long ds[4];
    int src_kind, dst_kind;
    int x3;          // split operand (see store_split): 0 no; else hi at the destination, lo kseg further
    long long kseg;  // elements from the hi plane to the lo plane
};

// Fill n scalars (2n doubles if complex) with the counter-based uniforms in [-1,1).
struct RandTask {
    void* ptr;
    long long n;
    unsigned long long stream;
    int* active;  // if set, the fit's active flag is reset to 1
    int warm;     // 1: leave the buffer as it is once *warm_ctr > 0 (warm start)
    int pad;
    const int* warm_ctr;  // the lattice's sweep counter (warm tasks)
};

// One zip-up fit's convergence check after a sweep (App. A stop rule).
struct CheckTask {
    const double* losses;  // count values of this sweep
    int* active;
    int* counter;          // incremented for every sweep that ran (fit sweeps executed)
    int count;
    int pad;
};

// Fit-sweep loop state in device memory.  In a CUDA graph the loop body is a
// conditional WHILE node; the check kernel clears the condition once no fit of the
// group is active or `max` sweeps have run.  handle is written after capture.
struct LoopDesc {
    int iter;
    int max;
    unsigned long long handle;
    int use_handle;
    int total;  // iterations run since creation (statistics)
};

// Scale an array by 1/||.||_F (the fitted column MPS in mixed canonical form).
struct ScaleTask {
    void* ptr;
    long long n;
};

// Message assembly: sites 1..nsites of the final column MPS into the message slot,
// the two corner scalars multiplied into the first site.
struct AssembleTask {
    const void* src[16];   // column MPS sites 1..nsites (contiguous [a][k][b])
    void* dst[16];         // message sites (contiguous [a][k][b])
    long long size[16];
    const void* corner0;   // 1x1x1
    const void* corner1;   // 1x1x1
    int nsites;
    int pad;
};

// Message normalisation and residual term: uses <m|m> and <m|m_old> from the
// overlap chains, the identity trace tau (computed here), scales site 0 of the
// message by conj(tau)/|tau|/||m|| and writes ||m_hat - m_old||^2.
struct NormTask {
    void* site0;
    long long size0;
    const void* sites[16];
    int a[16], k[16], b[16];
    int nsites, D;
    int ones;            // phase reference <1|m> (single-layer network) instead of <I|m>
    const void* mm;      // <m|m> (1 scalar)
    const void* mo;      // <m|m_old> (1 scalar)
    double* resid;       // output term
    int* status;         // set nonzero on a zero or non-finite norm
};

// Double layer E[(u u'),(l l'),(d d'),(r r')] = sum_{p,p'} O[p',p] T[p,u,l,d,r] conj(T[p',...]).
struct DLTask {
    const void* T;   // [d][Du][Dl][Dd][Dr]
    void* E;         // [Du^2][Dl^2][Dd^2][Dr^2]
    const void* O;   // d x d row-major (nullptr: identity)
    int d, Du, Dl, Dd, Dr;
    int hb;          // 1: T and O complex, E real in the Hermitian basis (launch_double_layer_hb)
};

// Two neighbouring column operators of one row fused over their shared horizontal
// leg m (read-out of a horizontal pair):
//   out[(u1 u2)][l1][(d1 d2)][r2] = sum_m A[u1][l1][d1][m] B[u2][m][d2][r2]
// with A, B given as strided 4-leg views (u, l, d, r); out is contiguous.
// Inner product (step aux 0): *out = 2^(*ea + *eb) sum_x A[x] B[x] over n scalars of the
// program's scalar type, no conjugation (a null exponent pointer reads as 0).
// Power-of-two normalisation (step aux 1): A (n scalars) is multiplied in place by 2^-e,
// 2^(e-1) <= max |component| < 2^e (e = 0 for a zero or non-finite buffer), and the int
// *out becomes e + *ea.  B and eb are unused.
struct DotTask {
    const void* A;
    const void* B;
    void* out;
    long long n;
    const int* ea;
    const int* eb;
};

struct FuseTask {
    const void* A;
    const void* B;
    void* out;
    int u1, l1, d1, m, u2, d2, r2;
    int pad;
    long long a_u, a_l, a_d, a_r;
    long long b_u, b_l, b_d, b_r;
};

// Initial state of one message (App. A: messages start from a chosen state): bond-1 sites,
// each a K-vector written at element [0][k][0] of its slot (k * kstride from dst), the slots
// zero beforehand.  mode 0: the product of delta_{ket,bra} (the all-ones product on a
// single-layer network); mode 1: a random positive MPDO G G^T per site, G with normal entries
// (Box-Muller on the counter-based uniforms; positive uniform entries on a single-layer
// network).  The first site is divided by the product of the site norms (unit 2-norm).
struct MsgInitTask {
    double* dst[16];
    long long kstride[16];
    int nsites, K, D, mode;
    int single;             // single-layer network
    int hb;                 // Hermitian-basis coordinates
    int cw;                 // doubles per scalar (2: complex storage, imaginary part left 0)
    int pad;
    unsigned long long seed, stream;  // generator key and the stream of site 0 (site s: stream + s)
};

// One read-out ratio (App. A read-out): <O> = (sum_k c_k N_k) / N_I, N_k and N_I closed
// networks (results of the read-out's closings, complex if the lattice is), c_k the complex
// coefficients of the operator's parts (O = H + i A in the Hermitian basis).
struct RatioTask {
    int nparts;     // 1..4
    int part[4];    // closing index of each part
    int denom;      // closing index of N_I
    int pad[2];
    double c_re[4], c_im[4];
};

// Launchers (kernels.cu).  cplx selects double2 (complex) over double.
// mode bit 0: 16x16 output tiles, one output per thread (steps whose outputs have a
// dimension of at most 16); max_tiles counts tiles of the chosen size.  mode | GC_F32: FP64
// operands and results, FP32 arithmetic.
constexpr int GC_F32 = 1 << 8;
// mode | GC_LAYER: layered pair contractions (GTask::layer_d > 0); max_tiles counts CTAs of
// LAYER_APT_F32 (with GC_F32) or LAYER_APT_F64 pairs, smem_bytes is the largest dynamic shared
// memory of the step's tasks (layer_smem_bytes).
constexpr int GC_LAYER = 1 << 9;
constexpr int LAYER_APT_F32 = 8, LAYER_APT_F64 = 4;   // pairs (consecutive m2) per CTA
constexpr size_t LAYER_SMEM_MAX = 160 * 1024;
size_t layer_smem_bytes(int d, int UL, int DR, bool f32);
cudaError_t layer_prepare();  // sets the dynamic shared memory limit of the layered kernels once
cudaError_t launch_gcontract(const GTask* d_tasks, int ntasks, int max_tiles, bool cplx, cudaStream_t s, int mode,
                             long long smem_bytes = 0);
cudaError_t qr_prepare(int max_m, bool cplx);  // sets the dynamic shared memory limit once
// max_mn: largest m*n of the launch; small problems keep their matrices in shared memory.
// cluster (low byte) > 0: spread each task over that many CTAs (if its matrices fit; else the
// smallest larger C that fits); 0: the built-in rule.  The result does not depend on it.
// cluster | QR_F32: every task has in_float == 2 and is factored in FP32 arithmetic.
constexpr int QR_F32 = 1 << 8;
cudaError_t launch_qr(const QRTask* d_tasks, int ntasks, int max_m, long long max_mn, bool cplx, cudaStream_t s,
                      int cluster = 0);
// whether one QR of the given maximal shape fits a cluster of C CTAs
bool qr_cluster_fits(int max_m, long long max_mn, bool cplx, int C);
// sweep_ctr != nullptr: the current sweep index is OR-ed into bits 36.. of each stream.
cudaError_t launch_rand(const RandTask* d_tasks, int ntasks, unsigned long long seed, const int* sweep_ctr,
                        bool cplx, cudaStream_t s);
cudaError_t launch_set_int(int* p, int n, int v, cudaStream_t s);
cudaError_t launch_add_int(int* p, int v, cudaStream_t s);
cudaError_t launch_check(const CheckTask* d_tasks, int ntasks, double tol, LoopDesc* loop, cudaStream_t s);
cudaError_t launch_scale(const ScaleTask* d_tasks, int ntasks, bool cplx, int* status, cudaStream_t s);
cudaError_t launch_assemble(const AssembleTask* d_tasks, int ntasks, bool cplx, cudaStream_t s);
cudaError_t launch_normalise(const NormTask* d_tasks, int ntasks, bool cplx, cudaStream_t s);
cudaError_t launch_dot(const DotTask* d_tasks, int ntasks, bool cplx, cudaStream_t s, int normalise);
cudaError_t launch_mean(const double* in, int n, double* out, cudaStream_t s);
cudaError_t launch_double_layer(const DLTask* d_tasks, int ntasks, long long max_out, bool cplx, cudaStream_t s);
// complex T and O (Hermitian), real E in the Hermitian basis of every merged leg
cudaError_t launch_double_layer_hb(const DLTask* d_tasks, int ntasks, long long max_out, cudaStream_t s);
cudaError_t launch_convert(const void* in, int in_dtype, void* out, long long n, bool cplx_out, cudaStream_t s);
cudaError_t launch_copy(const void* in, void* out, long long bytes, cudaStream_t s);
cudaError_t launch_fuse(const FuseTask* d_tasks, int ntasks, long long max_out, bool cplx, cudaStream_t s);
cudaError_t launch_relayout(const RelayoutTask* d_tasks, int ntasks, long long max_elems, cudaStream_t s);
cudaError_t launch_msg_init(const MsgInitTask* d_tasks, int ntasks, cudaStream_t s);
// out[2t], out[2t+1] = Re, Im of task t's ratio; *status = 1 where a denominator vanishes
cudaError_t launch_ratio(const RatioTask* d_tasks, int ntasks, const void* closings, bool cplx, double* out,
                         int* status, cudaStream_t s);

// Self-test of the QR's refined scalars: for x[i] in [2^-100, 2^100], the refined 1/sqrt(x)
// and 1/x that the cluster QR uses, and CUDA's 1.0 / sqrt(x) and 1.0 / x (device buffers).
cudaError_t launch_scalar_selftest(const double* x, long long n, double* rsqrt_ours, double* rcp_ours,
                                   double* rsqrt_cuda, double* rcp_cuda, cudaStream_t s);

// Host-side SplitMix64 (same definition as the device one) for host-drawn values.
uint64_t splitmix64(uint64_t z);
double uniform_pm1(uint64_t seed, uint64_t stream, uint64_t idx);

}  // namespace bbp
