/*
 * bbp.h -- C ABI of the GB300 block belief propagation (blockBP) library.
 *
 * Method: Guo, Poletti & Arad, "Block belief propagation algorithm for
 * two-dimensional tensor networks" (arXiv:2301.05844).  The library runs the
 * data-parallel part of blockBP on one GPU: the double-layer build (Fig. 1(a,b)),
 * the synchronous block-message update of Eq. 1 by boundary-MPS contraction with
 * the variational zip-up fit of App. A (Eq. "update", the A/B environment
 * recurrences, QR/LQ truncation), message normalisation and the fixed-point
 * residual (Sec. "The blockBP algorithm", stop rule; App. A, stop rule), and the
 * expectation-value read-out from a block and its converged incoming messages
 * (App. A, chi = 2D^2+10 read-out; Fig. 1(f)).
 *
 * Conventions shared by every call
 *   - PEPS site tensor T[p][u][l][d][r] (physical, up, left, down, right), C order.
 *     With open boundaries the legs on the lattice edge have dimension 1
 *     (Sec. "The blockBP algorithm": an OBC PEPS is a PBC PEPS with bond 1 on the
 *     boundary).  Complex data is interleaved (re, im).
 *   - Sites are numbered row-major, s = r*Lx + c (r = row, c = column).
 *   - All functions return BBP_OK (0), a positive warning, or a negative error
 *     code; on error bbp_last_error() holds a message for the calling thread.
 *     No C++ exception crosses this boundary.
 *   - Calls on one handle are not thread-safe; different handles are independent.
 *   - Device memory is allocated by the library at bbp_create_lattice (one arena
 *     per handle) and released by bbp_destroy; caller buffers are never retained.
 */
#ifndef BBP_H
#define BBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define BBP_OK 0
#define BBP_NOT_CONVERGED 1 /* max_sweeps reached; results are still valid      */
#define BBP_ERR_INVALID (-1) /* bad argument, dimensions or term geometry         */
#define BBP_ERR_OOM (-2)     /* device (or host) allocation failed                */
#define BBP_ERR_CUDA (-3)    /* a CUDA runtime call failed                        */
#define BBP_ERR_TIMEOUT (-4) /* a device wait exceeded its bound                  */
#define BBP_ERR_NUMERIC (-5) /* NaN/Inf or a message of zero norm                 */
#define BBP_ERR_STATE (-6)   /* call out of order (e.g. sweep before set_tensors) */

typedef struct bbp_lattice bbp_lattice; /* opaque; owned by the caller until bbp_destroy */

typedef enum { BBP_OBC = 0, BBP_INFINITE = 1 } bbp_boundary;
/* Element type of the tensors passed to bbp_set_tensors. */
typedef enum { BBP_F64 = 0, BBP_C128 = 1, BBP_F32 = 2, BBP_C64 = 3 } bbp_dtype;
/* Arithmetic of the contractions.  FP64: every step in FP64 on the GPU.  TF32 and
 * BF16: the site-update contractions on tensor cores with FP32 accumulation, while
 * the message normalisation, residual and read-out ratios stay FP64.
 * TF32X3: as TF32, but every operand is split into a TF32 high part and a TF32 low part
 * (the rounding remainder) and each product is A_hi B_hi + A_lo B_hi + A_hi B_lo, all in
 * one FP32 accumulator: FP32-level contraction accuracy at three times the MMA work.
 * BF16X3: the same split with BF16 parts (hi = bf16(x), lo = bf16(x - hi)): operands carry
 * 16 significant bits, at three BF16 MMAs per product (1.5 times the TF32 MMA time).
 * On the four tensor-core paths the QR/LQ truncations and the read-out closings run in FP32
 * arithmetic unless desc->keep_fp64 is set. */
typedef enum {
    BBP_PREC_FP64 = 0,
    BBP_PREC_TF32 = 1,
    BBP_PREC_BF16 = 2,
    BBP_PREC_TF32X3 = 3,
    BBP_PREC_BF16X3 = 4
} bbp_prec;

typedef struct {
    int Lx, Ly;              /* OBC: lattice columns, rows.  INFINITE: unit cell columns, rows */
    int boundary;            /* bbp_boundary */
    int d, D;                /* physical and virtual bond dimension */
    int bx, by;              /* block columns, rows.  OBC: must divide Lx, Ly.
                                INFINITE: multiples of the unit cell (one block, Sec. "The
                                blockBP algorithm": the block messages itself) */
    int chi;                 /* message bond chi_m (Sec. "The blockBP algorithm", default D^2) */
    int chi_exp;             /* read-out bond; <= 0 selects max(chi, 2 K + 10) (App. A: 2 D^2 + 10),
                                K = D^2 (or D for a single-layer network) */
    int dtype;               /* bbp_dtype of the input tensors */
    int prec;                /* bbp_prec */
    double tol;              /* residual tolerance (main text: 1e-5) */
    int max_sweeps;          /* cap on sweeps when running to tolerance (10) */
    int stop_relative;       /* 0: residual < tol (main text); 1: r_l / r_1 < tol (App. A) */
    double fit_tol;          /* zip-up fit: std/|mean| of -||Yt||^2 over a sweep (App. A: 1e-6);
                                on the TF32 / BF16 / split (TF32X3, BF16X3) paths at least
                                3e-3 / 3e-2 / 3e-5, the noise of a loss computed with FP32
                                accumulation of contractions in that precision (FP64: as given) */
    int fit_max_sweeps;      /* zip-up fit sweep cap (App. A: 10) */
    unsigned long long seed; /* counter-based generator key (fit initial states, init_mode 1) */
    int init_mode;           /* 0: identity-product messages; 1: random MPDO (App. A) */
    int warm_start;          /* 0: every zip-up fit starts from a random state (App. A);
                                1: from the second sweep on, each fit starts from its own
                                result of the previous sweep; 2: as 1, and when chi_exp = chi
                                the read-out's environment columns of a one-block region (the
                                fits the sweep runs for that block's left and right messages)
                                start from the sweep's last fits in the same frame */
    int hermitian_basis;     /* complex tensors only.  0: complex arithmetic on the FP64 path;
                                1: Hermitian basis on the FP64 path too.  The TF32 / BF16
                                paths always use it.  In the Hermitian basis every merged
                                ket/bra leg of the double layer (Fig. 1(b)) is rotated by a
                                fixed unitary V: a vector v indexed by (ket a, bra b) gets
                                the coordinate v_(a,a) at k = a*D + a, (v_(a,b) + v_(b,a)) / sqrt 2
                                at k = a*D + b for a < b and (v_(b,a) - v_(a,b)) / (i sqrt 2)
                                at k = a*D + b for a > b, on up and left legs; down and right
                                legs take conj(V) (the a > b coordinate changes sign), so
                                that every bond contracts through V^T conj(V) = I.  The
                                double layer of a Hermitian operator and the (Hermitian)
                                messages are real there, so sweeps and read-out run in real
                                arithmetic at a quarter of the complex flops; V is unitary,
                                so overlaps, residuals and <O> are unchanged.
                                bbp_get_message and bbp_set_message then use real messages
                                in the basis of the legs they carry: V for messages sent
                                left or up, conj(V) for messages sent right or down. */
    void* stream;            /* cudaStream_t for all work; NULL = library-owned stream */
    int single_layer;        /* 0: the tensors are PEPS tensors, contracted as the double layer
                                (Fig. 1(a,b)).  1: they are the network's own site tensors
                                E[u][l][d][r] (a 2D classical model's partition function, Sec.
                                on the 2D Ising model), used as they are with bond K = D on
                                every leg: d must be 1 and dtype real.  The initial messages
                                are then the all-ones product (init_mode 0) or positive uniform
                                entries (init_mode 1), the phase reference of the normalisation
                                is <1|m> (all-ones vector) instead of <I|m>, and a term's
                                op_re[k] is the impurity tensor that replaces E at site[k]. */
    int shift_x, shift_y;    /* the partition shifted by shift_x columns and shift_y rows (the
                                paper covers every bond from a block centre by such shifted
                                partitions, Sec. "The blockBP algorithm").  INFINITE:
                                0 <= shift < Lx (Ly), block site (r, c) is lattice site
                                (r + shift_y, c + shift_x).  OBC: 0 <= shift < bx (by), block
                                boundaries at columns shift_x, shift_x + bx, ... and rows
                                shift_y, shift_y + by, ..., so the blocks on the lattice edges
                                are narrower (the periodic embedding's blocks that straddle its
                                seam, which split into two pieces joined only by bonds of
                                dimension 1); the block index stays row-major over the blocks */
    int launch_mode;         /* 0: each sweep is one CUDA graph whose fit loops are conditional
                                nodes that stop when the fits have met the stop rule; 1: the
                                same kernels launched one by one on the stream, each fit loop
                                run to fit_max_sweeps with the converged fits skipped (same
                                results; lets a kernel profiler see every launch) */
    int keep_fp64;           /* TF32 / BF16 / TF32X3 / BF16X3 paths: 0 runs the stages outside
                                the tensor cores in FP32 arithmetic: the QR/LQ truncations
                                (their input is already an FP32 contraction result; Q is
                                still stored in FP64 and the fit loss summed in FP64) and the
                                read-out closings (FP64 operands rounded to FP32, FP32
                                accumulation compensated by TwoSum over the environment bonds,
                                plain FP32 sums of at most d D^2 terms in the layered site
                                rows of real lattices, FP64 results, every environment of a
                                strip rescaled by a power of two so that nothing overflows);
                                1 keeps
                                FP64 arithmetic there.  The FP64 path always uses FP64. */
} bbp_lattice_desc;

/* Validate desc, allocate the device arena (double layer, message store, work
 * buffers) and plan one sweep.  *out receives the handle.  Limits checked here:
 * Lx, Ly <= 4096; bx, by <= 16; D <= 16; d <= 64; 1 <= fit_max_sweeps <= 64;
 * init_mode, hermitian_basis, single_layer, launch_mode and keep_fp64 0 or 1; warm_start 0..2; 0 <= shift_x < Lx and
 * 0 <= shift_y < Ly on infinite lattices, 0 <= shift_x < bx and 0 <= shift_y < by with OBC.
 * Errors: INVALID, OOM, CUDA. */
int bbp_create_lattice(const bbp_lattice_desc* desc, bbp_lattice** out);

/* Device bytes a lattice with this desc would hold (arena plus task descriptors),
 * from the same planning as bbp_create_lattice, without allocating.  Used for
 * admission by footprint.  Errors: INVALID. */
int bbp_lattice_footprint(const bbp_lattice_desc* desc, size_t* bytes);

/* Upload every site tensor and build the double-layer network (Fig. 1(a,b)); on a
 * single-layer network (desc->single_layer) the tensors are its site tensors E[u][l][d][r].
 * data: OBC -> Lx*Ly tensors in row-major site order; INFINITE -> Lx*Ly unit-cell
 * tensors.  Each tensor T[p][u][l][d][r] in C order with the OBC edge legs of
 * dimension 1, element type desc->dtype, concatenated without padding.
 * on_device != 0: data is a device pointer (read on the handle's stream).
 * The library copies; the caller keeps ownership.  Resets the messages to their
 * initial state.  Errors: INVALID (NULL data), CUDA. */
int bbp_set_tensors(bbp_lattice* lat, const void* data, int on_device);

/* Synchronous message sweeps, Eq. 1: every block message of sweep l+1 is computed
 * from the messages of sweep l.  n_sweeps > 0 runs exactly that many; n_sweeps <= 0
 * runs until the residual meets desc->tol (absolute or relative) or max_sweeps.
 * residual_out (may be NULL): last residual, the mean over messages of
 * ||m^l - m^{l-1}||^2 of the unit-norm, phase-fixed messages.  sweeps_done (may be
 * NULL): sweeps run by this call.  Returns OK, NOT_CONVERGED, STATE (no tensors),
 * NUMERIC, TIMEOUT or CUDA. */
int bbp_sweep(bbp_lattice* lat, int n_sweeps, double* residual_out, int* sweeps_done);

/* One expectation-value term: a product of nsite (1 or 2) single-site d x d
 * operators, row-major, real and imaginary parts (op_im may be NULL).  On a
 * single-layer network op_re[k] (and op_im[k], if not NULL) hold instead the impurity
 * tensor that replaces the site tensor at site[k]: its shape (Du, Dl, Dd, Dr) with the
 * OBC edge legs of dimension 1, C order; <O> is then the ratio of the network with the
 * impurities to the network without them.
 * OBC sites are lattice sites; INFINITE sites index the bx x by block (row-major). */
typedef struct {
    int nsite;
    int site[2];
    const double* op_re[2];
    const double* op_im[2];
} bbp_term;

/* <O> = N_O / N_I for each term, read from its block and the block's converged
 * incoming messages with bond chi_exp (App. A; Fig. 1(f)).  Two sites must lie in
 * one block, or be nearest neighbours in adjacent blocks (then read from the merged
 * two-block region whose outer messages are joined by a bond of dimension 1), and
 * span at most two adjacent columns of their region.  out_re/out_im: n_terms
 * doubles each (host memory; out_im may be NULL).  Errors: INVALID, STATE, CUDA. */
int bbp_expect(bbp_lattice* lat, const bbp_term* terms, int n_terms, double* out_re, double* out_im);

/* Read-out over several partitions of one OBC lattice (the same tensors run with different
 * desc.shift_x / shift_y): blockBP's observables are accurate near a block's centre, and the
 * paper covers every bond from a block centre by shifted partitions (Sec. "The blockBP
 * algorithm").  Each term is read (bbp_expect) from the lattice in which its sites lie deepest
 * inside one block: the smallest distance of its sites to that block's edges, a pair split
 * between two blocks counting -1, the first lattice on a tie.  chosen (n_terms ints, may be
 * NULL) receives that lattice's index per term.  Errors: INVALID (no lattice, a NULL one,
 * lattices of different Lx, Ly or d, an infinite one, a bad term), and bbp_expect's. */
int bbp_expect_centred(bbp_lattice* const* lats, int n_lats, const bbp_term* terms, int n_terms, double* out_re,
                       double* out_im, int* chosen);

/* Reduced density matrix of nsite (1 or 2) sites, rho = Tr_rest |psi><psi| / <psi|psi>/* Reduced density matrix of nsite (1 or 2) sites, rho = Tr_rest |psi><psi| / <psi|psi>
 * (the 2-local RDMs that the paper compares between methods by their trace distance
 * D(rho, sigma) = ||rho - sigma||_1 / 2, Sec. on the transverse Ising model).  Entry
 * (a, b) = <a|rho|b> is the read-out of the matrix unit |b><a| (a product of single-site
 * units for two sites, site[0] the leading index digit), so Tr(rho O) = <O>; the sites
 * follow bbp_expect's rules.  rho_re / rho_im: d^nsite x d^nsite doubles each, row-major
 * (host memory; rho_im may be NULL).  Errors: INVALID (also for a single-layer network),
 * STATE, NUMERIC, TIMEOUT, CUDA. */
int bbp_rdm(bbp_lattice* lat, int nsite, const int* sites, double* rho_re, double* rho_im);

/* Free the handle and its device arena.  NULL is a no-op. */
void bbp_destroy(bbp_lattice* lat);

/* Message of the last failing call on this thread ("" if none). */
const char* bbp_last_error(void);

/* ---- inspection, checkpoint / resume ------------------------------------------- */

/* Outgoing message of block `block` (row-major block index) toward direction dir
 * (0 left, 1 right, 2 up, 3 down).  nsites/bonds (may be NULL) receive the site
 * count and the nsites+1 bond dimensions; the message has physical dimension D^2 (D on a
 * single-layer network).
 * If out != NULL the sites are written in order, each [a][k][b] in C order, as
 * doubles (complex interleaved).  Errors: INVALID (no such message), STATE. */
int bbp_get_message(bbp_lattice* lat, int block, int dir, int* nsites, int* bonds, double* out);

/* Replace that message (same layout as bbp_get_message); for checkpoint / resume. */
int bbp_set_message(bbp_lattice* lat, int block, int dir, const double* in);

/* ---- standalone truncation step ------------------------------------------------- */

/* Batched thin QR with diag(R) real and non-negative: the truncation step of the
 * zip-up fit (App. A: QR on the left-to-right half sweep, keep Q).  For b < batch the
 * m x n matrix A_b (row-major, FP64, or interleaved complex FP64 if complex_values)
 * gives Q_b (m x n, orthonormal columns), matrices packed back to back.  A, Q and
 * loss are device pointers; loss (may be NULL) receives -||A_b||^2, the fit loss of
 * App. A.  Requires 1 <= n <= m and n <= 512.  stream: cudaStream_t (NULL: legacy
 * stream); the call returns after the stream has finished the work.  Allocates a
 * workspace of 2*m*n scalars per matrix for the duration of the call.
 * Errors: INVALID, OOM, CUDA. */
int bbp_qr_batched(int batch, int m, int n, int complex_values, const double* A, double* Q, double* loss,
                   void* stream);

/* The same batched QR for callers that cannot allocate device memory while they
 * run: programs that reserve the whole GPU up front under their own memory manager,
 * or that must not risk an allocation failure (or the implicit synchronisation of an
 * allocation) in the middle of their work.  The paper has no counterpart: this is a
 * deployment variant of bbp_qr_batched.
 *   - Allocates nothing: no cudaMalloc / cudaFree / allocating library call.  The
 *     workspace is a fixed device array of BBP_QR_NOALLOC_SCRATCH_BYTES (16 MiB),
 *     held by every GPU that loads the library until the process exits.
 *   - A request needs round_up(batch * 144, 256) bytes of task descriptors plus
 *     batch * 2*m*n scalars (8 bytes real, 16 complex) of that array; larger requests
 *     fail with BBP_ERR_INVALID.
 *   - The first call on a device resolves the array's device address
 *     (cudaGetSymbolAddress; with CUDA's lazy module loading this is also when the
 *     library's module is loaded on that device and the 16 MiB are committed) and sets
 *     the QR kernels' shared-memory limits for real and complex matrices of up to 512
 *     rows (cudaFuncSetAttribute).  Make that first call at start-up, before the caller
 *     reserves the rest of the GPU and before any stream capture; if the array cannot
 *     be committed it returns BBP_ERR_OOM.  First calls from several host threads are
 *     serialised.  Later calls with m > 512 raise the limit again.
 *   - Asynchronous: returns once the work is queued on `stream`.  All calls share the
 *     array, so calls whose work overlaps on the GPU (different streams, or different
 *     host threads) race on it; serialise them.  Nothing in the array needs to start
 *     at zero: every call writes all of the workspace it reads.
 * Same arguments, layout and results as bbp_qr_batched.  Errors: INVALID, OOM, CUDA. */
#define BBP_QR_NOALLOC_SCRATCH_BYTES (16u << 20)
int bbp_qr_batched_noalloc(int batch, int m, int n, int complex_values, const double* A, double* Q, double* loss,
                           void* stream);

typedef struct {
    double flops;            /* algorithmic flops executed: the K2-K5 contractions of every site
                                update (App. A, Eq. "update" and the A/B recurrences) at their
                                actual bonds, plus the read-out's contractions */
    double qr_flops;         /* FP64 QR/LQ flops executed (4mn^2 - 4n^3/3 per m x n matrix) */
    long long kernels;       /* kernel launches issued by the library */
    long long fit_sweeps;    /* zip-up fit sweeps executed, summed over the fit loops */
    long long fits;          /* zip-up fit loops executed (one per column stage of a message
                                sweep, the fits of all messages in lockstep) */
    int sweeps;              /* message sweeps executed since set_tensors */
    double last_residual;
    double first_residual;
    long long fit_loop_iters; /* fit sweeps the lockstep fit loops ran: each loop runs until every
                                fit of its group has met the stop rule (or the cap), the fits
                                that have met it skipping their work */
} bbp_stats;

/* Counters since bbp_set_tensors (flops are counted on the host from the planned
 * shapes, each fit's work times the fit sweeps it ran; fit sweeps and loop iterations
 * are read back from the device). */
int bbp_get_stats(bbp_lattice* lat, bbp_stats* out);

/* ---- diagnostics ------------------------------------------------------------------
 * Not a step of the paper's method: a self-test of the library's tensor-core GEMM
 * kernel (the contraction engine of the TF32/BF16 path) on host matrices.
 * C[m][n] = sum_k A[m][k] B[n][k]; A is M x K, B is N x K, C is M x N, all row-major
 * FP32 on the host; prec is BBP_PREC_TF32 or BBP_PREC_BF16 (operands rounded to it).
 * Errors: INVALID, CUDA, TIMEOUT (a pipeline wait hit its bound). */
int bbp_selftest_gemm(int M, int N, int K, int prec, const float* A, const float* B, float* C);

/* Not a step of the method: the self-test of the bounded pipeline waits (a device wait
 * that must end with a status, never hang).  Launches a small tensor-core GEMM whose
 * operand copies are withheld, so that the first wait on a loaded stage can never succeed:
 * it gives up after its poll bound (well under a second), raises the error word, the CTAs
 * release their tensor memory and return, and the call returns BBP_ERR_TIMEOUT with the
 * context still usable.  Any other result means the bound did not work.  Errors: CUDA. */
int bbp_selftest_gemm_timeout(void);

/* Not a step of the method: the self-test of the FP64 scalars of the cluster QR (Householder
 * step, App. A truncation), whose 1/sqrt(s) and 1/d are FP32 seeds refined by one
 * third-order iteration (Householder's for s^(-1/2), Newton-Raphson's for 1/d).  For the n
 * host values x[i] in [2^-100, 2^100] it writes those refined values and CUDA's own
 * 1.0 / sqrt(x) and 1.0 / x, all computed on the device.  Errors: INVALID (x out of range),
 * OOM, CUDA. */
int bbp_selftest_scalar(long long n, const double* x, double* rsqrt_ours, double* rcp_ours, double* rsqrt_cuda,
                        double* rcp_cuda);

/* Not a step of the method: the self-test of the FP32-arithmetic blocked Householder QR that
 * the tensor-core paths use for the truncation of App. A (Q with diag(R) >= 0).  A holds
 * batch row-major m x n FP32 matrices on the host; Q receives their thin Q factors (FP64,
 * same layout) and loss (may be NULL) -||A_b||^2.  Every task's 2 m n workspace is followed by
 * guard words; *workspace_intact is 1 if the QR left them unchanged.  Errors: INVALID, OOM,
 * CUDA. */
int bbp_selftest_qr_fp32(int batch, int m, int n, const float* A, double* Q, double* loss, int* workspace_intact);

/* Not a step of the method: the self-test of the layered pair contraction that the read-out
 * uses on the site rows of real double-layer lattices (App. A read-out closings, contracted
 * with the ket and bra tensors in turn instead of E = sum_p Tk_p (x) Tb_p):
 *   Y[m1][m2][(n1 n1')][(n2 n2')] = sum_p sum_{k1 k2 k1' k2'} Tk[p][k1][k2][n1][n2]
 *                                   X[(k1 k1')][m1][(k2 k2')][m2] Tb[p][k1'][k2'][n1'][n2'],
 * merged indices ket-major (k1 K1 + k1').  All arrays on the host, FP64, C order; f32 != 0
 * runs the FP32-arithmetic instance (tensor-core lattices).  Requires K1 K2 <= 32 and
 * N1 N2 <= 32 (and the shared memory that d and these imply).  Errors: INVALID, OOM, CUDA. */
int bbp_selftest_layer(int f32, int d, int K1, int K2, int N1, int N2, int M1, int M2, const double* X,
                       const double* Tk, const double* Tb, double* Y);

/* Kernel-class timing of one planned sweep, for roofline measurements: replays, on
 * the handle's stream and bracketed by CUDA events, only the launches of one class
 * (0: tensor-core GEMM steps, 1: FP64 strided contractions, 2: FP64 QR/LQ),
 * reps times.  The replay writes only work buffers, never
 * the message store, so the next bbp_sweep is unaffected.  Outputs (may be NULL):
 * total device milliseconds, launches, algorithmic flops of those launches (real
 * multiply-adds counted as 2; complex x4), and the bytes the launches must move at
 * least (operands read once, results written once).  Errors: INVALID, STATE, CUDA. */
int bbp_time_kernels(bbp_lattice* lat, int kernel_class, int reps, double* ms, long long* launches,
                     double* flops, double* bytes);

/* One row of bbp_time_steps: a launch of the planned sweep, in program order. */
typedef struct {
    int index;               /* step index in the sweep program */
    int kernel_class;        /* 0 tensor-core GEMM, 1 FP64 strided contraction, 2 QR/LQ */
    int tasks;               /* task descriptors (independent problems) in the launch */
    int tile_n;              /* tensor-core steps: tile width BN; otherwise 0 */
    long long max_m, max_n, max_k;  /* largest task dimensions (QR: m, n; K 0) */
    double flops, bytes;     /* algorithmic work of the launch, as bbp_time_kernels counts it */
    double ms;               /* device milliseconds per launch */
} bbp_step_time;

/* Per-launch timing of one planned sweep: every launch of classes 0-2 replayed on its own
 * (reps times after one warm-up, CUDA events on the handle's stream, every fit stage active;
 * a fit loop's body appears once), in program order.  Writes min(cap, launches) rows to out
 * (may be NULL with cap 0) and the number of such launches to *n_steps.  Like
 * bbp_time_kernels it writes only work buffers.  Errors: INVALID, STATE, CUDA, TIMEOUT. */
int bbp_time_steps(bbp_lattice* lat, int reps, int cap, bbp_step_time* out, int* n_steps);

/* Launch-shape autotuner (the batching pattern's tiles chosen per workload rather than by a
 * fixed rule).  Must run after bbp_set_tensors and before the first bbp_sweep.  It times,
 * with CUDA events on the handle's stream and every fit stage active, reps launches of each
 * candidate after one warm-up, and keeps the fastest:
 *  - tensor-core steps (TF32 / BF16 paths): tile width BN in {32, 64, 128, 256} (up to the
 *    widest result), TMA ring stages of one or two k-blocks and ring depth in {2, 3, 4, 6, 8}
 *    (up to what the K extent needs and shared memory holds); the K-accumulation order of a
 *    tile is the same for every candidate;
 *  - QR/LQ steps (every path): the number of CTAs (1-8) one matrix is spread over, kept
 *    only if clearly faster than the built-in rule; every column's arithmetic, and the fit
 *    loss, are the same for every cluster size.
 * Results therefore do not change.  The replays write only work buffers (the fits start from
 * fresh draws at the first sweep).  Outputs (may be NULL): summed per-launch milliseconds of
 * the tuned steps with the default and with the chosen shapes, and how many steps changed.
 * Errors: INVALID, STATE (no tensors, or sweeps already run), TIMEOUT, CUDA. */
int bbp_autotune(bbp_lattice* lat, int reps, double* ms_before, double* ms_after, int* steps_changed);

/* The library's counter-based generator (the one that draws the initial fit states
 * and the random initial messages, App. A), evaluated on the host: out[i] for
 * i < n, each an exact double in [-1, 1).  Runs without a GPU. */
int bbp_selftest_rng(unsigned long long seed, unsigned long long stream, long long n, double* out);

/* ---- Request server: continuous batching of whole solves (Sec. III workflow) ----
 * A solve is one lattice run to convergence under its desc (tol, stop_relative,
 * max_sweeps), then read out.  A worker thread owned by the server admits queued
 * solves in submission order whenever their resident footprint (bbp_lattice_footprint)
 * fits in max_bytes and fewer than max_active are running; a solve that does not fit
 * yet does not hold back smaller ones queued after it.  Every running solve has its
 * own stream and keeps one sweep in flight, so sweeps of different solves overlap on
 * the device; a finished solve is read out with bbp_expect and its memory released at
 * once.  The transient read-out buffers are not part of the footprint.  Results of a
 * solve are the same as those of bbp_create_lattice / bbp_set_tensors / bbp_sweep /
 * bbp_expect on its own (desc->stream is ignored). */
typedef struct bbp_server bbp_server; /* opaque; owned by the caller until bbp_server_destroy */

/* Start a server on the current device.  Errors: INVALID (max_bytes 0, max_active < 1). */
int bbp_server_create(size_t max_bytes, int max_active, bbp_server** out);

/* Queue one solve.  tensors: host memory laid out as for bbp_set_tensors; terms as for
 * bbp_expect (n_terms may be 0).  Both are copied before the call returns.  *id
 * receives the request id.  Errors: INVALID (bad desc or term), OOM (footprint above
 * max_bytes: the request could never be admitted). */
int bbp_server_submit(bbp_server* srv, const bbp_lattice_desc* desc, const void* tensors, const bbp_term* terms,
                      int n_terms, long long* id);

/* Non-blocking status of request id.  *state: 0 queued, 1 running, 2 done, or the
 * negative error code the solve failed with (bbp_last_error then holds its message).
 * When done, out_re/out_im (n_terms each, may be NULL) receive the expectation values.
 * sweeps / residual: sweeps run so far and the last residual; latency_s: seconds from
 * submission to completion (0 while not finished).  Any output may be NULL.
 * Errors: INVALID (unknown id). */
int bbp_server_poll(bbp_server* srv, long long id, int* state, double* out_re, double* out_im, int* sweeps,
                    double* residual, double* latency_s);

/* Block until request id has finished or timeout_s has passed.  Returns OK when done,
 * the solve's error code when it failed, TIMEOUT when still running. */
int bbp_server_wait(bbp_server* srv, long long id, double timeout_s);

/* Requests submitted and done, sweeps run by all solves, and admitted bytes in use. */
int bbp_server_stats(bbp_server* srv, long long* submitted, long long* done, long long* sweeps, size_t* bytes_in_use);

/* Finish the running solves, drop the queued ones (their state becomes STATE) and
 * stop the worker.  Results of finished requests are released with the server. */
void bbp_server_destroy(bbp_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* BBP_H */
