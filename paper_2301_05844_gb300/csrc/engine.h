// Program: a recorded list of grouped launches with their task arrays; one
// program is one message sweep (or one read-out), replayed as a CUDA graph.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "bbp_internal.h"
#include "plan.h"
#include "tc_gemm.h"

namespace bbp {

extern thread_local std::string g_err;
int fail(int code, const std::string& msg);
// Handler of every C entry point (a function-try-block around its body): turns the C++
// exception in flight (a failed host allocation, a thread that could not start) into an
// error code and message, so that no exception crosses the C boundary.
int abi_error() noexcept;
int bond_cap(const std::vector<int>& phys, int i, int chi);
std::vector<int> bond_caps(const std::vector<int>& phys, int chi);
uint64_t stream_id(uint64_t tag, uint64_t outer, uint64_t msg, uint64_t col, uint64_t site);

// <M|N> chain for one pair of MPS with equal physical dims.
struct OverlapSpec {
    std::vector<View3> M, N;  // M is conjugated
    size_t one = 0;           // constant 1 (element offset)
    size_t E[2] = {0, 0};     // ping-pong environment slabs (a x a')
    size_t T = 0;             // scratch (a x k x b')
    size_t result = 0;        // final 1x1 environment = the overlap
};

// Operand geometry of one tensor-core task, kept until the arena exists so that
// the TMA tensor maps can be encoded with real addresses.
struct TCSpec {
    size_t a_off = 0, b_off = 0;          // byte offsets
    long long a_rows = 1, b_rows = 1, K = 1, a_ld = 1, b_ld = 1;
    long long a_pl = 0, b_pl = 0;         // split operands: elements from the hi plane to the lo plane
    int kind = 0, bn = 32;
};

struct Program {
    bool cplx = false;
    int tc_kind = 0;                      // 0 TF32, 1 BF16 (tensor-core path)
    int* tc_err = nullptr;                // device word raised by a timed-out pipeline wait
    std::vector<TCTask> tcs;
    std::vector<TCSpec> tcspec;
    std::vector<RelayoutTask> rel;
    TCTask* d_tcs = nullptr;
    RelayoutTask* d_rel = nullptr;
    std::vector<Step> steps;
    std::vector<GTask> gc;
    std::vector<QRTask> qr;
    std::vector<RandTask> rnd;
    std::vector<CheckTask> chk;
    std::vector<ScaleTask> scl;
    std::vector<AssembleTask> asmb;
    std::vector<NormTask> nrm;
    std::vector<FuseTask> fus;
    std::vector<DLTask> dl;
    std::vector<DotTask> dots;
    GTask* d_gc = nullptr;
    QRTask* d_qr = nullptr;
    RandTask* d_rnd = nullptr;
    CheckTask* d_chk = nullptr;
    ScaleTask* d_scl = nullptr;
    AssembleTask* d_asm = nullptr;
    NormTask* d_nrm = nullptr;
    FuseTask* d_fus = nullptr;
    DLTask* d_dl = nullptr;
    DotTask* d_dot = nullptr;
    long long dl_max_out = 1;
    int* status = nullptr;  // device error word (relocated separately)
    double fit_tol = 0.0;
    int max_qr_m = 0;
    size_t warm_ctr_off = 0;  // byte offset of the lattice's sweep counter (warm-started fits)
    size_t arena_used = 256;  // offset 0 stays unused so that 0 means "no buffer"
    double static_flops = 0, gated_flops = 0, static_qr_flops = 0, gated_qr_flops = 0;
    // flops of one fit sweep of each fit, keyed by its active flag's arena offset (the value the
    // task pointers hold before relocation), and that key for each check task
    std::map<uintptr_t, double> fit_flops, fit_qr_flops;
    std::vector<uintptr_t> chk_keys;
    void count_flops(const int* active, double f, bool qr_step);
    cudaGraphExec_t exec = nullptr;

    std::vector<std::pair<size_t, size_t>> allocs;  // (byte offset, bytes) of every arena buffer
    const Program* parent = nullptr;                // lattice program whose arena lies below `split`
    size_t split = (size_t)-1;

    size_t arena_alloc(size_t bytes);
    // Low-precision operand buffer of `elems` elements of esz bytes; a split operand (hi and lo
    // planes) takes two planes of that size and is recorded in `planes`.
    std::map<size_t, long long> planes;  // byte offset of a split buffer -> elements per plane
    size_t lp_alloc(size_t elems, int esz, bool split);
    long long plane_of(size_t byte_off) const;
    // Check, before any launch, that every operand range of every task lies inside one
    // arena buffer.  Returns an empty string or a description of the first violation.
    std::string validate() const;
    void gc_step(std::vector<GTask>& ts);
    void layer_step(std::vector<GTask>& ts);  // layered pair contractions (GTask::layer_d > 0)
    void qr_step(std::vector<QRTask>& ts);
    // inner products (normalise = false) or power-of-two normalisations (true), see DotTask
    void dot_step(std::vector<DotTask>& ts, bool normalise = false);
    bool gc_f32 = false;  // contraction steps added from now on run in FP32 arithmetic
    void simple(int kind, void* p0, void* p1, long long n, int aux);
    void relocate(char* base, size_t split = (size_t)-1, char* base2 = nullptr);
    void tc_step(std::vector<TCTask>& ts, std::vector<TCSpec>& sp, int kind);
    void rel_step(std::vector<RelayoutTask>& ts);
    // encode every TMA tensor map (after relocate)
    cudaError_t encode_maps(char* base, size_t split = (size_t)-1, char* base2 = nullptr);
    // give tensor-core step si the tile width bn and a TMA ring of `depth` stages of ksub
    // k-blocks: its B maps re-encoded, its tile count updated and its task descriptors
    // re-uploaded on st (after upload_tasks)
    cudaError_t tc_retile(size_t si, int bn, int depth, char* base, size_t split, char* base2, cudaStream_t st,
                          int ksub = 1);
    // task descriptors to the device (stream-ordered allocation on st)
    cudaError_t upload_tasks(cudaStream_t st);
    std::vector<std::pair<size_t, int>> loop_descs;  // (arena byte offset, max iterations)
    std::vector<void*> loop_ptr;                      // relocated LoopDesc addresses
    cudaError_t launch_step(const Step& s, cudaStream_t st, const int* sweep_ctr, unsigned long long seed) const;
    size_t loop_end(size_t begin) const;
    cudaError_t launch_all(cudaStream_t st, const int* sweep_ctr, unsigned long long seed) const;
    // write every LoopDesc (max, and the conditional handle when running as a graph)
    cudaError_t init_loops(cudaStream_t st, bool in_graph, const unsigned long long* handles) const;
    cudaError_t reset_loop_totals(cudaStream_t st) const;
    // capture the program as one graph with a conditional WHILE node per loop
    cudaError_t build_graph(cudaStream_t st, const int* sweep_ctr, unsigned long long seed);
    // set every fit's active flag (so that a replay runs every gated stage)
    cudaError_t reset_active(cudaStream_t st) const;
    // class of a step (0 tensor-core GEMM, 1 FP64 contraction, 2 QR/LQ, 3 other) and its
    // algorithmic work: flops, bytes (operands once, results once), largest task dimensions
    int step_class_of(const Step& s) const;
    void step_work(const Step& s, double* flops, double* bytes, long long* max_m, long long* max_n,
                   long long* max_k) const;
    // launch only the steps of one class (see bbp_time_kernels); returns launches
    cudaError_t launch_class(cudaStream_t st, const int* sweep_ctr, unsigned long long seed, int cls,
                             long long* launches, double* flops, double* bytes) const;
    // release the graph and the task descriptors (stream-ordered on st)
    void free_all(cudaStream_t st);
    long long kernel_count() const;
    // launches and algorithmic flops actually executed over `runs` runs of the program (loop
    // bodies counted by the iterations the device ran; a fit's gated work by the fit sweeps it
    // ran while active), and the iterations all fit loops ran
    cudaError_t executed(long long runs, long long* launches, double* flops, double* qr_flops,
                         long long* loop_iters = nullptr) const;
};

// warm: the random initial state is drawn only while the sweep counter is 0; later
// sweeps start each fit from the Y buffer as the previous sweep left it.
void emit_fits(Program& pr, int ss, std::vector<FitSpec*>& fits, int max_sweeps, double fit_tol, bool warm,
               bool rand_uses_sweep);
void emit_overlaps(Program& pr, int ss, std::vector<OverlapSpec>& ov);

// Tensor-core (TF32 / BF16) variant of emit_fits: same stages and generator streams, with
// every contraction on tcgen05 and the QR/LQ in FP32 (or FP64, MixCtx::qr_f32) arithmetic.
struct MixCtx {
    int ss = 8;      // canonical (FP64) scalar bytes
    int esz = 4;     // low-precision element bytes
    int pe = 4;      // row padding unit in elements (16 bytes)
    int lpk = 4;     // relayout / QR store kind of low-precision operands
    int tck = 0;     // tensor-core kind: 0 TF32, 1 BF16
    int tco = 1;     // tensor-core epilogue kind of low-precision results
    bool x3 = false; // split TF32 operands: every K-major row holds three K-segments
    bool qr_f32 = true;  // QR/LQ truncations in FP32 arithmetic (QRTask::in_float = 2)
};
void emit_fits_mixed(Program& pr, const MixCtx& cx, std::vector<FitSpec*>& fits, int max_sweeps, double fit_tol,
                     bool warm, bool rand_uses_sweep);
long long padded(const MixCtx& cx, long long x);

}  // namespace bbp
