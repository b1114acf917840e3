// Program: a recorded list of grouped launches with their task arrays; one
// program is one message sweep (or one read-out), replayed as a CUDA graph.
#pragma once

#include <string>
#include <vector>

#include "bbp_internal.h"
#include "plan.h"

namespace bbp {

extern thread_local std::string g_err;
int fail(int code, const std::string& msg);
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

struct Program {
    bool cplx = false;
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
    GTask* d_gc = nullptr;
    QRTask* d_qr = nullptr;
    RandTask* d_rnd = nullptr;
    CheckTask* d_chk = nullptr;
    ScaleTask* d_scl = nullptr;
    AssembleTask* d_asm = nullptr;
    NormTask* d_nrm = nullptr;
    FuseTask* d_fus = nullptr;
    DLTask* d_dl = nullptr;
    long long dl_max_out = 1;
    int* status = nullptr;  // device error word (relocated separately)
    double fit_tol = 0.0;
    int max_qr_m = 0;
    size_t arena_used = 256;  // offset 0 stays unused so that 0 means "no buffer"
    double static_flops = 0, gated_flops = 0, static_qr_flops = 0, gated_qr_flops = 0;
    cudaGraphExec_t exec = nullptr;

    std::vector<std::pair<size_t, size_t>> allocs;  // (byte offset, bytes) of every arena buffer
    const Program* parent = nullptr;                // lattice program whose arena lies below `split`
    size_t split = (size_t)-1;

    size_t arena_alloc(size_t bytes);
    // Check, before any launch, that every operand range of every task lies inside one
    // arena buffer.  Returns an empty string or a description of the first violation.
    std::string validate() const;
    void gc_step(std::vector<GTask>& ts);
    void qr_step(std::vector<QRTask>& ts);
    void simple(int kind, void* p0, void* p1, long long n, int aux);
    void relocate(char* base, size_t split = (size_t)-1, char* base2 = nullptr);
    cudaError_t upload_tasks();
    cudaError_t launch_all(cudaStream_t st, const int* sweep_ctr, unsigned long long seed) const;
    void free_all();
    long long kernel_count() const;
};

void emit_fits(Program& pr, int ss, std::vector<FitSpec*>& fits, int max_sweeps, double fit_tol,
               const int* unused, bool rand_uses_sweep);
void emit_overlaps(Program& pr, int ss, std::vector<OverlapSpec>& ov);

}  // namespace bbp
