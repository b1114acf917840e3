// The lattice handle behind bbp_lattice*: geometry, arena layout, the planned
// sweep program and the message store.
#pragma once

#include <array>
#include <vector>

#include "bbp.h"
#include "engine.h"

namespace bbp {

enum { DIR_LEFT = 0, DIR_RIGHT = 1, DIR_UP = 2, DIR_DOWN = 3 };
inline int opposite(int d) { return d ^ 1; }

// One outgoing block message = one item of the sweep.
struct Item {
    int block = 0, dir = 0, msgid = 0;
    int H = 0, W = 0, n = 0, b = 0;  // frame rows/cols, column-MPS length H+2, message sites
    std::vector<int> mb;             // message bonds (b+1)
    std::vector<size_t> site_off;    // element offsets of the message sites inside a region
    size_t region_off = 0;           // element offset of this item's slot inside the message region
    size_t region_elems = 0;
    std::vector<FitSpec> fits;       // one per frame column
};

struct FrameMsgs {
    std::vector<View3> T, R, B;  // frame top (W sites), right (H sites), bottom (W sites)
};

// One bMPS column sweep over a region in a rotated frame (App. A): its fits, one per
// frame column, are planned by plan_column_sweeps.
struct ColumnSweep {
    int dir = 0, r0 = 0, c0 = 0, bh = 0, bw = 0;  // frame direction, region origin and size
    FrameMsgs fm;
    int chi = 1;
    bool keep = false;  // keep every column's fitted MPS (read-out) instead of two buffers
    uint64_t tag = 0, outer = 0, msg = 0;  // generator stream fields
    int H = 0, W = 0;
    std::vector<FitSpec> fits;
    // Warm start from another column sweep's fits of the same shapes (the read-out's environment
    // columns of a block from the sweep's fits of that block's message in the same frame): each
    // column's fit starts from a copy of that sweep's fitted MPS once the sweep counter is > 0.
    const std::vector<FitSpec>* warm_from = nullptr;
};

// Words read back after every sweep (pinned host memory).
struct PinnedWords {
    double residual;
    int status;
    int tc_err;
};

}  // namespace bbp

struct bbp_lattice;
namespace bbp {
std::vector<View4> column_mpo(const bbp_lattice* L, int dir, int r0, int c0, int bh, int bw, const FrameMsgs& fm, int c);
int plan_column_sweeps(bbp_lattice* L, Program& pr, std::vector<ColumnSweep>& cs, int max_sweeps, double fit_tol,
                       bool rand_uses_sweep, bool mixed, bool warm = false);
}  // namespace bbp

struct bbp_lattice {
    bbp_lattice_desc desc{};
    bool cplx = false;  // complex arithmetic (complex tensors on the FP64 path)
    bool hb = false;    // complex tensors in the Hermitian basis: real arithmetic, complex T
    int ss = 8;  // scalar bytes
    int K = 1;          // leg dimension of the network: D^2 (double layer) or D (single layer)
    bool single = false;  // single-layer network: the tensors are used as they are
    int nbx = 1, nby = 1, nblocks = 1;
    // block boundaries: block (R, C) holds rows ys[R] .. ys[R+1]-1 and columns xs[C] .. xs[C+1]-1
    // (OBC: every bx columns from shift_x, every by rows from shift_y; infinite: the one block)
    std::vector<int> xs, ys;
    int ntens = 0;
    std::vector<std::array<int, 4>> tdims;  // Du, Dl, Dd, Dr per distinct tensor
    std::vector<size_t> T_off, E_off;       // element offsets
    size_t T_elems = 0, raw_off = 0, raw_bytes = 0;
    size_t one_off = 0;                     // element offset of the constant 1
    std::vector<bbp::Item> items;
    std::vector<int> item_of;               // block*4+dir -> item index or -1
    size_t msg_cur = 0, msg_new = 0, msg_elems = 0;  // element offsets of the two regions
    bbp::Program sweep;
    bool mixed = false;                     // tensor-core (TF32/BF16) sweep
    bbp::MixCtx cx;
    std::vector<std::array<size_t, 4>> EL_off, ER_off;  // per tensor and frame direction (bytes)
    size_t one_lp = 0;                      // low-precision constant 1 (bytes), A-operand form
    size_t one_lp_b = 0;                    // the same as a B operand (the same buffer: a split operand's
                                            // planes serve either role)
    int* d_tcerr = nullptr;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int* d_sweep = nullptr;
    int* d_status = nullptr;
    double* d_residual = nullptr;
    double* d_resid_terms = nullptr;
    int* d_counters = nullptr;
    int ncounters = 0;
    bbp::PinnedWords* h_pinned = nullptr;
    cudaEvent_t done = nullptr;  // recorded after each sweep's read-back copies
    bool has_tensors = false;
    bool direct_ready = false;  // launch_mode 1: loop descriptors written for direct launches
    // stats
    int sweeps = 0;
    double first_residual = 0, last_residual = 0;
    long long kernels = 0;
    double readout_flops = 0;
    long long readout_kernels = 0;

    int tensor_index(int r, int c) const;
    std::array<int, 4> site_dims(int r, int c) const;
    int neighbour(int blk, int dir) const;
    void block_origin(int blk, int& r0, int& c0) const;
    void block_size(int blk, int& h, int& w) const;
    int block_of(int r, int c) const;  // OBC: the block holding lattice site (r, c)
    bbp::View3 msg_site(int item, int s, bool cur) const;
    std::vector<bbp::View3> incoming(int blk, int dir) const;  // message into blk from side dir
    bbp::View4 frame_E(int dir, int r0, int c0, int bh, int bw, int rf, int cf, int* tensor = nullptr) const;
    bbp::View4 E_view(int t, int dir) const;  // MPO view O[w,p,q,w2] of E_t in the frame of dir
    bbp::FrameMsgs frame_msgs(int dir, const std::vector<bbp::View3> in[4]) const;
};

namespace bbp {
// Asynchronous sweep interface (used by bbp_sweep and the request server).
int sweep_launch(bbp_lattice* L);
bool sweep_ready(bbp_lattice* L);
int sweep_collect(bbp_lattice* L, double* residual, bool* stop);
// Plan a lattice without allocating device memory (arena_bytes set); nullptr on error.
int plan_lattice(const bbp_lattice_desc* desc, bbp_lattice** out);
// Lower bound on the zip-up fit tolerance on the path of precision prec (bbp_prec).
double fit_tol_floor(int prec);
// Resident device bytes of a planned lattice: arena plus sweep task descriptors.
size_t planned_bytes(const bbp_lattice* L);
}  // namespace bbp
