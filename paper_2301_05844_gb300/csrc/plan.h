// Host-side planning structures: views into the device arena, per-fit
// descriptions, and the recorded program (a list of grouped launches).
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "bbp_internal.h"

namespace bbp {

// MPS site [a][k][b] at arena element offset `off` with element strides.
struct View3 {
    size_t off = 0;
    int a = 1, k = 1, b = 1;
    long long sa = 0, sk = 0, sb = 0;
};
// MPO site [w][p][q][w2] (left MPO bond, input phys, output phys, right MPO bond).
struct View4 {
    size_t off = 0;
    int w = 1, p = 1, q = 1, w2 = 1;
    long long sw = 0, sp = 0, sq = 0, sw2 = 0;
};

// Device pointer of an arena byte offset: offsets are recorded during planning and
// relocated after the single arena allocation (offset 0 is never a buffer).
inline void* P(size_t byte_off) { return (void*)(uintptr_t)byte_off; }

inline View3 contiguous3(size_t off, int a, int k, int b) {
    View3 v;
    v.off = off;
    v.a = a;
    v.k = k;
    v.b = b;
    v.sa = (long long)k * b;
    v.sk = b;
    v.sb = 1;
    return v;
}
// Mirror of an MPS site (bonds swapped) for a reversed MPS.
inline View3 reversed3(const View3& s) {
    View3 v = s;
    v.a = s.b;
    v.b = s.a;
    v.sa = s.sb;
    v.sb = s.sa;
    return v;
}

// Low-precision operand buffers of one fit on the tensor-core path (byte offsets).
// Every operand is K-major with its row padded to 16 bytes; no contraction index
// has padding inside it, so the padding is never read.
struct MixBufs {
    std::vector<size_t> XL, XR;      // X as [x2][p][pad x] and [x][p][pad x2]
    std::vector<size_t> OL, OR;      // MPO as [q][w2][pad(w p)] and [w][q][pad(p w2)]
    std::vector<size_t> YS, YT;      // Y as [y][pad(q y2)] and [y2][pad(y q)]
    std::vector<size_t> AR, AK, BR, BK;  // envs as [y][w][pad x] (R) and [y][pad(w x)] (K)
    size_t T1 = 0, T2a = 0, T2b = 0, Ytf = 0;
};

// One zip-up fit Y ~ O X (App. A) inside a lockstep group.
struct FitSpec {
    std::vector<View3> X;     // n input sites
    std::vector<View4> O;     // n MPO sites
    std::vector<int> ybond;   // n+1 output bonds
    std::vector<size_t> Y;    // n output slabs (contiguous [a][q][b])
    std::vector<size_t> Aenv, Benv;  // n+1 env slabs (contiguous [y][w][x]); [0] / [n] are the constant 1
    size_t T1 = 0, T2 = 0, Yt = 0, qrw = 0;  // per-item scratch (element offsets)
    size_t losses = 0, active = 0, counter = 0;  // byte offsets: doubles, int flag, int counter
    uint64_t stream = 0;      // generator stream of site 0 (site i adds i)
    bool mixed = false;
    bool warm = false;        // start from Y as it is once the sweep counter is > 0
    MixBufs mx;
    int n() const { return (int)X.size(); }
};

enum StepKind {
    ST_GC = 0, ST_QR, ST_RAND, ST_SETACT, ST_CHECK, ST_SCALE, ST_ASM, ST_NORM, ST_MEAN, ST_COPY, ST_INC, ST_FUSE, ST_DL,
    ST_TC, ST_REL, ST_DOT,
    ST_LOOP_BEGIN,  // p0: LoopDesc; aux: max iterations; the body runs until the matching ST_LOOP_END
    ST_LOOP_END
};

struct Step {
    int kind;
    size_t first = 0;   // index of first task in the per-kind task array
    int count = 0;
    int aux = 0;        // GC: max tiles; QR: max m; TC: tile N
    int aux2 = 0;       // TC: 0 TF32, 1 BF16 | ring depth << 8 | k-blocks per stage << 16 (0: 1);
                        // QR: cluster size (0: rule); GC: 16x16 tiles
    // direct-argument steps
    void* p0 = nullptr;
    void* p1 = nullptr;
    long long n = 0;
};

}  // namespace bbp
