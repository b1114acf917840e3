// Host engine of the blockBP library: geometry of blocks and frames, the lockstep
// planner that turns every message update of a sweep into grouped launches, the
// device arena, CUDA-graph capture of one sweep, and the C ABI of include/bbp.h.
//
// One sweep (Eq. 1) is planned once: every outgoing block message is an "item";
// all items advance together through the columns of their block (App. A: bMPS
// column by column, right to left in the rotated frame), each column being a
// zip-up fit (App. A) whose site updates, QR/LQ steps and environment updates are
// one grouped launch per step across all items.  The whole sweep is captured in a
// CUDA graph and replayed.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <complex>
#include <new>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "bbp.h"
#include "bbp_internal.h"
#include "engine.h"
#include "plan.h"

namespace bbp {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int abi_error() noexcept {
    int code = BBP_ERR_INVALID;
    try {
        try {
            throw;
        } catch (const std::bad_alloc&) {
            code = BBP_ERR_OOM;
            g_err = "host allocation failed";
        } catch (const std::exception& e) {
            g_err = std::string("host error: ") + e.what();
        } catch (...) {
            g_err = "host error";
        }
    } catch (...) {  // the message itself could not be stored
    }
    return code;
}

int bond_cap(const std::vector<int>& phys, int i, int chi) {
    // bond between site i-1 and i of an MPS with physical dims phys
    if (i <= 0 || i >= (int)phys.size()) return 1;
    double left = 1, right = 1;
    for (int j = 0; j < i; ++j) left *= phys[j];
    for (int j = i; j < (int)phys.size(); ++j) right *= phys[j];
    double b = std::min((double)chi, std::min(left, right));
    return (int)b;
}
std::vector<int> bond_caps(const std::vector<int>& phys, int chi) {
    std::vector<int> b(phys.size() + 1);
    for (size_t i = 0; i <= phys.size(); ++i) b[i] = bond_cap(phys, (int)i, chi);
    return b;
}

uint64_t stream_id(uint64_t tag, uint64_t outer, uint64_t msg, uint64_t col, uint64_t site) {
    return (tag << 56) | (outer << 36) | (msg << 16) | (col << 8) | site;
}

// ------------------------------------------------------------------ program recording
size_t Program::arena_alloc(size_t bytes) {
    size_t off = (arena_used + 255) & ~(size_t)255;
    arena_used = off + ((bytes + 15) & ~(size_t)15);
    allocs.push_back({off, bytes});
    return off;
}

// ------------------------------------------------------------------ host-side bounds check
namespace {
struct Checker {
    const Program& pr;
    int ss;
    std::string err;
    bool inside(const std::vector<std::pair<size_t, size_t>>& a, size_t lo, size_t hi) const {
        // a is sorted by offset (allocation order)
        size_t l = 0, r = a.size();
        while (l < r) {
            size_t m = (l + r) / 2;
            if (a[m].first <= lo) l = m + 1;
            else r = m;
        }
        if (l == 0) return false;
        const auto& b = a[l - 1];
        return lo >= b.first && hi <= b.first + b.second;
    }
    void range(const void* p, long long extent_elems, int elem_bytes, const char* what, size_t task) {
        if (!err.empty() || !p) return;
        const size_t lo = (size_t)(uintptr_t)p, hi = lo + (size_t)extent_elems * elem_bytes;
        bool ok;
        if (lo < pr.split || !pr.parent) ok = inside(lo < pr.split && pr.parent ? pr.parent->allocs : pr.allocs, lo, hi);
        else ok = inside(pr.allocs, lo, hi);
        if (!ok) err = std::string(what) + " of task " + std::to_string(task) + " leaves its buffer";
    }
};
long long ext2(long long n1, long long s1, long long n2, long long s2) { return (n1 - 1) * s1 + (n2 - 1) * s2; }
}  // namespace

std::string Program::validate() const {
    Checker c{*this, cplx ? 16 : 8, ""};
    const int ss = c.ss;
    for (size_t i = 0; i < gc.size(); ++i) {
        const GTask& t = gc[i];
        if (t.M1 < 1 || t.M2 < 1 || t.N1 < 1 || t.N2 < 1 || t.K1 < 1 || t.K2 < 1) return "empty contraction " + std::to_string(i);
        if (t.layer_d > 0) {
            const int UL = t.K1 * t.K2, DR = t.N1 * t.N2;
            if (cplx || UL > 32 || DR > 32 || layer_smem_bytes(t.layer_d, UL, DR, false) > LAYER_SMEM_MAX ||
                layer_smem_bytes(t.layer_d, UL, DR, true) > LAYER_SMEM_MAX)
                return "layered contraction out of range in task " + std::to_string(i);
            const long long vol = (long long)UL * DR;
            c.range(t.A, ext2(t.M1, t.a_m1, t.M2, t.a_m2) + ext2((long long)t.K1 * t.K1, t.a_k1, (long long)t.K2 * t.K2, t.a_k2) + 1,
                    ss, "layered A", i);
            const long long text = (t.layer_d - 1) * vol + ext2(t.K1, t.b_k1, t.K2, t.b_k2) + ext2(t.N1, t.b_n1, t.N2, t.b_n2) + 1;
            c.range(t.B, text, ss, "layered Tk", i);
            c.range((const char*)t.B + t.tb_off * ss, text, ss, "layered Tb", i);
            // one offset from the ket to the bra survives relocation only inside one region
            const size_t kb = (size_t)(uintptr_t)t.B, bb = kb + (size_t)(t.tb_off * ss);
            if (parent && t.tb_off != 0 && ((kb < split) != (bb < split)))
                return "layered tensors of task " + std::to_string(i) + " lie in different buffers";
            c.range(t.C, ext2(t.M1, t.c_m1, t.M2, t.c_m2) + ext2((long long)t.N1 * t.N1, t.c_n1, (long long)t.N2 * t.N2, t.c_n2) + 1,
                    ss, "layered C", i);
            c.range(t.active, 1, 4, "active", i);
            continue;
        }
        c.range(t.A, ext2(t.M1, t.a_m1, t.M2, t.a_m2) + ext2(t.K1, t.a_k1, t.K2, t.a_k2) + 1, ss, "A", i);
        c.range(t.B, ext2(t.K1, t.b_k1, t.K2, t.b_k2) + ext2(t.N1, t.b_n1, t.N2, t.b_n2) + 1, ss, "B", i);
        c.range(t.C, ext2(t.M1, t.c_m1, t.M2, t.c_m2) + ext2(t.N1, t.c_n1, t.N2, t.c_n2) + 1, ss, "C", i);
        c.range(t.active, 1, 4, "active", i);
    }
    for (const Step& st : steps) {
        if (st.kind != ST_GC) continue;
        for (int k = 0; k < st.count; ++k)
            if ((gc[st.first + k].layer_d > 0) != ((st.aux2 & GC_LAYER) != 0))
                return "contraction step mixes layered and plain tasks";
    }
    for (size_t i = 0; i < qr.size(); ++i) {
        const QRTask& t = qr[i];
        if (t.n > 512 || t.m < t.n) return "QR shape out of range in task " + std::to_string(i);
        c.range(t.in, ext2(t.m, t.in_rs, t.n, t.in_cs) + 1, t.in_float ? ss / 2 : ss, "QR in", i);
        c.range(t.out, ext2(t.m, t.out_rs, t.n, t.out_cs) + 1, ss, "QR out", i);
        c.range(t.work, 2LL * t.m * t.n, ss, "QR work", i);
        if (t.out2) {
            const int M2 = t.out2_M2 > 1 ? t.out2_M2 : 1;
            const long long ext = (long long)((t.m - 1) / M2) * t.out2_rs + (long long)(std::min(M2, t.m) - 1) * t.out2_rs2 +
                                  (long long)(t.n - 1) * t.out2_cs + 1 + (t.out2_x3 ? t.out2_kseg : 0);
            c.range(t.out2, ext, t.out2_kind == 0 ? 8 : t.out2_kind == 3 ? 2 : 4, "QR out2", i);
        }
        c.range(t.loss, 1, 8, "QR loss", i);
        c.range(t.active, 1, 4, "QR active", i);
    }
    for (size_t i = 0; i < rnd.size(); ++i) {
        c.range(rnd[i].ptr, rnd[i].n, ss, "rand", i);
        c.range(rnd[i].active, 1, 4, "rand active", i);
        c.range(rnd[i].warm_ctr, 1, 4, "rand warm counter", i);
    }
    for (size_t i = 0; i < chk.size(); ++i) {
        c.range(chk[i].losses, chk[i].count, 8, "losses", i);
        c.range(chk[i].active, 1, 4, "check active", i);
        c.range(chk[i].counter, 1, 4, "counter", i);
    }
    for (size_t i = 0; i < scl.size(); ++i) c.range(scl[i].ptr, scl[i].n, ss, "scale", i);
    for (size_t i = 0; i < asmb.size(); ++i) {
        const AssembleTask& t = asmb[i];
        for (int s = 0; s < t.nsites; ++s) {
            c.range(t.src[s], t.size[s], ss, "assemble src", i);
            c.range(t.dst[s], t.size[s], ss, "assemble dst", i);
        }
        c.range(t.corner0, 1, ss, "corner", i);
        c.range(t.corner1, 1, ss, "corner", i);
    }
    for (const Step& s : steps) {
        if (s.kind != ST_DOT) continue;
        for (int k = 0; k < s.count; ++k) {
            const size_t i = s.first + k;
            const DotTask& t = dots[i];
            c.range(t.A, t.n, ss, "dot A", i);
            if (s.aux == 0) c.range(t.B, t.n, ss, "dot B", i);
            c.range(t.out, 1, s.aux == 0 ? ss : 4, "dot out", i);
            c.range(t.ea, 1, 4, "dot exponent", i);
            if (s.aux == 0) c.range(t.eb, 1, 4, "dot exponent", i);
        }
    }
    for (size_t i = 0; i < nrm.size(); ++i) {
        const NormTask& t = nrm[i];
        c.range(t.site0, t.size0, ss, "norm site0", i);
        for (int s = 0; s < t.nsites; ++s) {
            if (t.b[s] > 1024 || t.a[s] > 1024) return "message bond above 1024";
            c.range(t.sites[s], (long long)t.a[s] * t.k[s] * t.b[s], ss, "norm site", i);
        }
        c.range(t.mm, 1, ss, "mm", i);
        c.range(t.mo, 1, ss, "mo", i);
        c.range(t.resid, 1, 8, "resid", i);
    }
    for (size_t i = 0; i < fus.size(); ++i) {
        const FuseTask& t = fus[i];
        c.range(t.A, (t.u1 - 1) * t.a_u + (t.l1 - 1) * t.a_l + (t.d1 - 1) * t.a_d + (t.m - 1) * t.a_r + 1, ss, "fuse A", i);
        c.range(t.B, (t.u2 - 1) * t.b_u + (t.m - 1) * t.b_l + (t.d2 - 1) * t.b_d + (t.r2 - 1) * t.b_r + 1, ss, "fuse B", i);
        c.range(t.out, (long long)t.u1 * t.u2 * t.l1 * t.d1 * t.d2 * t.r2, ss, "fuse out", i);
    }
    for (size_t i = 0; i < dl.size(); ++i) {
        const DLTask& t = dl[i];
        const long long vol = (long long)t.Du * t.Dl * t.Dd * t.Dr;
        const int ts = t.hb ? 16 : ss;  // complex T and O in the Hermitian basis
        c.range(t.T, t.d * vol, ts, "DL T", i);
        c.range(t.E, vol * vol, ss, "DL E", i);
        c.range(t.O, (long long)t.d * t.d, ts, "DL O", i);
    }
    for (size_t i = 0; i < qr.size(); ++i) {
        const QRTask& t = qr[i];
        if (t.in_float) {
            // FP32 input read with the same strides (already checked with the scalar size, which is larger)
        }
    }
    for (size_t i = 0; i < tcs.size(); ++i) {
        const TCTask& t = tcs[i];
        const TCSpec& sp = tcspec[i];
        const int esz = sp.kind == 0 ? 4 : 2;
        if ((sp.a_ld * esz) % 16 || (sp.b_ld * esz) % 16 || sp.K > sp.a_ld || sp.K > sp.b_ld)
            return "tensor-core operand rows not padded to 16 bytes in task " + std::to_string(i);
        if (t.M != sp.a_rows || t.N != sp.b_rows || t.M % t.M2 || t.N % t.N2) return "tensor-core shape mismatch " + std::to_string(i);
        if (t.nseg == 3 && (!sp.a_pl || !sp.b_pl || (sp.a_pl * esz) % 16 || (sp.b_pl * esz) % 16))
            return "split tensor-core operand without an aligned second plane in task " + std::to_string(i);
        c.range(P(sp.a_off), (sp.a_rows - 1) * sp.a_ld + sp.K + sp.a_pl, esz, "TC A", i);
        c.range(P(sp.b_off), (sp.b_rows - 1) * sp.b_ld + sp.K + sp.b_pl, esz, "TC B", i);
        const int osz = t.out_kind == 2 ? 2 : t.out_kind == 3 ? 8 : 4;
        const long long xc = (t.x3 & 3) ? t.kseg : 0, xd = ((t.x3 >> 2) & 3) ? t.kseg2 : 0;  // split: second plane
        c.range(t.C, ext2(t.M / t.M2, t.c_m1, t.M2, t.c_m2) + ext2(t.N / t.N2, t.c_n1, t.N2, t.c_n2) + 1 + xc, osz, "TC C", i);
        if (t.C2) c.range(t.C2, ext2(t.M / t.M2, t.d_m1, t.M2, t.d_m2) + ext2(t.N / t.N2, t.d_n1, t.N2, t.d_n2) + 1 + xd, osz, "TC C2", i);
        c.range(t.active, 1, 4, "TC active", i);
    }
    for (size_t i = 0; i < rel.size(); ++i) {
        const RelayoutTask& t = rel[i];
        long long se = 1, de = 1;
        for (int k = 0; k < 4; ++k) {
            se += (long long)(t.d[k] - 1) * t.ss[k];
            de += (long long)(t.d[k] - 1) * t.ds[k];
        }
        auto ksz = [](int k) { return k == 0 ? 8 : k == 3 ? 2 : 4; };
        c.range(t.src, se, ksz(t.src_kind), "relayout src", i);
        c.range(t.dst, de + (t.x3 ? t.kseg : 0), ksz(t.dst_kind), "relayout dst", i);
    }
    for (size_t i = 0; i < steps.size(); ++i) {
        const Step& s = steps[i];
        if (s.kind == ST_COPY) {
            c.range(s.p0, s.n, 1, "copy src", i);
            c.range(s.p1, s.n, 1, "copy dst", i);
            if (s.n % 16) return "copy size not a multiple of 16 bytes";
        }
        if (s.kind == ST_MEAN) {
            c.range(s.p0, s.n, 8, "mean in", i);
            c.range(s.p1, 1, 8, "mean out", i);
        }
        if (s.kind == ST_INC) c.range(s.p0, 1, 4, "counter", i);
        if (s.kind == ST_LOOP_BEGIN) c.range(s.p0, (long long)sizeof(LoopDesc), 1, "loop descriptor", i);
        if (s.kind == ST_CHECK && s.p1) c.range(s.p1, (long long)sizeof(LoopDesc), 1, "loop descriptor", i);
    }
    return c.err;
}

void Program::gc_step(std::vector<GTask>& ts) {
    if (ts.empty()) return;
    Step s;
    s.kind = ST_GC;
    s.first = gc.size();
    s.count = (int)ts.size();
    // 64x64 output tiles, or 16x16 ones (k_gcontract_small) when every task has an output
    // dimension of at most 16, where a 64x64 tile would be mostly padding
    bool small = true;
    for (auto& t : ts) small = small && std::min((long long)t.M1 * t.M2, (long long)t.N1 * t.N2) <= 16;
    const int tile = small ? 16 : 64;
    int mt = 1;
    for (auto& t : ts) {
        const long long M = (long long)t.M1 * t.M2, N = (long long)t.N1 * t.N2, K = (long long)t.K1 * t.K2;
        const int tiles = (int)(((M + tile - 1) / tile) * ((N + tile - 1) / tile));
        mt = std::max(mt, tiles);
        const double f = 2.0 * (double)M * (double)N * (double)K * (cplx ? 4.0 : 1.0);
        count_flops(t.active, f, false);
        gc.push_back(t);
    }
    s.aux = mt;
    s.aux2 = (small ? 1 : 0) | (gc_f32 ? GC_F32 : 0);
    steps.push_back(s);
    ts.clear();
}

void Program::layer_step(std::vector<GTask>& ts) {
    if (ts.empty()) return;
    Step s;
    s.kind = ST_GC;
    s.first = gc.size();
    s.count = (int)ts.size();
    int mt = 1;
    long long smem = 0;
    const int apt = gc_f32 ? LAYER_APT_F32 : LAYER_APT_F64;
    for (auto& t : ts) {
        const int UL = t.K1 * t.K2, DR = t.N1 * t.N2;
        mt = std::max(mt, t.M1 * ((t.M2 + apt - 1) / apt));
        smem = std::max(smem, (long long)layer_smem_bytes(t.layer_d, UL, DR, gc_f32));
        const double f = 2.0 * t.layer_d * UL * DR * (double)(UL + DR) * t.M1 * t.M2;
        count_flops(t.active, f, false);
        gc.push_back(t);
    }
    s.aux = mt;
    s.aux2 = GC_LAYER | (gc_f32 ? GC_F32 : 0);
    s.n = smem;
    steps.push_back(s);
    ts.clear();
}

void Program::count_flops(const int* active, double f, bool qr_step) {
    if (!active) {
        (qr_step ? static_qr_flops : static_flops) += f;
        return;
    }
    (qr_step ? gated_qr_flops : gated_flops) += f;
    (qr_step ? fit_qr_flops : fit_flops)[(uintptr_t)active] += f;
}

void Program::qr_step(std::vector<QRTask>& ts) {
    if (ts.empty()) return;
    Step s;
    s.kind = ST_QR;
    s.first = qr.size();
    s.count = (int)ts.size();
    int mm = 1;
    long long mn = 1;
    int f32 = 0;
    for (auto& t : ts) {
        f32 += t.in_float == 2;
        mm = std::max(mm, t.m);
        mn = std::max(mn, (long long)t.m * t.n);
        const double f = (4.0 * t.m * (double)t.n * t.n - 4.0 / 3.0 * (double)t.n * t.n * t.n) * (cplx ? 4.0 : 1.0);
        count_flops(t.active, f, true);
        qr.push_back(t);
    }
    s.aux = mm;
    s.n = mn;
    // FP32-arithmetic tasks form steps of their own (the planner never mixes the two)
    if (f32 != 0 && f32 != (int)ts.size()) throw std::logic_error("QR step mixes FP32 and FP64 arithmetic");
    s.aux2 = f32 ? QR_F32 : 0;
    max_qr_m = std::max(max_qr_m, mm);
    steps.push_back(s);
    ts.clear();
}

size_t Program::lp_alloc(size_t elems, int esz, bool split) {
    const size_t off = arena_alloc((split ? 2 : 1) * elems * (size_t)esz);
    if (split) planes[off] = (long long)elems;
    return off;
}

long long Program::plane_of(size_t byte_off) const {
    auto it = planes.find(byte_off);
    if (it != planes.end()) return it->second;
    if (parent && byte_off < split) return parent->plane_of(byte_off);  // the lattice's own buffers
    throw std::logic_error("internal: split operand without a second plane");
}

void Program::dot_step(std::vector<DotTask>& ts, bool normalise) {
    if (ts.empty()) return;
    Step s;
    s.kind = ST_DOT;
    s.first = dots.size();
    s.count = (int)ts.size();
    s.aux = normalise ? 1 : 0;
    for (auto& t : ts) {
        if (!normalise) count_flops(nullptr, 2.0 * (double)t.n * (cplx ? 4.0 : 1.0), false);
        dots.push_back(t);
    }
    steps.push_back(s);
    ts.clear();
}

template <typename T>
static size_t push_all(std::vector<T>& dst, std::vector<T>& src) {
    size_t f = dst.size();
    dst.insert(dst.end(), src.begin(), src.end());
    src.clear();
    return f;
}

void Program::simple(int kind, void* p0, void* p1, long long n, int aux) {
    Step s;
    s.kind = kind;
    s.p0 = p0;
    s.p1 = p1;
    s.n = n;
    s.aux = aux;
    steps.push_back(s);
}


// ------------------------------------------------------------------ the zip-up fit (App. A)
// Element offsets inside the arena are converted to byte offsets with the scalar size.
struct Emit {
    Program& pr;
    int ss;
    const int* none = nullptr;
    void* ep(size_t elem_off) const { return P(elem_off * (size_t)ss); }
};

// L->R site update at site i of fit f:  T1 = A X ; T2 = T1 O ; Yt = T2 B ; (QR) ; A' = conj(Y) T2
static void lr_gc(const Emit& e, const FitSpec& f, int i, int stage, const int* act, std::vector<GTask>& out) {
    const View3& X = f.X[i];
    const View4& O = f.O[i];
    const int y = f.ybond[i], y2 = f.ybond[i + 1];
    const int x = X.a, x2 = X.b, p = X.k, w = O.w, w2 = O.w2, q = O.q;
    GTask t{};
    t.active = act;
    if (stage == 0) {  // T1[y][w][p][x2] = sum_x A[y,w,x] X[x,p,x2]
        t.A = e.ep(f.Aenv[i]);
        t.B = e.ep(X.off);
        t.C = e.ep(f.T1);
        t.M1 = y; t.M2 = w; t.K1 = 1; t.K2 = x; t.N1 = p; t.N2 = x2;
        t.a_m1 = (long long)w * x; t.a_m2 = x; t.a_k2 = 1;
        t.b_k2 = X.sa; t.b_n1 = X.sk; t.b_n2 = X.sb;
        t.c_m1 = (long long)w * p * x2; t.c_m2 = (long long)p * x2; t.c_n1 = x2; t.c_n2 = 1;
    } else if (stage == 1) {  // T2[y][x2][q][w2] = sum_{w,p} T1[y,w,p,x2] O[w,p,q,w2]
        t.A = e.ep(f.T1);
        t.B = e.ep(O.off);
        t.C = e.ep(f.T2);
        t.M1 = y; t.M2 = x2; t.K1 = w; t.K2 = p; t.N1 = q; t.N2 = w2;
        t.a_m1 = (long long)w * p * x2; t.a_m2 = 1; t.a_k1 = (long long)p * x2; t.a_k2 = x2;
        t.b_k1 = O.sw; t.b_k2 = O.sp; t.b_n1 = O.sq; t.b_n2 = O.sw2;
        t.c_m1 = (long long)x2 * q * w2; t.c_m2 = (long long)q * w2; t.c_n1 = w2; t.c_n2 = 1;
    } else if (stage == 2) {  // Yt[y][q][y2] = sum_{x2,w2} T2[y,x2,q,w2] B[y2,w2,x2]
        t.A = e.ep(f.T2);
        t.B = e.ep(f.Benv[i + 1]);
        t.C = e.ep(f.Yt);
        t.M1 = y; t.M2 = q; t.K1 = x2; t.K2 = w2; t.N1 = 1; t.N2 = y2;
        t.a_m1 = (long long)x2 * q * w2; t.a_m2 = w2; t.a_k1 = (long long)q * w2; t.a_k2 = 1;
        t.b_k1 = 1; t.b_k2 = x2; t.b_n2 = (long long)w2 * x2;
        t.c_m1 = (long long)q * y2; t.c_m2 = y2; t.c_n2 = 1;
    } else {  // A_{i+1}[y2][w2][x2] = sum_{y,q} conj(Y[y,q,y2]) T2[y,x2,q,w2]
        t.A = e.ep(f.Y[i]);
        t.B = e.ep(f.T2);
        t.C = e.ep(f.Aenv[i + 1]);
        t.conjA = 1;
        t.M1 = 1; t.M2 = y2; t.K1 = y; t.K2 = q; t.N1 = w2; t.N2 = x2;
        t.a_m2 = 1; t.a_k1 = (long long)q * y2; t.a_k2 = y2;
        t.b_k1 = (long long)x2 * q * w2; t.b_k2 = w2; t.b_n1 = 1; t.b_n2 = (long long)q * w2;
        t.c_m2 = (long long)w2 * x2; t.c_n1 = x2; t.c_n2 = 1;
    }
    out.push_back(t);
}

// R->L site update at site i:  T1 = X B ; T2 = T1 O ; Yt = A T2 ; (LQ) ; B_i = conj(Y) T2
// With Ydst != 0 the Yt of stage 2 is written there (final update of the fit).
static void rl_gc(const Emit& e, const FitSpec& f, int i, int stage, const int* act, std::vector<GTask>& out,
                  size_t Ydst = 0) {
    const View3& X = f.X[i];
    const View4& O = f.O[i];
    const int y = f.ybond[i], y2 = f.ybond[i + 1];
    const int x = X.a, x2 = X.b, p = X.k, w = O.w, w2 = O.w2, q = O.q;
    GTask t{};
    t.active = act;
    if (stage == 0) {  // T1[x][p][y2][w2] = sum_x2 X[x,p,x2] B[y2,w2,x2]
        t.A = e.ep(X.off);
        t.B = e.ep(f.Benv[i + 1]);
        t.C = e.ep(f.T1);
        t.M1 = x; t.M2 = p; t.K1 = 1; t.K2 = x2; t.N1 = y2; t.N2 = w2;
        t.a_m1 = X.sa; t.a_m2 = X.sk; t.a_k2 = X.sb;
        t.b_k2 = 1; t.b_n1 = (long long)w2 * x2; t.b_n2 = x2;
        t.c_m1 = (long long)p * y2 * w2; t.c_m2 = (long long)y2 * w2; t.c_n1 = w2; t.c_n2 = 1;
    } else if (stage == 1) {  // T2[x][y2][w][q] = sum_{p,w2} T1[x,p,y2,w2] O[w,p,q,w2]
        t.A = e.ep(f.T1);
        t.B = e.ep(O.off);
        t.C = e.ep(f.T2);
        t.M1 = x; t.M2 = y2; t.K1 = p; t.K2 = w2; t.N1 = w; t.N2 = q;
        t.a_m1 = (long long)p * y2 * w2; t.a_m2 = w2; t.a_k1 = (long long)y2 * w2; t.a_k2 = 1;
        t.b_k1 = O.sp; t.b_k2 = O.sw2; t.b_n1 = O.sw; t.b_n2 = O.sq;
        t.c_m1 = (long long)y2 * w * q; t.c_m2 = (long long)w * q; t.c_n1 = q; t.c_n2 = 1;
    } else if (stage == 2) {  // Yt[y][q][y2] = sum_{w,x} A[y,w,x] T2[x,y2,w,q]
        t.A = e.ep(f.Aenv[i]);
        t.B = e.ep(f.T2);
        t.C = e.ep(Ydst ? Ydst : f.Yt);
        t.M1 = 1; t.M2 = y; t.K1 = w; t.K2 = x; t.N1 = q; t.N2 = y2;
        t.a_m2 = (long long)w * x; t.a_k1 = x; t.a_k2 = 1;
        t.b_k1 = q; t.b_k2 = (long long)y2 * w * q; t.b_n1 = 1; t.b_n2 = (long long)w * q;
        t.c_m2 = (long long)q * y2; t.c_n1 = y2; t.c_n2 = 1;
    } else {  // B_i[y][w][x] = sum_{q,y2} conj(Y[y,q,y2]) T2[x,y2,w,q]
        t.A = e.ep(f.Y[i]);
        t.B = e.ep(f.T2);
        t.C = e.ep(f.Benv[i]);
        t.conjA = 1;
        t.M1 = 1; t.M2 = y; t.K1 = q; t.K2 = y2; t.N1 = w; t.N2 = x;
        t.a_m2 = (long long)q * y2; t.a_k1 = y2; t.a_k2 = 1;
        t.b_k1 = 1; t.b_k2 = (long long)w * q; t.b_n1 = q; t.b_n2 = (long long)y2 * w * q;
        t.c_m2 = (long long)w * x; t.c_n1 = x; t.c_n2 = 1;
    }
    out.push_back(t);
}

static QRTask qr_task(const Emit& e, const FitSpec& f, int i, bool lq, size_t loss_elem, const int* act) {
    const int y = f.ybond[i], y2 = f.ybond[i + 1], q = f.O[i].q;
    QRTask t{};
    t.in = e.ep(f.Yt);
    t.out = e.ep(f.Y[i]);
    t.work = e.ep(f.qrw);
    t.loss = (double*)P(loss_elem);
    t.active = act;
    if (!lq) {
        t.m = y * q; t.n = y2;
        t.in_rs = y2; t.in_cs = 1; t.out_rs = y2; t.out_cs = 1; t.conj_io = 0;
    } else {
        t.m = q * y2; t.n = y;
        t.in_rs = 1; t.in_cs = (long long)q * y2; t.out_rs = 1; t.out_cs = (long long)q * y2; t.conj_io = 1;
    }
    return t;
}

// Emit a lockstep group of fits.  losses_byte / active / counters are byte offsets
// of per-fit arrays (losses: fit_max_sweeps * 2(n-1) doubles per fit).
void emit_fits(Program& pr, int ss, std::vector<FitSpec*>& fits, int max_sweeps, double fit_tol,
               bool warm, bool rand_uses_sweep) {
    Emit e{pr, ss};
    int nmax = 0;
    for (auto* f : fits) nmax = std::max(nmax, f->n());
    // 1. random initial Y (App. A initialises Y at random)
    {
        std::vector<RandTask> rt;
        for (auto* f : fits)
            for (int i = 0; i < f->n(); ++i) {
                RandTask t{};
                t.ptr = e.ep(f->Y[i]);
                t.n = (long long)f->ybond[i] * f->O[i].q * f->ybond[i + 1];
                t.stream = f->stream + (uint64_t)i;
                t.active = i == 0 ? (int*)P(f->active) : nullptr;
                t.warm = (warm || f->warm) ? 1 : 0;
                t.warm_ctr = t.warm ? (const int*)P(pr.warm_ctr_off) : nullptr;
                rt.push_back(t);
            }
        Step s;
        s.kind = ST_RAND;
        s.count = (int)rt.size();
        s.first = push_all(pr.rnd, rt);
        s.aux = rand_uses_sweep ? 1 : 0;
        pr.steps.push_back(s);
    }
    // 2. right environments from the initial Y (A_1 = B_{L+1} = 1)
    std::vector<GTask> g;
    for (int k = 0; k <= nmax - 2; ++k)
        for (int stage : {0, 1, 3}) {
            for (auto* f : fits) {
                const int i = f->n() - 1 - k;
                if (i >= 1) rl_gc(e, *f, i, stage, nullptr, g);
            }
            pr.gc_step(g);
        }
    // 3. sweeps
    std::vector<QRTask> qt;
    // the fit sweeps: one gated loop body (a conditional WHILE node in the graph)
    const size_t loopd = pr.arena_alloc(sizeof(LoopDesc));
    pr.loop_descs.push_back({loopd, max_sweeps});
    pr.simple(ST_LOOP_BEGIN, P(loopd), nullptr, 0, max_sweeps);
    {
        const int s = 0;
        for (int k = 0; k <= nmax - 2; ++k) {
            for (int stage = 0; stage < 3; ++stage) {
                for (auto* f : fits)
                    if (k <= f->n() - 2) lr_gc(e, *f, k, stage, (const int*)P(f->active), g);
                pr.gc_step(g);
            }
            for (auto* f : fits)
                if (k <= f->n() - 2) {
                    const size_t loss = f->losses + (size_t)k * sizeof(double);
                    qt.push_back(qr_task(e, *f, k, false, loss, (const int*)P(f->active)));
                }
            pr.qr_step(qt);
            for (auto* f : fits)
                if (k <= f->n() - 2) lr_gc(e, *f, k, 3, (const int*)P(f->active), g);
            pr.gc_step(g);
        }
        for (int k = 0; k <= nmax - 2; ++k) {
            for (int stage = 0; stage < 3; ++stage) {
                for (auto* f : fits) {
                    const int i = f->n() - 1 - k;
                    if (i >= 1) rl_gc(e, *f, i, stage, (const int*)P(f->active), g);
                }
                pr.gc_step(g);
            }
            for (auto* f : fits) {
                const int i = f->n() - 1 - k;
                if (i >= 1) {
                    const size_t loss = f->losses + (size_t)((f->n() - 1) + k) * sizeof(double);
                    qt.push_back(qr_task(e, *f, i, true, loss, (const int*)P(f->active)));
                }
            }
            pr.qr_step(qt);
            for (auto* f : fits) {
                const int i = f->n() - 1 - k;
                if (i >= 1) rl_gc(e, *f, i, 3, (const int*)P(f->active), g);
            }
            pr.gc_step(g);
        }
        // stop rule after the full sweep (App. A)
        std::vector<CheckTask> ct;
        for (auto* f : fits) {
            CheckTask t{};
            const int nu = 2 * (f->n() - 1);
            t.losses = (const double*)P(f->losses);
            t.active = (int*)P(f->active);
            t.count = nu;
            t.counter = (int*)P(f->counter);
            ct.push_back(t);
        }
        Step st;
        st.kind = ST_CHECK;
        st.p1 = P(loopd);
        st.count = (int)ct.size();
        st.first = push_all(pr.chk, ct);
        pr.steps.push_back(st);
        pr.fit_tol = fit_tol;
        (void)s;
    }
    pr.simple(ST_LOOP_END, nullptr, nullptr, 0, 0);
    // 4. final update at site 0 keeps Yt itself
    for (int stage = 0; stage < 3; ++stage) {
        for (auto* f : fits) rl_gc(e, *f, 0, stage, nullptr, g, stage == 2 ? f->Y[0] : 0);
        pr.gc_step(g);
    }
    // 5. unit norm (mixed canonical form around site 0)
    std::vector<ScaleTask> sc;
    for (auto* f : fits) {
        ScaleTask t{};
        t.ptr = e.ep(f->Y[0]);
        t.n = (long long)f->ybond[0] * f->O[0].q * f->ybond[1];
        sc.push_back(t);
    }
    Step st;
    st.kind = ST_SCALE;
    st.count = (int)sc.size();
    st.first = push_all(pr.scl, sc);
    pr.steps.push_back(st);
}

// <M|N> chains for a set of message pairs: per site T = E N, E' = conj(M) T.
void emit_overlaps(Program& pr, int ss, std::vector<OverlapSpec>& ov) {
    Emit e{pr, ss};
    int bmax = 0;
    for (auto& o : ov) bmax = std::max(bmax, (int)o.M.size());
    std::vector<GTask> g;
    for (int j = 0; j < bmax; ++j) {
        for (auto& o : ov) {
            if (j >= (int)o.M.size()) continue;
            const View3& M = o.M[j];
            const View3& N = o.N[j];
            const size_t Ein = j == 0 ? o.one : o.E[j % 2];
            GTask t{};
            t.A = e.ep(Ein);
            t.B = e.ep(N.off);
            t.C = e.ep(o.T);
            t.M1 = 1; t.M2 = M.a; t.K1 = 1; t.K2 = N.a; t.N1 = N.k; t.N2 = N.b;
            t.a_m2 = N.a; t.a_k2 = 1;
            t.b_k2 = N.sa; t.b_n1 = N.sk; t.b_n2 = N.sb;
            t.c_m2 = (long long)N.k * N.b; t.c_n1 = N.b; t.c_n2 = 1;
            g.push_back(t);
        }
        pr.gc_step(g);
        for (auto& o : ov) {
            if (j >= (int)o.M.size()) continue;
            const View3& M = o.M[j];
            const View3& N = o.N[j];
            const size_t Eout = (j + 1 == (int)o.M.size()) ? o.result : o.E[(j + 1) % 2];
            GTask t{};
            t.A = e.ep(M.off);
            t.B = e.ep(o.T);
            t.C = e.ep(Eout);
            t.conjA = 1;
            t.M1 = 1; t.M2 = M.b; t.K1 = M.a; t.K2 = M.k; t.N1 = 1; t.N2 = N.b;
            t.a_m2 = M.sb; t.a_k1 = M.sa; t.a_k2 = M.sk;
            t.b_k1 = (long long)N.k * N.b; t.b_k2 = N.b; t.b_n2 = 1;
            t.c_m2 = N.b; t.c_n2 = 1;
            g.push_back(t);
        }
        pr.gc_step(g);
    }
}

// ------------------------------------------------------------------ relocation and upload
// Offsets below `split` belong to the lattice arena (base), the rest to a second
// arena (base2) whose offsets start at `split`.
static inline char* reloc_ptr(uintptr_t off, char* base, size_t split, char* base2) {
    if (off < split) return base + off;
    return base2 + (off - split);
}
#define RELOC(field)                                                                                        \
    field = (std::remove_reference_t<decltype(field)>)((field) ? reloc_ptr((uintptr_t)(field), base, split, base2) \
                                                               : nullptr)

void Program::relocate(char* base, size_t split, char* base2) {
    for (auto& t : gc) {
        RELOC(t.A); RELOC(t.B); RELOC(t.C); RELOC(t.active);
    }
    for (auto& t : qr) {
        RELOC(t.in); RELOC(t.out); RELOC(t.work); RELOC(t.loss); RELOC(t.active);
    }
    for (auto& t : rnd) {
        RELOC(t.ptr); RELOC(t.active); RELOC(t.warm_ctr);
    }
    if (chk_keys.empty())
        for (auto& t : chk) chk_keys.push_back((uintptr_t)t.active);
    for (auto& t : chk) {
        RELOC(t.losses); RELOC(t.active); RELOC(t.counter);
    }
    for (auto& t : scl) RELOC(t.ptr);
    for (auto& t : asmb) {
        for (int s = 0; s < t.nsites; ++s) {
            RELOC(t.src[s]); RELOC(t.dst[s]);
        }
        RELOC(t.corner0); RELOC(t.corner1);
    }
    for (auto& t : nrm) {
        RELOC(t.site0);
        for (int s = 0; s < t.nsites; ++s) RELOC(t.sites[s]);
        RELOC(t.mm); RELOC(t.mo); RELOC(t.resid); RELOC(t.status);
    }
    for (auto& t : fus) {
        RELOC(t.A); RELOC(t.B); RELOC(t.out);
    }
    for (auto& t : dl) {
        RELOC(t.T); RELOC(t.E); RELOC(t.O);
    }
    for (auto& t : dots) {
        RELOC(t.A); RELOC(t.B); RELOC(t.out); RELOC(t.ea); RELOC(t.eb);
    }
    for (auto& t : tcs) {
        RELOC(t.C); RELOC(t.C2); RELOC(t.active);
    }
    for (auto& t : rel) {
        RELOC(t.src); RELOC(t.dst);
    }
    for (auto& t : qr) {
        RELOC(t.out2);
    }
    for (auto& s : steps) {
        RELOC(s.p0); RELOC(s.p1);
    }
    loop_ptr.clear();
    for (auto& l : loop_descs) loop_ptr.push_back(reloc_ptr(l.first, base, split, base2));
}

cudaError_t Program::encode_maps(char* base, size_t split, char* base2) {
    for (size_t i = 0; i < tcs.size(); ++i) {
        const TCSpec& sp = tcspec[i];
        const int esz = sp.kind == 0 ? 4 : 2;
        cudaError_t e = tc_make_map(&tcs[i].map_a, reloc_ptr(sp.a_off, base, split, base2), sp.kind, sp.a_rows, sp.K,
                                    sp.a_ld, 128);
        if (e != cudaSuccess) return e;
        e = tc_make_map(&tcs[i].map_b, reloc_ptr(sp.b_off, base, split, base2), sp.kind, sp.b_rows, sp.K, sp.b_ld, sp.bn);
        if (e != cudaSuccess) return e;
        if (tcs[i].nseg == 3) {  // the lo planes
            e = tc_make_map(&tcs[i].map_a2, reloc_ptr(sp.a_off, base, split, base2) + sp.a_pl * esz, sp.kind, sp.a_rows,
                            sp.K, sp.a_ld, 128);
            if (e != cudaSuccess) return e;
            e = tc_make_map(&tcs[i].map_b2, reloc_ptr(sp.b_off, base, split, base2) + sp.b_pl * esz, sp.kind, sp.b_rows,
                            sp.K, sp.b_ld, sp.bn);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t Program::tc_retile(size_t si, int bn, int depth, char* base, size_t split, char* base2, cudaStream_t st,
                               int ksub) {
    Step& s = steps[si];
    int tiles = 1;
    for (int i = 0; i < s.count; ++i) {
        const size_t k = s.first + (size_t)i;
        TCSpec& sp = tcspec[k];
        sp.bn = bn;
        cudaError_t e = tc_make_map(&tcs[k].map_b, reloc_ptr(sp.b_off, base, split, base2), sp.kind, sp.b_rows, sp.K,
                                    sp.b_ld, bn);
        if (e != cudaSuccess) return e;
        if (tcs[k].nseg == 3) {
            e = tc_make_map(&tcs[k].map_b2, reloc_ptr(sp.b_off, base, split, base2) + sp.b_pl * (sp.kind == 0 ? 4 : 2),
                            sp.kind, sp.b_rows, sp.K, sp.b_ld, bn);
            if (e != cudaSuccess) return e;
        }
        tiles = std::max(tiles, ((tcs[k].M + 127) / 128) * ((tcs[k].N + bn - 1) / bn));
    }
    s.aux = bn;
    s.n = tiles;
    s.aux2 = (s.aux2 & 0xFF) | (depth << 8) | (ksub << 16);
    return cudaMemcpyAsync(d_tcs + s.first, tcs.data() + s.first, (size_t)s.count * sizeof(TCTask), cudaMemcpyHostToDevice,
                           st);
}

// Stream-ordered allocations (cudaMallocAsync / cudaFreeAsync) do not synchronise the
// device, so creating or destroying one lattice never waits for another's kernels.
template <typename T>
static cudaError_t upload(std::vector<T>& v, T** dptr, cudaStream_t st) {
    *dptr = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMallocAsync((void**)dptr, v.size() * sizeof(T), st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

cudaError_t Program::upload_tasks(cudaStream_t st) {
    cudaError_t e;
    if ((e = upload(gc, &d_gc, st)) != cudaSuccess) return e;
    if ((e = upload(qr, &d_qr, st)) != cudaSuccess) return e;
    if ((e = upload(rnd, &d_rnd, st)) != cudaSuccess) return e;
    if ((e = upload(chk, &d_chk, st)) != cudaSuccess) return e;
    if ((e = upload(scl, &d_scl, st)) != cudaSuccess) return e;
    if ((e = upload(asmb, &d_asm, st)) != cudaSuccess) return e;
    if ((e = upload(nrm, &d_nrm, st)) != cudaSuccess) return e;
    if ((e = upload(fus, &d_fus, st)) != cudaSuccess) return e;
    if ((e = upload(dl, &d_dl, st)) != cudaSuccess) return e;
    if ((e = upload(dots, &d_dot, st)) != cudaSuccess) return e;
    if ((e = upload(tcs, &d_tcs, st)) != cudaSuccess) return e;
    if ((e = upload(rel, &d_rel, st)) != cudaSuccess) return e;
    if (!tcs.empty()) {
        if ((e = tc_prepare()) != cudaSuccess) return e;
    }
    if (max_qr_m > 0) {
        if ((e = qr_prepare(max_qr_m, cplx)) != cudaSuccess) return e;
    }
    for (const Step& s : steps)
        if (s.kind == ST_GC && (s.aux2 & GC_LAYER)) {
            if ((e = layer_prepare()) != cudaSuccess) return e;
            break;
        }
    return cudaSuccess;
}

cudaError_t Program::launch_step(const Step& s, cudaStream_t st, const int* sweep_ctr, unsigned long long seed) const {
    switch (s.kind) {
        case ST_GC: return launch_gcontract(d_gc + s.first, s.count, s.aux, cplx, st, s.aux2, s.n);
        case ST_QR: return launch_qr(d_qr + s.first, s.count, s.aux, s.n, cplx, st, s.aux2);
        case ST_RAND: return launch_rand(d_rnd + s.first, s.count, seed, s.aux ? sweep_ctr : nullptr, cplx, st);
        case ST_SETACT: return launch_set_int((int*)s.p0, (int)s.n, s.aux, st);
        case ST_CHECK: return launch_check(d_chk + s.first, s.count, fit_tol, (LoopDesc*)s.p1, st);
        case ST_SCALE: return launch_scale(d_scl + s.first, s.count, cplx, status, st);
        case ST_ASM: return launch_assemble(d_asm + s.first, s.count, cplx, st);
        case ST_NORM: return launch_normalise(d_nrm + s.first, s.count, cplx, st);
        case ST_MEAN: return launch_mean((const double*)s.p0, (int)s.n, (double*)s.p1, st);
        case ST_COPY: return launch_copy(s.p0, s.p1, s.n, st);
        case ST_INC: return launch_add_int((int*)s.p0, 1, st);
        case ST_FUSE: return launch_fuse(d_fus + s.first, s.count, s.n, cplx, st);
        case ST_DL:
            return s.aux2 == 1 ? launch_double_layer_hb(d_dl + s.first, s.count, s.n, st)
                               : launch_double_layer(d_dl + s.first, s.count, s.n, cplx, st);
        case ST_TC: return launch_tc_gemm(d_tcs + s.first, s.count, s.aux2 & 0xFF, s.aux, (int)s.n, (s.aux2 >> 8) & 0xFF, tc_err, st,
                                          (s.aux2 >> 16) & 0xFF);
        case ST_REL: return launch_relayout(d_rel + s.first, s.count, s.n, st);
        case ST_DOT: return launch_dot(d_dot + s.first, s.count, cplx, st, s.aux);
        case ST_LOOP_BEGIN: return launch_set_int((int*)s.p0, 1, 0, st);  // iteration counter = 0
        case ST_LOOP_END: return cudaSuccess;
        default: return cudaErrorInvalidValue;
    }
}

size_t Program::loop_end(size_t b) const {
    for (size_t e = b + 1; e < steps.size(); ++e)
        if (steps[e].kind == ST_LOOP_END) return e;
    return steps.size();
}

// Direct launches: a loop body runs its maximum number of times; the fits that have
// converged skip their work inside every kernel of the body.
cudaError_t Program::launch_all(cudaStream_t st, const int* sweep_ctr, unsigned long long seed) const {
    for (size_t i = 0; i < steps.size(); ++i) {
        cudaError_t e = launch_step(steps[i], st, sweep_ctr, seed);
        if (e != cudaSuccess) return e;
        if (steps[i].kind == ST_LOOP_BEGIN) {
            const size_t end = loop_end(i);
            for (int r = 0; r < steps[i].aux; ++r)
                for (size_t j = i + 1; j < end; ++j) {
                    e = launch_step(steps[j], st, sweep_ctr, seed);
                    if (e != cudaSuccess) return e;
                }
            i = end;
        }
    }
    return cudaSuccess;
}

cudaError_t Program::init_loops(cudaStream_t st, bool in_graph, const unsigned long long* handles) const {
    for (size_t k = 0; k < loop_descs.size(); ++k) {
        LoopDesc d{};
        d.iter = 0;
        d.total = 0;
        d.max = loop_descs[k].second;
        d.use_handle = in_graph ? 1 : 0;
        d.handle = in_graph ? handles[k] : 0ull;
        cudaError_t e = cudaMemcpyAsync(loop_ptr[k], &d, sizeof(d), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(st);
}

cudaError_t Program::reset_loop_totals(cudaStream_t st) const {
    for (void* p : loop_ptr) {
        cudaError_t e = cudaMemsetAsync((char*)p + offsetof(LoopDesc, total), 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    for (const auto& t : chk) {  // each fit's count of the fit sweeps it ran
        cudaError_t e = cudaMemsetAsync(t.counter, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One CUDA graph for the whole program; every loop becomes a conditional WHILE node
// whose body graph is captured on a second stream.
cudaError_t Program::build_graph(cudaStream_t st, const int* sweep_ctr, unsigned long long seed) {
    cudaStream_t body_stream = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&body_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    std::vector<unsigned long long> handles;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    for (size_t i = 0; e == cudaSuccess && i < steps.size(); ++i) {
        e = launch_step(steps[i], st, sweep_ctr, seed);
        if (e != cudaSuccess || steps[i].kind != ST_LOOP_BEGIN) continue;
        const size_t end = loop_end(i);
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
        if (e != cudaSuccess) break;
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) break;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
        e = cudaGraphAddNode(&node, cg, dv.data(), nullptr, dv.size(), &np);
        if (e != cudaSuccess) break;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        for (size_t j = i + 1; e == cudaSuccess && j < end; ++j) e = launch_step(steps[j], body_stream, sweep_ctr, seed);
        cudaGraph_t bout = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(body_stream, &bout);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) break;
        e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        handles.push_back((unsigned long long)h);
        i = end;
    }
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(body_stream);
    if (e != cudaSuccess) return e;
    return init_loops(st, true, handles.data());
}

cudaError_t Program::reset_active(cudaStream_t st) const {
    for (const RandTask& t : rnd)
        if (t.active) {
            cudaError_t e = launch_set_int(t.active, 1, 1, st);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

static int step_class(int kind) {
    if (kind == ST_TC) return 0;
    if (kind == ST_GC) return 1;
    if (kind == ST_QR) return 2;
    return 3;
}

int Program::step_class_of(const Step& s) const { return step_class(s.kind); }

void Program::step_work(const Step& s, double* flops, double* bytes, long long* max_m, long long* max_n,
                        long long* max_k) const {
    double f = 0, b = 0;
    long long mm = 0, mn = 0, mk = 0;
    const int ss = cplx ? 16 : 8;
    switch (s.kind) {
        case ST_GC:
            for (int i = 0; i < s.count; ++i) {
                const GTask& t = gc[s.first + i];
                const double M = (double)t.M1 * t.M2, N = (double)t.N1 * t.N2, K = (double)t.K1 * t.K2;
                if (t.layer_d > 0) {  // pairs: an input matrix K^2 in, an output N^2 out
                    f += 2.0 * t.layer_d * K * N * (K + N) * M;
                    b += M * (K * K + N * N) * ss;
                    mm = std::max(mm, (long long)M); mn = std::max(mn, (long long)(N * N)); mk = std::max(mk, (long long)(K * K));
                    continue;
                }
                f += 2.0 * M * N * K * (cplx ? 4.0 : 1.0);
                b += (M * K + K * N + M * N) * ss;
                mm = std::max(mm, (long long)M); mn = std::max(mn, (long long)N); mk = std::max(mk, (long long)K);
            }
            break;
        case ST_QR:
            for (int i = 0; i < s.count; ++i) {
                const QRTask& t = qr[s.first + i];
                f += (4.0 * t.m * (double)t.n * t.n - 4.0 / 3.0 * (double)t.n * t.n * t.n) * (cplx ? 4.0 : 1.0);
                b += 2.0 * t.m * (double)t.n * ss;
                mm = std::max(mm, (long long)t.m); mn = std::max(mn, (long long)t.n);
            }
            break;
        case ST_TC:
            for (int i = 0; i < s.count; ++i) {
                const TCTask& t = tcs[s.first + i];
                const TCSpec& sp = tcspec[s.first + i];
                const int esz = sp.kind == 0 ? 4 : 2, osz = t.out_kind == 2 ? 2 : t.out_kind == 3 ? 8 : 4;
                // split operands: three K-segments of MMA work over two planes of each operand;
                // a split result is written as two planes
                const int nseg = t.nseg == 3 ? 3 : 1, planes_in = nseg == 3 ? 2 : 1;
                const int parts = (t.x3 & 3 ? 2 : 1) + (t.C2 ? ((t.x3 >> 2) & 3 ? 2 : 1) : 0);
                f += 2.0 * (double)t.M * t.N * t.K * nseg;
                b += ((double)t.M * t.K + (double)t.N * t.K) * esz * planes_in + (double)t.M * t.N * osz * parts;
                mm = std::max(mm, (long long)t.M); mn = std::max(mn, (long long)t.N);
                mk = std::max(mk, (long long)t.K * nseg);
            }
            break;
        default:
            break;
    }
    if (flops) *flops = f;
    if (bytes) *bytes = b;
    if (max_m) *max_m = mm;
    if (max_n) *max_n = mn;
    if (max_k) *max_k = mk;
}

cudaError_t Program::launch_class(cudaStream_t st, const int* sweep_ctr, unsigned long long seed, int cls,
                                  long long* launches, double* flops, double* bytes) const {
    long long n = 0;
    double f = 0, b = 0;
    for (const Step& s : steps) {
        if (step_class(s.kind) != cls) continue;  // loop bodies count once: one fit sweep
        cudaError_t e = cudaSuccess;
        switch (s.kind) {
            case ST_GC:
                e = launch_gcontract(d_gc + s.first, s.count, s.aux, cplx, st, s.aux2, s.n);
                break;
            case ST_QR:
                e = launch_qr(d_qr + s.first, s.count, s.aux, s.n, cplx, st, s.aux2);
                break;
            case ST_TC:
                e = launch_tc_gemm(d_tcs + s.first, s.count, s.aux2 & 0xFF, s.aux, (int)s.n, (s.aux2 >> 8) & 0xFF, tc_err, st,
                                   (s.aux2 >> 16) & 0xFF);
                break;
            default:
                break;
        }
        if (e != cudaSuccess) return e;
        double sf = 0, sb = 0;
        step_work(s, &sf, &sb, nullptr, nullptr, nullptr);
        f += sf;
        b += sb;
        ++n;
    }
    if (launches) *launches = n;
    if (flops) *flops = f;
    if (bytes) *bytes = b;
    (void)sweep_ctr;
    (void)seed;
    return cudaSuccess;
}

void Program::free_all(cudaStream_t st) {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (void* p : {(void*)d_gc, (void*)d_qr, (void*)d_rnd, (void*)d_chk, (void*)d_scl, (void*)d_asm, (void*)d_nrm,
                    (void*)d_fus, (void*)d_dl, (void*)d_tcs, (void*)d_rel, (void*)d_dot})
        if (p) cudaFreeAsync(p, st);
    d_tcs = nullptr; d_rel = nullptr; d_dot = nullptr;
    d_gc = nullptr; d_qr = nullptr; d_rnd = nullptr; d_chk = nullptr;
    d_scl = nullptr; d_asm = nullptr; d_nrm = nullptr; d_fus = nullptr; d_dl = nullptr;
}

long long Program::kernel_count() const { return (long long)steps.size(); }

cudaError_t Program::executed(long long runs, long long* launches, double* flops, double* qr_flops,
                              long long* loop_iters) const {
    // steps outside loops run once per program run; a loop body runs `total` times
    long long n = 0;
    std::vector<int> totals(loop_ptr.size(), 0);
    for (size_t k = 0; k < loop_ptr.size(); ++k) {
        LoopDesc d{};
        cudaError_t e = cudaMemcpy(&d, loop_ptr[k], sizeof(d), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        totals[k] = d.total;
    }
    size_t loop = 0;
    for (size_t i = 0; i < steps.size(); ++i) {
        if (steps[i].kind == ST_LOOP_BEGIN) {
            const size_t end = loop_end(i);
            n += runs + (long long)(end - i - 1) * totals[loop++];
            i = end;
        } else {
            n += runs;
        }
    }
    long long body_runs = 0;
    for (int t : totals) body_runs += t;
    if (launches) *launches = n;
    if (loop_iters) *loop_iters = body_runs;
    // a fit's gated work is done in the fit sweeps it ran while active (its device counter);
    // the counters of the check tasks of one fit are the same word, read once
    double fl = runs * static_flops, qfl = runs * static_qr_flops;
    std::map<const int*, bool> seen;
    for (size_t i = 0; i < chk.size() && i < chk_keys.size(); ++i) {
        if (seen.count(chk[i].counter)) continue;
        seen[chk[i].counter] = true;
        int c = 0;
        cudaError_t e = cudaMemcpy(&c, chk[i].counter, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        auto a = fit_flops.find(chk_keys[i]);
        auto b = fit_qr_flops.find(chk_keys[i]);
        if (a != fit_flops.end()) fl += c * a->second;
        if (b != fit_qr_flops.end()) qfl += c * b->second;
    }
    if (flops) *flops = fl;
    if (qr_flops) *qr_flops = qfl;
    return cudaSuccess;
}

}  // namespace bbp
