// Tensor-core (TF32 / BF16) zip-up fit: the stages of App. A's fit with every
// contraction of Eq. (update) and of the A/B recurrences on the tcgen05 GEMM, FP32
// accumulation in TMEM, the QR/LQ truncation in FP32 (or FP64) arithmetic, and the
// normalisation and generator in FP64 exactly as on the FP64 path.
//
// Operand layouts (low precision, every row padded to 16 bytes; a split operand is two such
// planes, hi and lo, one plane apart):
//   X   : XL[x2][p][pad x]        XR[x][p][pad x2]
//   O   : OL[w2][q][pad(w p)]     OR[w][q][pad(p w2)]
//   env : ER[y][w][pad x]         EK[y][pad(w x)]      (A and B envs, both forms)
//   Y   : YS[y][pad(y2 q)]        YT[y2][pad(y q)]
//   L->R: T1[y][x2][pad(w p)]  T2a[y][q][pad(w2 x2)]  T2b[w2][x2][pad(y q)]
//   R->L: T1[y2][x][pad(p w2)] T2a[q][y2][pad(w x)]   T2b[w][x][pad(y2 q)]
// Row orders are chosen so that every destination of a GEMM is contiguous either
// along its columns (n2 stride 1) or along its rows (m2 stride 1), which the epilogue
// writes with vector stores.
// The site update is K2 (A X), K3 (T1 O), K4 (T2 B) in either direction, the env
// update K5 (conj(Y) T2); each GEMM's epilogue scatters its result straight into the
// layout(s) its consumers read, so no transpose kernel runs between them.
#include <algorithm>
#include <vector>

#include "engine.h"

namespace bbp {

// Row pitch of a K-major operand with K = x, padded to 16 bytes (a split operand has two
// planes of such rows, hi and lo).
long long padded(const MixCtx& cx, long long x) { return (x + cx.pe - 1) / cx.pe * cx.pe; }

void Program::tc_step(std::vector<TCTask>& ts, std::vector<TCSpec>& sp, int kind) {
    if (ts.empty()) return;
    int nmax = 1;
    for (auto& t : ts) nmax = std::max(nmax, t.N);
    const int bn = nmax <= 32 ? 32 : nmax <= 64 ? 64 : nmax <= 128 ? 128 : 256;
    int tiles = 1, kmax = 1;
    const int ek = kind == 0 ? 32 : 64;
    for (size_t i = 0; i < ts.size(); ++i) {
        sp[i].bn = bn;
        sp[i].kind = kind;
        tiles = std::max(tiles, ((ts[i].M + 127) / 128) * ((ts[i].N + bn - 1) / bn));
        kmax = std::max(kmax, (ts[i].K + ek - 1) / ek * (ts[i].nseg == 3 ? 3 : 1));
    }
    Step s;
    s.kind = ST_TC;
    s.first = tcs.size();
    s.count = (int)ts.size();
    s.aux = bn;
    s.aux2 = kind | (tc_default_stages(bn, kmax) << 8);  // kind, ring depth
    s.n = tiles;
    tcs.insert(tcs.end(), ts.begin(), ts.end());
    tcspec.insert(tcspec.end(), sp.begin(), sp.end());
    steps.push_back(s);
    ts.clear();
    sp.clear();
}

void Program::rel_step(std::vector<RelayoutTask>& ts) {
    if (ts.empty()) return;
    long long mx = 1;
    for (auto& t : ts) mx = std::max(mx, (long long)t.d[0] * t.d[1] * t.d[2] * t.d[3]);
    Step s;
    s.kind = ST_REL;
    s.first = rel.size();
    s.count = (int)ts.size();
    s.n = mx;
    rel.insert(rel.end(), ts.begin(), ts.end());
    steps.push_back(s);
    ts.clear();
}

namespace {

struct TB {  // tasks of one tensor-core step
    std::vector<TCTask> ts;
    std::vector<TCSpec> sp;
};

// A low-precision destination that is a split operand (hi and lo planes) of a later GEMM; the
// consumer decides the K-segment order (A: hi, lo, hi; B: hi, hi, lo), so either role reads the
// same two planes.  The argument is the consumer's K (documentation of the shape only).
constexpr int ROLE_A = 1, ROLE_B = 2;
struct Dst {
    int role = 0;
    long long kseg = 0;
};

// C = A B^T with A (a_rows x K, leading dim a_ld) and B (b_rows x K, b_ld), both K-major;
// result element (m, n), m = m1*M2 + m2, n = n1*N2 + n2, goes to C (and C2).  With split
// operands the GEMM runs three K-segments over the hi and lo planes of A and B.
void add(Program& pr, const MixCtx& cx, TB& tb, size_t a_off, long long a_rows, long long K, long long a_ld,
         size_t b_off, long long b_rows, long long b_ld, int M2, int N2, void* C, long long cm1, long long cm2,
         long long cn1, long long cn2, void* C2, long long dm1, long long dm2, long long dn1, long long dn2,
         int out_kind, const int* active, double alg_flops, Dst dc = Dst(), Dst dd = Dst()) {
    TCTask t{};
    t.M = (int)a_rows;
    t.N = (int)b_rows;
    t.K = (int)K;
    t.nseg = cx.x3 ? 3 : 1;
    if (cx.x3) {  // split destinations: hi plane, lo plane one plane further
        t.x3 = (dc.role ? 1 : 0) | ((dd.role ? 1 : 0) << 2);
        t.kseg = dc.role ? pr.plane_of((size_t)C) : 0;
        t.kseg2 = dd.role ? pr.plane_of((size_t)C2) : 0;
    }
    t.M2 = M2;
    t.N2 = N2;
    t.out_kind = out_kind;
    t.c_m1 = cm1; t.c_m2 = cm2; t.c_n1 = cn1; t.c_n2 = cn2;
    t.d_m1 = dm1; t.d_m2 = dm2; t.d_n1 = dn1; t.d_n2 = dn2;
    t.C = C;
    t.C2 = C2;
    t.active = active;
    t.alpha = 1.0f;
    TCSpec s;
    s.a_off = a_off; s.a_rows = a_rows; s.K = K; s.a_ld = a_ld;
    s.b_off = b_off; s.b_rows = b_rows; s.b_ld = b_ld;
    if (cx.x3) {
        s.a_pl = pr.plane_of(a_off);
        s.b_pl = pr.plane_of(b_off);
    }
    tb.ts.push_back(t);
    tb.sp.push_back(s);
    pr.count_flops(active, alg_flops, false);
}

// site dims of fit f at site i
struct Dims {
    long long y, y2, x, x2, w, w2, p, q;
};
Dims dims(const FitSpec& f, int i) {
    Dims d;
    d.y = f.ybond[i]; d.y2 = f.ybond[i + 1];
    d.x = f.X[i].a; d.x2 = f.X[i].b; d.p = f.X[i].k;
    d.w = f.O[i].w; d.w2 = f.O[i].w2; d.q = f.O[i].q;
    return d;
}

// ---- L->R site update: stage 0 K2, 1 K3, 2 K4, 3 K5
void lr(Program& pr, const MixCtx& cx, TB& tb, const FitSpec& f, int i, int stage, const int* act) {
    const Dims d = dims(f, i);
    const MixBufs& m = f.mx;
    const int lo = cx.tco;
    if (stage == 0) {  // T1[y][x2][pad(w p)] = sum_x ER_A[(y,w)][x] XL[(x2,p)][x]
        const long long WP = padded(cx, d.w * d.p);
        add(pr, cx, tb, m.AR[i], d.y * d.w, d.x, padded(cx, d.x), m.XL[i], d.x2 * d.p, padded(cx, d.x), (int)d.w, (int)d.p,
            P(m.T1), d.x2 * WP, d.p, WP, 1, nullptr, 0, 0, 0, 0, lo, act, 2.0 * d.y * d.w * d.x * d.p * d.x2,
            Dst{ROLE_A, d.w * d.p});
    } else if (stage == 1) {  // T2 = T1[(y,x2)][(w p)] OL[(w2,q)][(w p)]
        const long long WP = padded(cx, d.w * d.p), WX2 = padded(cx, d.w2 * d.x2), YQ = padded(cx, d.y * d.q);
        add(pr, cx, tb, m.T1, d.y * d.x2, d.w * d.p, WP, m.OL[i], d.w2 * d.q, WP, (int)d.x2, (int)d.q,
            P(m.T2a), d.q * WX2, 1, d.x2, WX2,                 // T2a[y][q][pad(w2 x2)]
            P(m.T2b), d.q, YQ, d.x2 * YQ, 1,                    // T2b[w2][x2][pad(y q)]
            lo, act, 2.0 * d.y * d.x2 * d.w * d.p * d.q * d.w2, Dst{ROLE_A, d.w2 * d.x2}, Dst{ROLE_B, d.y * d.q});
    } else if (stage == 2) {  // Yt[y][q][y2] = T2a[(y,q)][(w2 x2)] EK_B[y2][(w2 x2)]  (FP32)
        const long long WX2 = padded(cx, d.w2 * d.x2);
        add(pr, cx, tb, m.T2a, d.y * d.q, d.w2 * d.x2, WX2, m.BK[i + 1], d.y2, WX2, (int)d.q, (int)d.y2,
            P(m.Ytf), d.q * d.y2, d.y2, 0, 1, nullptr, 0, 0, 0, 0, 0, act, 2.0 * d.y * d.q * d.w2 * d.x2 * d.y2);
    } else {  // A_{i+1} = YT[y2][(y q)] T2b[(w2,x2)][(y q)] in both env forms
        const long long YQ = padded(cx, d.y * d.q), X2 = padded(cx, d.x2), WX2 = padded(cx, d.w2 * d.x2);
        add(pr, cx, tb, m.YT[i], d.y2, d.y * d.q, YQ, m.T2b, d.w2 * d.x2, YQ, (int)d.y2, (int)d.x2,
            P(m.AR[i + 1]), 0, d.w2 * X2, X2, 1,                // ER[y2][w2][pad x2]
            P(m.AK[i + 1]), 0, WX2, d.x2, 1,                    // EK[y2][pad(w2 x2)]
            lo, act, 2.0 * d.y2 * d.y * d.q * d.w2 * d.x2, Dst{ROLE_A, d.x2}, Dst{ROLE_A, d.w2 * d.x2});
    }
}

// ---- R->L site update: stage 0 K2r, 1 K3r, 2 K4r, 3 K5r; final != 0 writes Yt to FP64 Y[0]
void rl(Program& pr, const MixCtx& cx, TB& tb, const FitSpec& f, int i, int stage, const int* act, bool final_) {
    const Dims d = dims(f, i);
    const MixBufs& m = f.mx;
    const int lo = cx.tco;
    if (stage == 0) {  // T1[y2][x][pad(p w2)] = XR[(x,p)][x2] ER_B[(y2,w2)][x2]
        const long long PW = padded(cx, d.p * d.w2);
        add(pr, cx, tb, m.XR[i], d.x * d.p, d.x2, padded(cx, d.x2), m.BR[i + 1], d.y2 * d.w2, padded(cx, d.x2), (int)d.p,
            (int)d.w2, P(m.T1), PW, d.w2, d.x * PW, 1, nullptr, 0, 0, 0, 0, lo, act,
            2.0 * d.x * d.p * d.x2 * d.y2 * d.w2, Dst{ROLE_A, d.p * d.w2});
    } else if (stage == 1) {  // T2 = T1[(y2,x)][(p w2)] OR[(w,q)][(p w2)]
        const long long PW = padded(cx, d.p * d.w2), WX = padded(cx, d.w * d.x), QY2 = padded(cx, d.q * d.y2);
        add(pr, cx, tb, m.T1, d.y2 * d.x, d.p * d.w2, PW, m.OR[i], d.w * d.q, PW, (int)d.x, (int)d.q,
            P(m.T2a), WX, 1, d.x, d.y2 * WX,                    // T2a[q][y2][pad(w x)]
            P(m.T2b), d.q, QY2, d.x * QY2, 1,                   // T2b[w][x][pad(y2 q)]
            lo, act, 2.0 * d.x * d.y2 * d.p * d.w2 * d.w * d.q, Dst{ROLE_B, d.w * d.x}, Dst{ROLE_B, d.q * d.y2});
    } else if (stage == 2) {  // Yt[y][q][y2] = EK_A[y][(w x)] T2a[(q,y2)][(w x)]
        const long long WX = padded(cx, d.w * d.x);
        if (final_)
            add(pr, cx, tb, m.AK[i], d.y, d.w * d.x, WX, m.T2a, d.q * d.y2, WX, (int)d.y, (int)d.y2,
                P(f.Y[i] * (size_t)cx.ss), 0, d.q * d.y2, d.y2, 1, nullptr, 0, 0, 0, 0, 3, act,
                2.0 * d.y * d.w * d.x * d.q * d.y2);
        else
            add(pr, cx, tb, m.AK[i], d.y, d.w * d.x, WX, m.T2a, d.q * d.y2, WX, (int)d.y, (int)d.y2,
                P(m.Ytf), 0, d.q * d.y2, d.y2, 1, nullptr, 0, 0, 0, 0, 0, act, 2.0 * d.y * d.w * d.x * d.q * d.y2);
    } else {  // B_i = YS[y][(y2 q)] T2b[(w,x)][(y2 q)] in both env forms
        const long long QY2 = padded(cx, d.q * d.y2), X = padded(cx, d.x), WX = padded(cx, d.w * d.x);
        add(pr, cx, tb, m.YS[i], d.y, d.q * d.y2, QY2, m.T2b, d.w * d.x, QY2, (int)d.y, (int)d.x,
            P(m.BR[i]), 0, d.w * X, X, 1,                       // ER[y][w][pad x]
            P(m.BK[i]), 0, WX, d.x, 1,                          // EK[y][pad(w x)]
            lo, act, 2.0 * d.y * d.q * d.y2 * d.w * d.x, Dst{ROLE_B, d.x}, Dst{ROLE_B, d.w * d.x});
    }
}

QRTask qr_mixed(const Program& pr, const MixCtx& cx, const FitSpec& f, int i, bool lq, size_t loss_byte,
                const int* act) {
    const long long y = f.ybond[i], y2 = f.ybond[i + 1], q = f.O[i].q;
    QRTask t{};
    t.in = P(f.mx.Ytf);
    t.in_float = cx.qr_f32 ? 2 : 1;
    t.out = P(f.Y[i] * (size_t)cx.ss);
    t.work = P(f.qrw * (size_t)cx.ss);
    t.loss = (double*)P(loss_byte);
    t.active = act;
    t.out2_kind = cx.lpk;
    if (!lq) {
        t.m = (int)(y * q); t.n = (int)y2;
        t.in_rs = y2; t.in_cs = 1; t.out_rs = y2; t.out_cs = 1; t.conj_io = 0;
        t.out2 = P(f.mx.YT[i]);
        t.out2_M2 = 1; t.out2_rs = 1; t.out2_rs2 = 0; t.out2_cs = padded(cx, y * q);   // YT[y2][pad(y q)]
        t.out2_x3 = cx.x3 ? 1 : 0; t.out2_kseg = cx.x3 ? pr.plane_of(f.mx.YT[i]) : 0;
    } else {
        t.m = (int)(q * y2); t.n = (int)y;
        t.in_rs = 1; t.in_cs = q * y2; t.out_rs = 1; t.out_cs = q * y2; t.conj_io = 1;
        t.out2 = P(f.mx.YS[i]);
        // row i = (q, y2) of the LQ matrix goes to YS[y][pad(y2 q)]
        t.out2_M2 = (int)y2; t.out2_rs = 1; t.out2_rs2 = q; t.out2_cs = padded(cx, q * y2);
        t.out2_x3 = cx.x3 ? 1 : 0; t.out2_kseg = cx.x3 ? pr.plane_of(f.mx.YS[i]) : 0;
    }
    return t;
}

}  // namespace

void emit_fits_mixed(Program& pr, const MixCtx& cx, std::vector<FitSpec*>& fits, int max_sweeps, double fit_tol,
                     bool warm, bool rand_uses_sweep) {
    const int ss = cx.ss;
    int nmax = 0;
    for (auto* f : fits) nmax = std::max(nmax, f->n());
    // 1. random initial Y (canonical FP64), then its YS copy for the right environments
    {
        std::vector<RandTask> rt;
        for (auto* f : fits)
            for (int i = 0; i < f->n(); ++i) {
                RandTask t{};
                t.ptr = P(f->Y[i] * (size_t)ss);
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
        s.first = pr.rnd.size();
        pr.rnd.insert(pr.rnd.end(), rt.begin(), rt.end());
        s.aux = rand_uses_sweep ? 1 : 0;
        pr.steps.push_back(s);
        std::vector<RelayoutTask> rl_;
        for (auto* f : fits)
            for (int i = 1; i < f->n(); ++i) {
                const long long y = f->ybond[i], q = f->O[i].q, y2 = f->ybond[i + 1];
                RelayoutTask r{};
                r.src = P(f->Y[i] * (size_t)ss);
                r.dst = P(f->mx.YS[i]);
                r.d[0] = (int)y; r.d[1] = (int)q; r.d[2] = (int)y2; r.d[3] = 1;
                r.ss[0] = q * y2; r.ss[1] = y2; r.ss[2] = 1;
                r.ds[0] = padded(cx, q * y2); r.ds[1] = 1; r.ds[2] = q;  // YS[y][pad(y2 q)]
                r.x3 = cx.x3 ? 1 : 0;
                r.kseg = cx.x3 ? pr.plane_of(f->mx.YS[i]) : 0;
                r.src_kind = 0;
                r.dst_kind = cx.lpk;
                rl_.push_back(r);
            }
        pr.rel_step(rl_);
    }
    TB tb;
    // 2. right environments from the initial Y
    for (int k = 0; k <= nmax - 2; ++k)
        for (int stage : {0, 1, 3}) {
            for (auto* f : fits) {
                const int i = f->n() - 1 - k;
                if (i >= 1) rl(pr, cx, tb, *f, i, stage, nullptr, false);
            }
            pr.tc_step(tb.ts, tb.sp, cx.tck);
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
                    if (k <= f->n() - 2) lr(pr, cx, tb, *f, k, stage, (const int*)P(f->active));
                pr.tc_step(tb.ts, tb.sp, cx.tck);
            }
            for (auto* f : fits)
                if (k <= f->n() - 2) {
                    const int nu = 2 * (f->n() - 1);
                    qt.push_back(qr_mixed(pr, cx, *f, k, false, f->losses + (size_t)k * sizeof(double),
                                          (const int*)P(f->active)));
                }
            pr.qr_step(qt);
            for (auto* f : fits)
                if (k <= f->n() - 2) lr(pr, cx, tb, *f, k, 3, (const int*)P(f->active));
            pr.tc_step(tb.ts, tb.sp, cx.tck);
        }
        for (int k = 0; k <= nmax - 2; ++k) {
            for (int stage = 0; stage < 3; ++stage) {
                for (auto* f : fits) {
                    const int i = f->n() - 1 - k;
                    if (i >= 1) rl(pr, cx, tb, *f, i, stage, (const int*)P(f->active), false);
                }
                pr.tc_step(tb.ts, tb.sp, cx.tck);
            }
            for (auto* f : fits) {
                const int i = f->n() - 1 - k;
                if (i >= 1) {
                    const int nu = 2 * (f->n() - 1);
                    qt.push_back(qr_mixed(pr, cx, *f, i, true,
                                          f->losses + (size_t)((f->n() - 1) + k) * sizeof(double),
                                          (const int*)P(f->active)));
                }
            }
            pr.qr_step(qt);
            for (auto* f : fits) {
                const int i = f->n() - 1 - k;
                if (i >= 1) rl(pr, cx, tb, *f, i, 3, (const int*)P(f->active), false);
            }
            pr.tc_step(tb.ts, tb.sp, cx.tck);
        }
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
        st.first = pr.chk.size();
        pr.chk.insert(pr.chk.end(), ct.begin(), ct.end());
        pr.steps.push_back(st);
        pr.fit_tol = fit_tol;
        (void)s;
    }
    pr.simple(ST_LOOP_END, nullptr, nullptr, 0, 0);
    // 4. final update at site 0 (Yt kept, written in FP64)
    for (int stage = 0; stage < 3; ++stage) {
        for (auto* f : fits) rl(pr, cx, tb, *f, 0, stage, nullptr, true);
        pr.tc_step(tb.ts, tb.sp, cx.tck);
    }
    // 5. unit norm in FP64
    std::vector<ScaleTask> sc;
    for (auto* f : fits) {
        ScaleTask t{};
        t.ptr = P(f->Y[0] * (size_t)ss);
        t.n = (long long)f->ybond[0] * f->O[0].q * f->ybond[1];
        sc.push_back(t);
    }
    Step st;
    st.kind = ST_SCALE;
    st.count = (int)sc.size();
    st.first = pr.scl.size();
    pr.scl.insert(pr.scl.end(), sc.begin(), sc.end());
    pr.steps.push_back(st);
}

}  // namespace bbp
